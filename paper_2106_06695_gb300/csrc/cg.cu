// Batched conjugate gradients on (outputscale K~ + noise I) X = B (Sec. 2: Krylov
// solvers that need only MVMs; App. A: at most 500 iterations).
//
// Every right-hand side c is an independent CG with its own scalars; a column that has
// converged (||r_c|| / ||b_c|| <= tol), hit max_iter or broken down (<p, Ap> <= 0) is
// frozen by a device-side flag, so extra iterations leave it unchanged.  The iterate x and
// the residual r are kept in fp64 [n][k] (their recurrences are where fp32 rounding makes
// CG lose orthogonality); the search direction p and A p are fp32, the operands of the
// lattice MVM.  Dot products and norms are accumulated in fp64 per block (fixed column per
// thread, shared-memory tree) and the block partials are summed in a fixed order by one
// small kernel, so the result does not depend on scheduling.  One iteration is captured
// in a CUDA graph and replayed; the host reads the flags every check_every iterations.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sgp_internal.cuh"

namespace sgp {
namespace {

constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 4 * 152;

struct CgState {
  double* partial;  // [kDotBlocks][k]
  double* rho;      // <r, r> of the current residual
  double* pap;      // <p, A p>
  double* alpha;
  double* beta;
  double* bnorm;
  double* relres;
  int* active;
  int* iters;
};

// Column-fixed grid-stride mapping: blockDim = k * (kDotThreads / k) threads, so thread t
// always handles column t % k.
__device__ __forceinline__ void column_partial(double acc, int k, double* partial) {
  __shared__ double s[kDotThreads];
  s[threadIdx.x] = acc;
  __syncthreads();
  if ((int)threadIdx.x < k) {
    double t = 0.0;
    for (int j = threadIdx.x; j < (int)blockDim.x; j += k) t += s[j];
    partial[(int64_t)blockIdx.x * k + threadIdx.x] = t;
  }
}

// The solver's vectors live in the lattice's locality order: row p holds the caller's
// row perm[p], so the MVM's splat gathers and slice writes stay local.
__global__ void k_cg_init(const float* __restrict__ B, const int32_t* __restrict__ perm,
                          double* __restrict__ x, double* __restrict__ r, float* __restrict__ p,
                          int64_t n, int k, double* __restrict__ partial) {
  const int rows_per_block = blockDim.x / k;
  const int c = threadIdx.x % k;
  const int row0 = threadIdx.x / k;
  double acc = 0.0;
  if ((int)threadIdx.x < rows_per_block * k) {
    for (int64_t row = (int64_t)blockIdx.x * rows_per_block + row0; row < n;
         row += (int64_t)gridDim.x * rows_per_block) {
      const int64_t e = row * k + c;
      const float b = B[(int64_t)perm[row] * k + c];
      x[e] = 0.0;
      r[e] = (double)b;
      p[e] = b;
      acc += (double)b * (double)b;
    }
  }
  column_partial(acc, k, partial);
}

__global__ void k_cg_init_scalars(const double* __restrict__ partial, int nblk, int k,
                                  float tol, int max_iter, CgState S) {
  const int c = threadIdx.x;
  if (c >= k) return;
  double rr = 0.0;
  for (int b = 0; b < nblk; ++b) rr += partial[(int64_t)b * k + c];
  S.rho[c] = rr;
  S.bnorm[c] = sqrt(rr);
  S.iters[c] = 0;
  S.alpha[c] = 0.0;
  S.beta[c] = 0.0;
  if (rr == 0.0) {
    S.relres[c] = 0.0;
    S.active[c] = 0;
  } else {
    S.relres[c] = 1.0;
    S.active[c] = (1.0 > (double)tol && max_iter > 0) ? 1 : 0;
  }
}

__global__ void k_coldot(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                         int k, double* __restrict__ partial) {
  const int rows_per_block = blockDim.x / k;
  const int c = threadIdx.x % k;
  const int row0 = threadIdx.x / k;
  double acc = 0.0;
  if ((int)threadIdx.x < rows_per_block * k) {
    for (int64_t row = (int64_t)blockIdx.x * rows_per_block + row0; row < n;
         row += (int64_t)gridDim.x * rows_per_block) {
      const int64_t e = row * k + c;
      acc += (double)a[e] * (double)b[e];
    }
  }
  column_partial(acc, k, partial);
}

__global__ void k_cg_alpha(int nblk, int k, CgState S) {
  const int c = threadIdx.x;
  if (c >= k) return;
  double pap = 0.0;
  for (int b = 0; b < nblk; ++b) pap += S.partial[(int64_t)b * k + c];
  S.pap[c] = pap;
  double alpha = 0.0;
  if (S.active[c]) {
    if (pap > 0.0 && isfinite(pap)) {
      alpha = S.rho[c] / pap;
    } else {
      S.active[c] = 0;  // breakdown: the operator is not positive definite on p
    }
  }
  S.alpha[c] = alpha;
}

__global__ void k_cg_update_xr(double* __restrict__ x, double* __restrict__ r,
                               const float* __restrict__ p, const float* __restrict__ Ap,
                               int64_t n, int k, CgState S) {
  const int rows_per_block = blockDim.x / k;
  const int c = threadIdx.x % k;
  const int row0 = threadIdx.x / k;
  double acc = 0.0;
  if ((int)threadIdx.x < rows_per_block * k) {
    const bool on = S.active[c] != 0;
    const double a = S.alpha[c];
    for (int64_t row = (int64_t)blockIdx.x * rows_per_block + row0; row < n;
         row += (int64_t)gridDim.x * rows_per_block) {
      const int64_t e = row * k + c;
      double rv = r[e];
      if (on) {
        x[e] = fma(a, (double)p[e], x[e]);
        rv = fma(-a, (double)Ap[e], rv);
        r[e] = rv;
      }
      acc += rv * rv;
    }
  }
  column_partial(acc, k, S.partial);
}

__global__ void k_cg_beta(int nblk, int k, float tol, int max_iter, CgState S) {
  const int c = threadIdx.x;
  if (c >= k) return;
  if (!S.active[c]) return;
  double rr = 0.0;
  for (int b = 0; b < nblk; ++b) rr += S.partial[(int64_t)b * k + c];
  const int it = S.iters[c] + 1;
  S.iters[c] = it;
  const double rel = sqrt(rr) / S.bnorm[c];
  S.relres[c] = rel;
  if (rel <= (double)tol || it >= max_iter || !isfinite(rel)) {
    S.active[c] = 0;
    return;
  }
  S.beta[c] = rr / S.rho[c];
  S.rho[c] = rr;
}

__global__ void k_cg_update_p(float* __restrict__ p, const double* __restrict__ r, int64_t n,
                              int k, CgState S) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const int c = (int)(e % k);
  if (!S.active[c]) return;
  p[e] = (float)fma(S.beta[c], (double)p[e], r[e]);
}

__global__ void k_cg_store_x(const double* __restrict__ x, const int32_t* __restrict__ perm,
                             float* __restrict__ X, int64_t n, int k) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const int64_t row = e / k;
  X[(int64_t)perm[row] * k + (e - row * k)] = (float)x[e];
}

}  // namespace

sgp_status run_cg(Lattice* L, const float* B, int k, int blur, float noise, float tol,
                  int max_iter, float* X, int* iters, double* rel_res) {
  const int64_t n = L->n;
  // CUDA graphs cannot be captured on the legacy default stream: use a private blocking
  // stream then (it is ordered with the legacy stream like any blocking stream).
  cudaStream_t st = L->stream;
  cudaStream_t own = nullptr;
  if (st == nullptr) {
    cudaError_t e = cudaStreamCreateWithFlags(&own, cudaStreamDefault);
    if (e != cudaSuccess) return cuda_status(e, "creating the CG stream");
    st = own;
  }
  struct Cleanup {
    cudaStream_t st, own;
    std::vector<void*> ptrs;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    ~Cleanup() {
      if (exec) (void)cudaGraphExecDestroy(exec);
      if (graph) (void)cudaGraphDestroy(graph);
      for (void* p : ptrs) (void)cudaFreeAsync(p, st);
      if (own) {
        (void)cudaStreamSynchronize(own);
        (void)cudaStreamDestroy(own);
      }
      clear_pending_error();
    }
  } cl{st, own, {}};
  auto get = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) cl.ptrs.push_back(*p);
    return e;
  };
#define CG_CHECK(expr, what)                               \
  do {                                                     \
    cudaError_t e_ = (expr);                               \
    if (e_ != cudaSuccess) return cuda_status(e_, what);   \
  } while (0)

  double *x, *r;
  float *p, *Ap;
  CgState S{};
  CG_CHECK(get((void**)&x, n * k * sizeof(double)), "alloc x");
  CG_CHECK(get((void**)&r, n * k * sizeof(double)), "alloc r");
  CG_CHECK(get((void**)&p, n * k * sizeof(float)), "alloc p");
  CG_CHECK(get((void**)&Ap, n * k * sizeof(float)), "alloc Ap");
  CG_CHECK(get((void**)&S.partial, (size_t)kDotBlocks * k * sizeof(double)), "alloc partial");
  double* scal;
  CG_CHECK(get((void**)&scal, 6 * (size_t)k * sizeof(double)), "alloc scalars");
  S.rho = scal;
  S.pap = scal + k;
  S.alpha = scal + 2 * k;
  S.beta = scal + 3 * k;
  S.bnorm = scal + 4 * k;
  S.relres = scal + 5 * k;
  int* flags;
  CG_CHECK(get((void**)&flags, 2 * (size_t)k * sizeof(int)), "alloc flags");
  S.active = flags;
  S.iters = flags + k;
  sgp_status s = ensure_lattice_values(L, k, st);
  if (s != SGP_OK) return s;

  const int dot_threads = k * (kDotThreads / k);
  const int64_t rows_per_block = dot_threads / k;
  const int dot_blocks = (int)std::min<int64_t>(kDotBlocks, std::max<int64_t>(1, ceil_div(n, rows_per_block)));
  k_cg_init<<<dot_blocks, dot_threads, 0, st>>>(B, L->perm, x, r, p, n, k, S.partial);
  k_cg_init_scalars<<<1, kMaxK, 0, st>>>(S.partial, dot_blocks, k, tol, max_iter, S);
  note_launches(2);
  CG_CHECK(cudaGetLastError(), "CG init");

  cudaEvent_t* ev = L->profile ? L->prof_ev : nullptr;
  int passes = 0;
  auto iteration = [&]() {
    passes = enqueue_mvm(L, p, k, blur, L->outputscale, noise, Ap, st, ev, /*internal=*/true);
    k_coldot<<<dot_blocks, dot_threads, 0, st>>>(p, Ap, n, k, S.partial);
    k_cg_alpha<<<1, kMaxK, 0, st>>>(dot_blocks, k, S);
    k_cg_update_xr<<<dot_blocks, dot_threads, 0, st>>>(x, r, p, Ap, n, k, S);
    k_cg_beta<<<1, kMaxK, 0, st>>>(dot_blocks, k, tol, max_iter, S);
    k_cg_update_p<<<(unsigned)ceil_div(n * k, 256), 256, 0, st>>>(p, r, n, k, S);
    note_launches(5);
  };

  std::vector<int> hact(k);
  const int every = std::max(1, L->check_every);
  if (max_iter > 0) {
    // the captured launches run only when the graph is replayed: count them per replay
    const int64_t before = launches_so_far();
    CG_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    iteration();
    CG_CHECK(cudaStreamEndCapture(st, &cl.graph), "end capture");
    const int64_t per_iteration = launches_so_far() - before;
    note_launches(-per_iteration);
    CG_CHECK(cudaGraphInstantiate(&cl.exec, cl.graph, 0), "instantiate CG graph");
    CG_CHECK(cudaMemcpyAsync(hact.data(), S.active, k * sizeof(int), cudaMemcpyDeviceToHost, st),
             "read flags");
    CG_CHECK(cudaStreamSynchronize(st), "sync CG");
    int launched = 0;
    while (launched < max_iter && std::any_of(hact.begin(), hact.end(), [](int a) { return a; })) {
      const int batch = std::min(every, max_iter - launched);
      for (int b = 0; b < batch; ++b) CG_CHECK(cudaGraphLaunch(cl.exec, st), "launch CG graph");
      note_launches(per_iteration * batch);
      launched += batch;
      CG_CHECK(cudaMemcpyAsync(hact.data(), S.active, k * sizeof(int), cudaMemcpyDeviceToHost, st),
               "read flags");
      CG_CHECK(cudaStreamSynchronize(st), "sync CG");
      if (ev) {  // the events of the last replay bracket one MVM's blur passes
        float ms = 0.f;
        CG_CHECK(cudaEventElapsedTime(&ms, ev[0], ev[1]), "reading the blur timing events");
        L->prof_ms += ms;
        L->prof_passes += passes;
      }
    }
  }
  k_cg_store_x<<<(unsigned)ceil_div(n * k, 256), 256, 0, st>>>(x, L->perm, X, n, k);
  note_launches(1);
  CG_CHECK(cudaGetLastError(), "CG result");
  std::vector<double> hrel(k);
  std::vector<int> hit(k);
  CG_CHECK(cudaMemcpyAsync(hrel.data(), S.relres, k * sizeof(double), cudaMemcpyDeviceToHost, st),
           "read residuals");
  CG_CHECK(cudaMemcpyAsync(hit.data(), S.iters, k * sizeof(int), cudaMemcpyDeviceToHost, st),
           "read iterations");
  CG_CHECK(cudaStreamSynchronize(st), "sync CG");
  if (iters) std::copy(hit.begin(), hit.end(), iters);
  if (rel_res) std::copy(hrel.begin(), hrel.end(), rel_res);
  return SGP_OK;
#undef CG_CHECK
}

}  // namespace sgp
