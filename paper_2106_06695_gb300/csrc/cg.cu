// Batched conjugate gradients on (outputscale K~ + noise I) X = B (Sec. 2: Krylov
// solvers that need only MVMs; App. A: at most 500 iterations).
//
// Every right-hand side c is an independent CG with its own scalars; a column that has
// converged (||r_c|| / ||b_c|| <= tol), hit max_iter or broken down (<p, Ap> <= 0) is
// frozen by a device-side flag, so extra iterations leave it unchanged.  The iterate x and
// the residual r (whose recurrences are where fp32 rounding makes CG lose orthogonality)
// carry ~48 bits as double-float pairs (hi + lo fp32, updated with error-free
// transformations: FP64 arithmetic is slow on this part); the search direction p and A p
// are fp32, the operands of the lattice MVM.  Dot products are accumulated per thread in
// double-float, per block and across blocks in fp64 in a fixed order (fixed column per
// thread, shared-memory tree), so the result does not depend on scheduling.  One iteration is captured
// in a CUDA graph and replayed; the host reads the flags every check_every iterations.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sgp_internal.cuh"
#include "values.cuh"

namespace sgp {
namespace {

struct CgState {
  double* partial;  // [blocks][k] per-block column sums
  double* rho;      // <r, r> of the current residual
  double* pap;      // <p, A p>
  double* alpha;
  double* beta;
  double* bnorm;
  double* relres;
  int* active;
  int* iters;
  // optional Lanczos record (plain CG): alpha_j, beta_j of column c at [j][k], j < hcap
  double* ha;
  double* hb;
  int hcap;
  // optional residual history: ||r_c|| / ||b_c|| after iteration j of column c at [j][k]
  double* hist;
  int hist_cap;
  // optional: the preconditioner's split residual [n][64] (bf16; part p of column c < 16
  // at 16 p + c), written by the x, r update
  bf16* r3;
};

// VEC consecutive elements of a row: fp32 (one float4 when VEC = 4) and fp64 (two double2).
template <int VEC>
__device__ __forceinline__ void ldf(const float* p, float (&v)[VEC]) {
  if (VEC == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[VEC - 1] = t.w;
  } else {
    v[0] = *p;
  }
}
template <int VEC>
__device__ __forceinline__ void stf(float* p, const float (&v)[VEC]) {
  if (VEC == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[VEC - 1]);
  else *p = v[0];
}
// Grid-stride over rows with a fixed column group per thread: G = k / VEC threads per row,
// blockDim.x = a whole number of rows.
#define SGP_ROWS_LOOP(row)                                                                  \
  const int G = k / VEC;                                                                    \
  const int rows_per_block = blockDim.x / G;                                                \
  const int c0 = (int)(threadIdx.x % G) * VEC;                                              \
  for (int64_t row = (int64_t)blockIdx.x * rows_per_block + threadIdx.x / G; row < n;       \
       row += (int64_t)gridDim.x * rows_per_block)

// The solver's vectors live in the lattice's locality order: row p holds the caller's
// row perm[p], so the MVM's splat gathers and slice writes stay local.  B and X are the
// caller's buffers (any alignment): read and written element by element.
// The caller's B has kb <= k columns; columns kb .. k - 1 of the solver's vectors are zero
// right-hand sides (inactive from the start).
template <int VEC>
__global__ void k_cg_init(const float* __restrict__ B, int kb, const int32_t* __restrict__ perm,
                          float* __restrict__ xh, float* __restrict__ xl,
                          float* __restrict__ rh, float* __restrict__ rl, float* __restrict__ p,
                          int64_t n, int k, double* __restrict__ partial) {
  dfloat acc[VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) acc[j] = {0.f, 0.f};
  SGP_ROWS_LOOP(row) {
    const float* b = B + (int64_t)perm[row] * kb + c0;
    float bv[VEC], zero[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      bv[j] = c0 + j < kb ? b[j] : 0.f;
      zero[j] = 0.f;
      acc[j] = df_add(acc[j], df_two_prod(bv[j], bv[j]));
    }
    const int64_t e = row * k + c0;
    stf<VEC>(xh + e, zero);
    stf<VEC>(xl + e, zero);
    stf<VEC>(rh + e, bv);
    stf<VEC>(rl + e, zero);
    stf<VEC>(p + e, bv);
  }
  double dd[VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) dd[j] = df_to_double(acc[j]);
  block_column_sums<VEC>(dd, k, partial + (int64_t)blockIdx.x * k);
}

// Column c's sum over `nblk` block partials, in a fixed order (strided per thread, then a
// shared-memory tree); blockIdx.x = c, blockDim.x = 256.
__device__ __forceinline__ double column_total(const double* __restrict__ partial, int nblk, int k) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  double t = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) t += partial[(int64_t)b * k + c];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int half = blockDim.x / 2; half >= 1; half /= 2) {
    if ((int)threadIdx.x < half) red[threadIdx.x] += red[threadIdx.x + half];
    __syncthreads();
  }
  return red[0];
}

__global__ void k_cg_init_scalars(const double* __restrict__ partial, int nblk, int k,
                                  float tol, int max_iter, CgState S) {
  const double rr = column_total(partial, nblk, k);
  if (threadIdx.x != 0) return;
  const int c = blockIdx.x;
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

// <p, A p> from the slice's block partials, then alpha = rho / <p, A p>.
__global__ void k_cg_alpha(int nblk, int k, CgState S) {
  const double pap = column_total(S.partial, nblk, k);
  if (threadIdx.x != 0) return;
  const int c = blockIdx.x;
  S.pap[c] = pap;
  double alpha = 0.0;
  if (S.active[c]) {
    if (pap > 0.0 && isfinite(pap)) {
      alpha = S.rho[c] / pap;
      if (S.ha && S.iters[c] < S.hcap) S.ha[(int64_t)S.iters[c] * k + c] = alpha;
    } else {
      S.active[c] = 0;  // breakdown: the operator is not positive definite on p
    }
  }
  S.alpha[c] = alpha;
}

// x += alpha p, r -= alpha A p on active columns (double-float); block partials of <r, r>.
// With S.r3 (VEC = 4), also the three bf16 parts of r = rh + rl for columns 0..15, the
// operand of the preconditioner's B^T r (as its split kernel would write them).
template <int VEC>
__global__ void k_cg_update_xr(float* __restrict__ xh, float* __restrict__ xl,
                               float* __restrict__ rh, float* __restrict__ rl,
                               const float* __restrict__ p, const float* __restrict__ Ap,
                               int64_t n, int k, CgState S) {
  dfloat acc[VEC], a[VEC], na[VEC];
  bool on[VEC];
  {
    const int c = (int)(threadIdx.x % (k / VEC)) * VEC;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      acc[j] = {0.f, 0.f};
      on[j] = S.active[c + j] != 0;
      a[j] = df_from_double(S.alpha[c + j]);
      na[j] = {-a[j].hi, -a[j].lo};
    }
  }
  SGP_ROWS_LOOP(row) {
    const int64_t e = row * k + c0;
    float pv[VEC], qv[VEC], xhv[VEC], xlv[VEC], rhv[VEC], rlv[VEC];
    ldf<VEC>(p + e, pv);
    ldf<VEC>(Ap + e, qv);
    ldf<VEC>(xh + e, xhv);
    ldf<VEC>(xl + e, xlv);
    ldf<VEC>(rh + e, rhv);
    ldf<VEC>(rl + e, rlv);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      if (on[j]) {
        const dfloat x = df_add({xhv[j], xlv[j]}, df_mul_f(a[j], pv[j]));
        const dfloat r = df_add({rhv[j], rlv[j]}, df_mul_f(na[j], qv[j]));
        xhv[j] = x.hi, xlv[j] = x.lo, rhv[j] = r.hi, rlv[j] = r.lo;
      }
      dfloat sq = df_two_prod(rhv[j], rhv[j]);
      sq = df_fast_two_sum(sq.hi, __fmaf_rn(2.f * rhv[j], rlv[j], sq.lo));
      acc[j] = df_add(acc[j], sq);
    }
    stf<VEC>(xh + e, xhv);
    stf<VEC>(xl + e, xlv);
    stf<VEC>(rh + e, rhv);
    stf<VEC>(rl + e, rlv);
    if constexpr (VEC == 4) {
      if (S.r3 && c0 < 16) {
        bf16 q[4][3];
#pragma unroll
        for (int j = 0; j < 4; ++j) split3(__fadd_rn(rhv[j], rlv[j]), q[j][0], q[j][1], q[j][2]);
#pragma unroll
        for (int part = 0; part < 3; ++part) {
          uint2 w;
          w.x = (uint32_t)__bfloat16_as_ushort(q[0][part]) |
                ((uint32_t)__bfloat16_as_ushort(q[1][part]) << 16);
          w.y = (uint32_t)__bfloat16_as_ushort(q[2][part]) |
                ((uint32_t)__bfloat16_as_ushort(q[3][part]) << 16);
          *reinterpret_cast<uint2*>(S.r3 + row * 64 + part * 16 + c0) = w;
        }
      }
    }
  }
  double dd[VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) dd[j] = df_to_double(acc[j]);
  block_column_sums<VEC>(dd, k, S.partial + (int64_t)blockIdx.x * k);
}

__global__ void k_cg_beta(int nblk, int k, float tol, int max_iter, CgState S) {
  const double rr = column_total(S.partial, nblk, k);
  if (threadIdx.x != 0) return;
  const int c = blockIdx.x;
  if (!S.active[c]) return;
  const int it = S.iters[c] + 1;
  S.iters[c] = it;
  const double rel = sqrt(rr) / S.bnorm[c];
  S.relres[c] = rel;
  if (S.hist && it <= S.hist_cap) S.hist[(int64_t)(it - 1) * k + c] = rel;
  if (rel <= (double)tol || it >= max_iter || !isfinite(rel)) {
    S.active[c] = 0;
    return;
  }
  S.beta[c] = rr / S.rho[c];
  S.rho[c] = rr;
  if (S.hb && it - 1 < S.hcap) S.hb[(int64_t)(it - 1) * k + c] = S.beta[c];
}

// Preconditioned CG: convergence check on <r, r> (no beta yet).
__global__ void k_cg_check(int nblk, int k, float tol, int max_iter, CgState S) {
  const double rr = column_total(S.partial, nblk, k);
  if (threadIdx.x != 0) return;
  const int c = blockIdx.x;
  if (!S.active[c]) return;
  const int it = S.iters[c] + 1;
  S.iters[c] = it;
  const double rel = sqrt(rr) / S.bnorm[c];
  S.relres[c] = rel;
  if (S.hist && it <= S.hist_cap) S.hist[(int64_t)(it - 1) * k + c] = rel;
  if (rel <= (double)tol || it >= max_iter || !isfinite(rel)) S.active[c] = 0;
}

// Preconditioned CG: rho = <r, z> at the start.
__global__ void k_cg_rho_init(int nblk, int k, CgState S) {
  const double rz = column_total(S.partial, nblk, k);
  if (threadIdx.x != 0) return;
  const int c = blockIdx.x;
  S.rho[c] = rz;
  if (!(rz > 0.0) || !isfinite(rz)) S.active[c] = 0;
}

// Preconditioned CG: beta = <r, z>_new / <r, z>_old on active columns.
__global__ void k_cg_beta_pcg(int nblk, int k, CgState S) {
  const double rz = column_total(S.partial, nblk, k);
  if (threadIdx.x != 0) return;
  const int c = blockIdx.x;
  if (!S.active[c]) return;
  if (!(rz > 0.0) || !isfinite(rz)) {
    S.active[c] = 0;
    return;
  }
  S.beta[c] = rz / S.rho[c];
  S.rho[c] = rz;
}

// Preconditioned CG: p = z + beta p on active columns (first == true: p = z).
template <int VEC, bool FIRST>
__global__ void k_cg_update_p_z(float* __restrict__ p, const float* __restrict__ z, int64_t n,
                                int k, CgState S) {
  dfloat b[VEC];
  bool on[VEC];
  {
    const int c = (int)(threadIdx.x % (k / VEC)) * VEC;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      on[j] = S.active[c + j] != 0;
      b[j] = df_from_double(S.beta[c + j]);
    }
  }
  SGP_ROWS_LOOP(row) {
    const int64_t e = row * k + c0;
    float pv[VEC], zv[VEC];
    ldf<VEC>(p + e, pv);
    ldf<VEC>(z + e, zv);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      if (FIRST) {
        pv[j] = zv[j];
      } else if (on[j]) {
        const dfloat t = df_add(df_mul_f(b[j], pv[j]), {zv[j], 0.f});
        pv[j] = __fadd_rn(t.hi, t.lo);
      }
    }
    stf<VEC>(p + e, pv);
  }
}

// p = r + beta p on active columns (double-float sum, rounded to fp32).
template <int VEC>
__global__ void k_cg_update_p(float* __restrict__ p, const float* __restrict__ rh,
                              const float* __restrict__ rl, int64_t n, int k, CgState S) {
  dfloat b[VEC];
  bool on[VEC];
  {
    const int c = (int)(threadIdx.x % (k / VEC)) * VEC;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      on[j] = S.active[c + j] != 0;
      b[j] = df_from_double(S.beta[c + j]);
    }
  }
  SGP_ROWS_LOOP(row) {
    const int64_t e = row * k + c0;
    float pv[VEC], rhv[VEC], rlv[VEC];
    ldf<VEC>(p + e, pv);
    ldf<VEC>(rh + e, rhv);
    ldf<VEC>(rl + e, rlv);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      if (on[j]) {
        const dfloat t = df_add({rhv[j], rlv[j]}, df_mul_f(b[j], pv[j]));
        pv[j] = __fadd_rn(t.hi, t.lo);
      }
    }
    stf<VEC>(p + e, pv);
  }
}

template <int VEC>
__global__ void k_cg_store_x(const float* __restrict__ xh, const float* __restrict__ xl,
                             const int32_t* __restrict__ perm, float* __restrict__ X, int kb,
                             int64_t n, int k) {
  SGP_ROWS_LOOP(row) {
    float hv[VEC], lv[VEC];
    ldf<VEC>(xh + row * k + c0, hv);
    ldf<VEC>(xl + row * k + c0, lv);
    float* dst = X + (int64_t)perm[row] * kb + c0;
#pragma unroll
    for (int j = 0; j < VEC; ++j)
      if (c0 + j < kb) dst[j] = __fadd_rn(hv[j], lv[j]);
  }
}

}  // namespace

sgp_status run_cg(Lattice* L, const float* B, int k, int blur, float noise, float tol,
                  int max_iter, float* X, int* iters, double* rel_res, int precond_rank,
                  uint64_t seed, const LanczosRecord* rec, double* history) {
  const int64_t n = L->n;
  // The solver works on k rounded up to a multiple of 4 (zero right-hand sides in the
  // extra columns, inactive from the start), so that its vectors and the lattice values
  // are rows of float4 and the MVM takes its vectorised kernels.  The Lanczos record of
  // sgp_logdet is laid out for the caller's k: no padding then.
  const int kb = k;
  if (!rec) k = (k + 3) / 4 * 4;
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
    ShiftedNystrom pre;
    ~Cleanup() {
      pre.release(st);
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
    cudaError_t e = dev_malloc(p, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) cl.ptrs.push_back(*p);
    return e;
  };
#define CG_CHECK(expr, what)                               \
  do {                                                     \
    cudaError_t e_ = (expr);                               \
    if (e_ != cudaSuccess) return cuda_status(e_, what);   \
  } while (0)

  float *xh, *xl, *rh, *rl, *p, *Ap;
  CgState S{};
  const int vec = k % 4 == 0 ? 4 : 1;
  const int T = column_block_threads(k, vec);
  const int64_t rows_per_block = T / (k / vec);
  const int vblocks = (int)std::min<int64_t>(kVecBlocks, std::max<int64_t>(1, ceil_div(n, rows_per_block)));
  const int64_t sblocks = slice_dot_blocks(L, k);
  const bool want_pre = precond_rank > 0 && noise > 0.f && !rec;
  // bounds ShiftedNystrom::dot_blocks (its z blocks: at most one per 128-row tile)
  const int64_t pblocks = want_pre ? ceil_div(n, 128) : 0;
  CG_CHECK(get((void**)&xh, n * k * sizeof(float)), "alloc x");
  CG_CHECK(get((void**)&xl, n * k * sizeof(float)), "alloc x");
  CG_CHECK(get((void**)&rh, n * k * sizeof(float)), "alloc r");
  CG_CHECK(get((void**)&rl, n * k * sizeof(float)), "alloc r");
  CG_CHECK(get((void**)&p, n * k * sizeof(float)), "alloc p");
  CG_CHECK(get((void**)&Ap, n * k * sizeof(float)), "alloc Ap");
  CG_CHECK(get((void**)&S.partial,
               (size_t)std::max<int64_t>(std::max<int64_t>(vblocks, sblocks), pblocks) * k *
                   sizeof(double)),
           "alloc partial");
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
  if (rec) {
    S.ha = rec->alpha;
    S.hb = rec->beta;
    S.hcap = rec->cap;
  }
  if (history && max_iter > 0) {
    CG_CHECK(get((void**)&S.hist, (size_t)max_iter * k * sizeof(double)), "alloc history");
    S.hist_cap = max_iter;
    // iterations a column does not run read back as NaN
    std::vector<double> nan((size_t)max_iter * k, std::nan(""));
    CG_CHECK(cudaMemcpyAsync(S.hist, nan.data(), nan.size() * sizeof(double),
                             cudaMemcpyHostToDevice, st),
             "clear history");
    CG_CHECK(cudaStreamSynchronize(st), "sync history");
  }
  sgp_status s = ensure_lattice_values(L, k, st);
  if (s != SGP_OK) return s;

  // the preconditioner (built before anything is captured); needs noise > 0
  bool use_pre = false;
  float* z = nullptr;
  if (want_pre) {
    s = cl.pre.build(L, precond_rank, seed, noise, blur, L->precond_power_iters, st);
    if (s != SGP_OK) return s;
    use_pre = cl.pre.ok;
    if (use_pre) CG_CHECK(get((void**)&z, n * k * sizeof(float)), "alloc z");
    // the x, r update writes the split residual the preconditioner's B^T r reads
    if (use_pre && vec == 4) S.r3 = static_cast<bf16*>(cl.pre.r3);
  }

  if (vec == 4)
    k_cg_init<4><<<vblocks, T, 0, st>>>(B, kb, L->perm, xh, xl, rh, rl, p, n, k, S.partial);
  else
    k_cg_init<1><<<vblocks, T, 0, st>>>(B, kb, L->perm, xh, xl, rh, rl, p, n, k, S.partial);
  k_cg_init_scalars<<<k, 256, 0, st>>>(S.partial, vblocks, k, tol, max_iter, S);
  note_launches(2);
  if (use_pre) {  // z = P^-1 r, rho = <r, z>, p = z
    cl.pre.apply(rh, rl, k, z, S.partial, st);
    k_cg_rho_init<<<k, 256, 0, st>>>((int)cl.pre.dot_blocks(), k, S);
    if (vec == 4) k_cg_update_p_z<4, true><<<vblocks, T, 0, st>>>(p, z, n, k, S);
    else k_cg_update_p_z<1, true><<<vblocks, T, 0, st>>>(p, z, n, k, S);
    note_launches(2);
  }
  CG_CHECK(cudaGetLastError(), "CG init");

  cudaEvent_t* ev = L->profile ? L->prof_ev : nullptr;
  int passes = 0;
  auto iteration = [&]() {
    // Ap = outputscale K~ p + noise p, with the slice also summing <p, Ap> per block
    passes = enqueue_mvm(L, p, k, blur, L->outputscale, noise, Ap, st, ev, /*internal=*/true,
                         S.partial);
    k_cg_alpha<<<k, 256, 0, st>>>((int)sblocks, k, S);
    if (vec == 4) k_cg_update_xr<4><<<vblocks, T, 0, st>>>(xh, xl, rh, rl, p, Ap, n, k, S);
    else k_cg_update_xr<1><<<vblocks, T, 0, st>>>(xh, xl, rh, rl, p, Ap, n, k, S);
    if (use_pre) {
      k_cg_check<<<k, 256, 0, st>>>(vblocks, k, tol, max_iter, S);
      cl.pre.apply(rh, rl, k, z, S.partial, st, ev ? ev + 4 : nullptr, S.r3 != nullptr);
      k_cg_beta_pcg<<<k, 256, 0, st>>>((int)cl.pre.dot_blocks(), k, S);
      if (vec == 4) k_cg_update_p_z<4, false><<<vblocks, T, 0, st>>>(p, z, n, k, S);
      else k_cg_update_p_z<1, false><<<vblocks, T, 0, st>>>(p, z, n, k, S);
      note_launches(5);
    } else {
      k_cg_beta<<<k, 256, 0, st>>>(vblocks, k, tol, max_iter, S);
      if (vec == 4) k_cg_update_p<4><<<vblocks, T, 0, st>>>(p, rh, rl, n, k, S);
      else k_cg_update_p<1><<<vblocks, T, 0, st>>>(p, rh, rl, n, k, S);
      note_launches(4);
    }
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
      if (ev) {  // the events of the last replay bracket one MVM's splat, blur and slice
        float ms[kProfStages] = {};
        const int from[kProfStages] = {2, 0, 1, 4, 6}, to[kProfStages] = {0, 1, 3, 5, 7};
        for (int q = 0; q < (use_pre ? kProfStages : 3); ++q)
          CG_CHECK(cudaEventElapsedTime(&ms[q], ev[from[q]], ev[to[q]]),
                   "reading the stage timing events");
        L->prof_ms += ms[1];
        L->prof_passes += passes;
        for (int q = 0; q < kProfStages; ++q) L->prof_stage_ms[q] += ms[q];
        L->prof_mvms += 1;
      }
    }
  }
  if (vec == 4) k_cg_store_x<4><<<vblocks, T, 0, st>>>(xh, xl, L->perm, X, kb, n, k);
  else k_cg_store_x<1><<<vblocks, T, 0, st>>>(xh, xl, L->perm, X, kb, n, k);
  note_launches(1);
  CG_CHECK(cudaGetLastError(), "CG result");
  std::vector<double> hrel(k);
  std::vector<int> hit(k);
  CG_CHECK(cudaMemcpyAsync(hrel.data(), S.relres, k * sizeof(double), cudaMemcpyDeviceToHost, st),
           "read residuals");
  CG_CHECK(cudaMemcpyAsync(hit.data(), S.iters, k * sizeof(int), cudaMemcpyDeviceToHost, st),
           "read iterations");
  CG_CHECK(cudaStreamSynchronize(st), "sync CG");
  if (use_pre && (s = cl.pre.check(st)) != SGP_OK) return s;
  if (iters) std::copy(hit.begin(), hit.begin() + kb, iters);
  if (rel_res) std::copy(hrel.begin(), hrel.begin() + kb, rel_res);
  if (S.hist) {  // [max_iter][k] on the device, the caller's [max_iter][kb] on the host
    std::vector<double> h((size_t)max_iter * k);
    CG_CHECK(cudaMemcpyAsync(h.data(), S.hist, h.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, st),
             "read history");
    CG_CHECK(cudaStreamSynchronize(st), "sync CG");
    for (int j = 0; j < max_iter; ++j)
      std::copy(h.begin() + (size_t)j * k, h.begin() + (size_t)j * k + kb,
                history + (size_t)j * kb);
  }
  if (rec) {  // ||b_c|| and the iteration counts stay on the device for the quadrature
    CG_CHECK(cudaMemcpyAsync(rec->bnorm, S.bnorm, k * sizeof(double), cudaMemcpyDeviceToDevice,
                             st),
             "copy norms");
    CG_CHECK(cudaMemcpyAsync(rec->iters, S.iters, k * sizeof(int), cudaMemcpyDeviceToDevice, st),
             "copy iterations");
    CG_CHECK(cudaStreamSynchronize(st), "sync CG");
  }
  return SGP_OK;
#undef CG_CHECK
}

}  // namespace sgp
