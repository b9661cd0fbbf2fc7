// Rank-l preconditioner for the CG solve (App. A: CG pre-conditioner of rank 100).
//
// The lattice operator A = outputscale W M^T M W^T has no cheap entries or diagonal, so
// the low-rank part is a randomized Nystrom approximation built from products with A
// only:
//   Omega  n x l Rademacher sketch, entry (i, j) = sign bit of SplitMix64(seed, i l + j)
//          for the caller's point i (counter-based: anyone can regenerate it);
//   Y      = A Omega + nu Omega                 (one l-column lattice MVM, small shift nu);
//   C      = Omega^T Y = R R^T                  (Cholesky, l x l, fp64);
//   B      = Y R^-T                             (so that B B^T = Y C^-1 Y^T);
//   P      = B B^T + noise I,
//   P^-1 r = (r - B (noise I + B^T B)^-1 B^T r) / noise       (Woodbury).
// P is symmetric positive definite for any computed B, so CG stays a CG whatever the
// rounding in B; the Cholesky factors of the l x l matrices are computed in fp64 by one
// block, the tall n x l products in fp32 with fixed-order partial sums (deterministic).
// All row-indexed arrays are in the lattice's locality order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sgp_internal.cuh"

namespace sgp {
namespace {

constexpr int kRowsPerStage = 32;  // rows staged in shared memory per step
constexpr int kTallBlocks = 2 * 152;

// SplitMix64 (Steele, Lea & Flood 2014) at counter c: one +-1 per (point, column).
__device__ __forceinline__ float rademacher(uint64_t seed, int64_t i, int j, int l) {
  uint64_t z = seed + ((uint64_t)(i * l + j) + 1ull) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (z >> 63) ? -1.f : 1.f;
}

__global__ void k_fill_sketch(const int32_t* __restrict__ perm, int64_t n, int l, uint64_t seed,
                              float* __restrict__ om) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * l) return;
  const int64_t p = e / l;
  om[e] = rademacher(seed, perm[p], (int)(e - p * l), l);
}

// Y += nu Omega (Omega regenerated).
__global__ void k_shift(const int32_t* __restrict__ perm, int64_t n, int l, uint64_t seed,
                        float nu, float* __restrict__ Y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * l) return;
  const int64_t p = e / l;
  Y[e] = fmaf(nu, rademacher(seed, perm[p], (int)(e - p * l), l), Y[e]);
}

// Per-block partial of L^T X over the block's rows, L = Omega (regenerated) when OMEGA,
// else L = X.  X: [n][l] fp32.  out: partial[block][l][l] (fp64 of fp32 block sums).
template <bool OMEGA>
__global__ void k_gram(const float* __restrict__ X, const int32_t* __restrict__ perm, int64_t n,
                       int l, uint64_t seed, double* __restrict__ partial) {
  extern __shared__ float sh[];
  float* xs = sh;                               // [kRowsPerStage][l]
  float* ls = sh + kRowsPerStage * l;           // [kRowsPerStage][l] (OMEGA only)
  const int outs = l * l;
  constexpr int kMaxOwn = 64;                   // l <= 128 -> l*l/256 <= 64
  float acc[kMaxOwn];
#pragma unroll
  for (int q = 0; q < kMaxOwn; ++q) acc[q] = 0.f;
  const int64_t rows_per_block = ceil_div(n, gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = std::min<int64_t>(n, r0 + rows_per_block);
  for (int64_t base = r0; base < r1; base += kRowsPerStage) {
    const int rows = (int)std::min<int64_t>(kRowsPerStage, r1 - base);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * l; e += blockDim.x) {
      const int rr = e / l, j = e - rr * l;
      xs[e] = X[(base + rr) * l + j];
      if (OMEGA) ls[e] = rademacher(seed, perm[base + rr], j, l);
    }
    __syncthreads();
    const float* L = OMEGA ? ls : xs;
#pragma unroll
    for (int q = 0; q < kMaxOwn; ++q) {
      const int o = threadIdx.x + q * blockDim.x;
      if (o < outs) {
        const int i = o / l, j = o - i * l;
        float a = acc[q];
        for (int rr = 0; rr < rows; ++rr) a = fmaf(L[rr * l + i], xs[rr * l + j], a);
        acc[q] = a;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kMaxOwn; ++q) {
    const int o = threadIdx.x + q * blockDim.x;
    if (o < outs) partial[(int64_t)blockIdx.x * outs + o] = (double)acc[q];
  }
}

// out[e] = sum over blocks of partial[b][e], in block order.
__global__ void k_sum_blocks(const double* __restrict__ partial, int nblk, int count,
                             double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t += partial[(int64_t)b * count + e];
  out[e] = t;
}

// In-place lower Cholesky of the l x l fp64 matrix A (+ shift on the diagonal), one block;
// the strict upper triangle is zeroed.  *status = 1 when a pivot is not positive.
__global__ void k_cholesky(double* __restrict__ A, int l, double shift, int* __restrict__ status) {
  __shared__ double piv;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e / l, j = e % l;
    if (i == j) A[e] += shift;
    if (j > i) A[e] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    if (threadIdx.x == 0) {
      const double d = A[j * l + j];
      if (!(d > 0.0) || !isfinite(d)) {
        *status = 1;
        piv = 1.0;
      } else {
        piv = sqrt(d);
      }
      A[j * l + j] = piv;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < l; i += blockDim.x) A[i * l + j] /= piv;
    __syncthreads();
    const int rem = l - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e / rem, c = j + 1 + e % rem;
      if (c <= i) A[i * l + c] -= A[i * l + j] * A[c * l + j];
    }
    __syncthreads();
  }
}

// T = (R^-1)^T for lower-triangular R (fp64), written as fp32 [l][l] (upper triangular):
// thread c solves R x = e_c by forward substitution.
__global__ void k_tri_inv_t(const double* __restrict__ R, int l, double* __restrict__ work,
                            float* __restrict__ T) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= l) return;
  double* x = work + (int64_t)c * l;
  for (int i = 0; i < l; ++i) {
    double s = (i == c) ? 1.0 : 0.0;
    for (int j = c; j < i; ++j) s -= R[i * l + j] * x[j];
    x[i] = (i < c) ? 0.0 : s / R[i * l + i];
  }
  for (int i = 0; i < l; ++i) T[c * l + i] = (float)x[i];  // T[c][i] = (R^-1)[i][c]
}

// In place, row by row: Y[row] <- Y[row] T  (T in shared memory).
__global__ void k_rows_times(float* __restrict__ Y, const float* __restrict__ T, int64_t n,
                             int l) {
  extern __shared__ float sh[];
  float* ts = sh;              // [l][l]
  float* ys = sh + l * l;      // [rows_per_block][l]
  const int rows = blockDim.x / l;  // blockDim.x = rows * l
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) ts[e] = T[e];
  const int rr = threadIdx.x / l, c = threadIdx.x - rr * l;
  for (int64_t base = (int64_t)blockIdx.x * rows; base < n; base += (int64_t)gridDim.x * rows) {
    __syncthreads();
    const int64_t row = base + rr;
    if (rr < rows && row < n) ys[rr * l + c] = Y[row * l + c];
    __syncthreads();
    if (rr < rows && row < n) {
      float a = 0.f;
      for (int j = 0; j < l; ++j) a = fmaf(ys[rr * l + j], ts[j * l + c], a);
      Y[row * l + c] = a;
    }
  }
}

// Per-block partial of B^T r (l x k) with r = rh + rl; blockIdx.y selects a range of
// kOutsPerBlock outputs, each thread owning up to kOwn of them.
constexpr int kOwn = 8;
constexpr int kOutsPerBlock = 256 * kOwn;
__global__ void k_bt_r(const float* __restrict__ Bm, const float* __restrict__ rh,
                       const float* __restrict__ rl, int64_t n, int l, int k,
                       double* __restrict__ partial) {
  extern __shared__ float sh[];
  float* bs = sh;                          // [kRowsPerStage][l]
  float* rs = sh + kRowsPerStage * l;      // [kRowsPerStage][k]
  const int outs = l * k;
  const int o0 = blockIdx.y * kOutsPerBlock;
  float acc[kOwn];
#pragma unroll
  for (int q = 0; q < kOwn; ++q) acc[q] = 0.f;
  const int64_t rows_per_block = ceil_div(n, gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = std::min<int64_t>(n, r0 + rows_per_block);
  for (int64_t base = r0; base < r1; base += kRowsPerStage) {
    const int rows = (int)std::min<int64_t>(kRowsPerStage, r1 - base);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * l; e += blockDim.x) bs[e] = Bm[base * l + e];
    for (int e = threadIdx.x; e < rows * k; e += blockDim.x)
      rs[e] = __fadd_rn(rh[base * k + e], rl[base * k + e]);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kOwn; ++q) {
      const int o = o0 + threadIdx.x + q * blockDim.x;
      if (o < outs) {
        const int j = o / k, c = o - j * k;
        float a = acc[q];
        for (int rr = 0; rr < rows; ++rr) a = fmaf(bs[rr * l + j], rs[rr * k + c], a);
        acc[q] = a;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kOwn; ++q) {
    const int o = o0 + threadIdx.x + q * blockDim.x;
    if (o < outs) partial[(int64_t)blockIdx.x * outs + o] = (double)acc[q];
  }
}

// u = (Q Q^T)^-1 t for each of the k columns (Q lower, fp64); one block, one thread per
// column.  u is written as fp32 [l][k].
__global__ void k_solve_qqt(const double* __restrict__ Q, const double* __restrict__ t, int l,
                            int k, double* __restrict__ work, float* __restrict__ u) {
  const int c = threadIdx.x;
  if (c >= k) return;
  double* y = work + (int64_t)c * l;
  for (int i = 0; i < l; ++i) {  // Q y = t
    double s = t[i * k + c];
    for (int j = 0; j < i; ++j) s -= Q[i * l + j] * y[j];
    y[i] = s / Q[i * l + i];
  }
  for (int i = l - 1; i >= 0; --i) {  // Q^T x = y
    double s = y[i];
    for (int j = i + 1; j < l; ++j) s -= Q[j * l + i] * y[j];
    y[i] = s / Q[i * l + i];
  }
  for (int i = 0; i < l; ++i) u[i * k + c] = (float)y[i];
}

// z = (r - B u) / noise per row (u in shared memory) and per-block column sums of r z.
template <int VEC>
__global__ void k_apply_z(const float* __restrict__ Bm, const float* __restrict__ u,
                          const float* __restrict__ rh, const float* __restrict__ rl,
                          float inv_noise, int64_t n, int l, int k, float* __restrict__ z,
                          double* __restrict__ partial) {
  extern __shared__ float us[];  // [l][k]
  for (int e = threadIdx.x; e < l * k; e += blockDim.x) us[e] = u[e];
  __syncthreads();
  const int G = k / VEC;
  const int rows_per_block = blockDim.x / G;
  const int c0 = (int)(threadIdx.x % G) * VEC;
  dfloat acc[VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) acc[j] = {0.f, 0.f};
  for (int64_t row = (int64_t)blockIdx.x * rows_per_block + threadIdx.x / G; row < n;
       row += (int64_t)gridDim.x * rows_per_block) {
    float s[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) s[j] = 0.f;
    const float* b = Bm + row * l;
    for (int q = 0; q < l; ++q) {
      const float bq = b[q];
#pragma unroll
      for (int j = 0; j < VEC; ++j) s[j] = fmaf(bq, us[q * k + c0 + j], s[j]);
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      const int64_t e = row * k + c0 + j;
      const float r = __fadd_rn(rh[e], rl[e]);
      const float zz = (r - s[j]) * inv_noise;
      z[e] = zz;
      acc[j] = df_add(acc[j], df_two_prod(r, zz));
    }
  }
  double dd[VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) dd[j] = df_to_double(acc[j]);
  block_column_sums<VEC>(dd, k, partial + (int64_t)blockIdx.x * k);
}

}  // namespace

sgp_status Nystrom::build(Lattice* L, int rank, uint64_t seed, float noise, int blur,
                          cudaStream_t st) {
  const int64_t n = L->n;
  l = rank;
  this->noise = noise;
  this->n = n;
#define NY_CHECK(expr, what)                                  \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return cuda_status(e_, what);      \
  } while (0)
  auto get = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  };
  float* om = nullptr;
  NY_CHECK(get((void**)&Bm, (size_t)n * l * sizeof(float)), "alloc Nystrom B");
  NY_CHECK(cudaMallocAsync((void**)&om, (size_t)n * l * sizeof(float), st), "alloc sketch");
  NY_CHECK(get((void**)&partial, (size_t)kTallBlocks * l * std::max(l, kMaxK) * sizeof(double)),
           "alloc partial");
  static bool attrs = false;  // shared-memory sizes beyond the 48 KB default
  if (!attrs) {
    const int big = 200 * 1024;
    cudaFuncSetAttribute(k_gram<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_gram<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_rows_times, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_bt_r, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_apply_z<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_apply_z<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    attrs = true;
  }
  NY_CHECK(get((void**)&C, (size_t)l * l * sizeof(double)), "alloc C");
  NY_CHECK(get((void**)&Q, (size_t)l * l * sizeof(double)), "alloc Q");
  NY_CHECK(get((void**)&T, (size_t)l * l * sizeof(float)), "alloc T");
  NY_CHECK(get((void**)&work, (size_t)std::max(l, kMaxK) * l * sizeof(double)), "alloc work");
  NY_CHECK(get((void**)&tvec, (size_t)l * kMaxK * sizeof(double)), "alloc t");
  NY_CHECK(get((void**)&u, (size_t)l * kMaxK * sizeof(float)), "alloc u");
  NY_CHECK(get((void**)&status, sizeof(int)), "alloc status");
  NY_CHECK(cudaMemsetAsync(status, 0, sizeof(int), st), "clear status");

  // Y = A Omega (one l-column product in locality order), then Y += nu Omega
  sgp_status s = ensure_lattice_values(L, l, st);
  if (s != SGP_OK) return s;
  const unsigned g1 = (unsigned)ceil_div(n * l, 256);
  k_fill_sketch<<<g1, 256, 0, st>>>(L->perm, n, l, seed, om);
  enqueue_mvm(L, om, l, blur, L->outputscale, 0.f, Bm, st, nullptr, /*internal=*/true);
  NY_CHECK(cudaFreeAsync(om, st), "free sketch");
  // nu: a small shift keeps C positive definite when A Omega is rank deficient
  const float nu = 1e-3f * noise;
  k_shift<<<g1, 256, 0, st>>>(L->perm, n, l, seed, nu, Bm);
  note_launches(2);
  // C = Omega^T Y, Cholesky C = R R^T
  const size_t gram_smem = 2 * (size_t)kRowsPerStage * l * sizeof(float);
  k_gram<true><<<kTallBlocks, 256, gram_smem, st>>>(Bm, L->perm, n, l, seed, partial);
  k_sum_blocks<<<(unsigned)ceil_div(l * l, 256), 256, 0, st>>>(partial, kTallBlocks, l * l, C);
  k_cholesky<<<1, 1024, 0, st>>>(C, l, 0.0, status);
  // B = Y R^-T
  k_tri_inv_t<<<1, 128, 0, st>>>(C, l, work, T);
  const int rows = std::max(1, 1024 / l);
  const size_t rt_smem = ((size_t)l * l + (size_t)rows * l) * sizeof(float);
  k_rows_times<<<kTallBlocks, rows * l, rt_smem, st>>>(Bm, T, n, l);
  // M = noise I + B^T B, Cholesky M = Q Q^T
  k_gram<false><<<kTallBlocks, 256, gram_smem, st>>>(Bm, L->perm, n, l, seed, partial);
  k_sum_blocks<<<(unsigned)ceil_div(l * l, 256), 256, 0, st>>>(partial, kTallBlocks, l * l, Q);
  k_cholesky<<<1, 1024, 0, st>>>(Q, l, (double)noise, status);
  note_launches(8);
  NY_CHECK(cudaGetLastError(), "building the Nystrom preconditioner");
  int hs = 0;
  NY_CHECK(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st), "read status");
  NY_CHECK(cudaStreamSynchronize(st), "sync Nystrom");
  ok = hs == 0;
  return SGP_OK;
#undef NY_CHECK
}

void Nystrom::apply(const float* rh, const float* rl, int k, float* z, double* dot_partial,
                    int64_t dot_blocks, int block_threads, cudaStream_t st) const {
  const size_t bt_smem = (size_t)kRowsPerStage * (l + k) * sizeof(float);
  const dim3 bt_grid(kTallBlocks, (unsigned)ceil_div((int64_t)l * k, kOutsPerBlock));
  k_bt_r<<<bt_grid, 256, bt_smem, st>>>(Bm, rh, rl, n, l, k, partial);
  k_sum_blocks<<<(unsigned)ceil_div(l * k, 256), 256, 0, st>>>(partial, kTallBlocks, l * k, tvec);
  k_solve_qqt<<<1, kMaxK, 0, st>>>(Q, tvec, l, k, work, u);
  const size_t z_smem = (size_t)l * k * sizeof(float);
  if (k % 4 == 0)
    k_apply_z<4><<<(unsigned)dot_blocks, block_threads, z_smem, st>>>(Bm, u, rh, rl, 1.f / noise, n,
                                                                      l, k, z, dot_partial);
  else
    k_apply_z<1><<<(unsigned)dot_blocks, block_threads, z_smem, st>>>(Bm, u, rh, rl, 1.f / noise, n,
                                                                      l, k, z, dot_partial);
  note_launches(4);
}

void Nystrom::release(cudaStream_t st) {
  for (void* p : ptrs) (void)cudaFreeAsync(p, st);
  ptrs.clear();
}

}  // namespace sgp
