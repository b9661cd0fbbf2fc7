// Rank-l Nystrom factor of the training block of a GP request's operator (App. A: CG
// pre-conditioner of rank 100), for the server's preconditioned CG.
//
// The lattice operator A = outputscale W M^T M W^T has no cheap entries or diagonal, so
// the low-rank part is a randomized Nystrom approximation built from products with A
// only:
//   Omega  n x l Rademacher sketch over the training rows, entry (i, j) = sign bit of
//          SplitMix64(seed, i l + j) for the caller's point i (counter-based: anyone can
//          regenerate it);
//   Y      = A Omega + nu Omega                 (l-column lattice MVMs, small shift nu);
//   C      = Omega^T Y = R R^T                  (Cholesky, l x l, fp64);
//   B      = Y R^-T                             (so that B B^T = Y C^-1 Y^T);
//   P      = B B^T + noise I,
//   P^-1 r = (r - B (noise I + B^T B)^-1 B^T r) / noise       (Woodbury; applied by the
//          server's table-driven kernels).
// P is symmetric positive definite for any computed B, so CG stays a CG whatever the
// rounding in B; the Cholesky factors of the l x l matrices are computed in fp64 by one
// block, the tall n x l products in fp32 with fixed-order partial sums (deterministic).
// B is stored in fp32 with rows padded to a multiple of 4 columns (zeros) and B^T B is
// formed from the stored values.  All row-indexed arrays are in the lattice's locality
// order.  (The library CG's large-rank preconditioner is precond.cu.)
#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

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

__device__ __forceinline__ float to_f(float x) { return x; }

// Per-block partial of L^T X over the block's rows, L = Omega (regenerated) when OMEGA,
// else L = X.  X: [n][ld] (first l columns used).  out: partial[block][l][l] (fp64 of
// fp32 block sums).
template <bool OMEGA, class TX>
__global__ void k_gram(const TX* __restrict__ X, int ld, const int32_t* __restrict__ perm,
                       int64_t n, int l, uint64_t seed, double* __restrict__ partial) {
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
      xs[e] = to_f(X[(base + rr) * ld + j]);
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

// In-place lower Cholesky of the symmetric part (A + A^T) / 2 of the l x l fp64 matrix A,
// plus shift + rel_shift max_j A[j][j] on the diagonal; one block.  The strict upper
// triangle is zeroed.  *status = 1 when a pivot is not positive.
__global__ void k_cholesky(double* __restrict__ A, int l, double shift, double rel_shift,
                           int* __restrict__ status) {
  __shared__ double piv, dmax;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e / l, j = e % l;
    if (i > j) A[e] = 0.5 * (A[e] + A[j * l + i]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int j = 0; j < l; ++j) m = fmax(m, A[j * l + j]);
    dmax = m;
  }
  __syncthreads();
  const double sh = shift + rel_shift * dmax;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e / l, j = e % l;
    if (i == j) A[e] += sh;
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

// Minv = (Q Q^T)^-1 for lower-triangular Q (fp64): W = Q^-1 by forward substitution per
// column (thread c), then Minv = W^T W.  `work` holds W ([l][l]).
__global__ void k_inv_from_cholesky(const double* __restrict__ Q, int l, double* __restrict__ W,
                                    double* __restrict__ Minv) {
  for (int c = threadIdx.x; c < l; c += blockDim.x) {
    for (int i = 0; i < l; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int j = c; j < i; ++j) s -= Q[i * l + j] * W[j * l + c];
      W[i * l + c] = (i < c) ? 0.0 : s / Q[i * l + i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int a = e / l, b = e % l;
    double s = 0.0;
    for (int i = max(a, b); i < l; ++i) s += W[i * l + a] * W[i * l + b];
    Minv[e] = s;
  }
}

// Masked sketch columns [c0, c0 + kp) in locality order: V[p][c] = Omega[perm[p]][c0 + c]
// on training rows (perm[p] < n_train) and columns c0 + c < l, else 0.
__global__ void k_fill_sketch_chunk(const int32_t* __restrict__ perm, int64_t n, int64_t n_train,
                                    int l, int c0, int kp, uint64_t seed, float* __restrict__ V) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * kp) return;
  const int64_t p = e / kp;
  const int c = (int)(e - p * kp);
  const int32_t i = perm[p];
  V[e] = (i < n_train && c0 + c < l) ? rademacher(seed, i, c0 + c, l) : 0.f;
}

// Y[p][c0 + c] = KV[p][c] + nu Omega[perm[p]][c0 + c] on training rows, 0 on masked rows;
// the last chunk also zeroes the padding columns l..ld-1.
__global__ void k_gather_chunk(const int32_t* __restrict__ perm, int64_t n, int64_t n_train,
                               int l, int ld, int c0, int kp, uint64_t seed, float nu,
                               const float* __restrict__ KV, float* __restrict__ Y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * kp) return;
  const int64_t p = e / kp;
  const int c = (int)(e - p * kp);
  const int j = c0 + c;
  if (j >= ld) return;
  const int32_t i = perm[p];
  float y = 0.f;
  if (j < l && i < n_train) y = fmaf(nu, rademacher(seed, i, j, l), KV[e]);
  Y[p * ld + j] = y;
}

// In place, row by row: Y[row][0..l) = Y[row][0..l) T (T in shared memory).  Each block
// stages its rows before it writes any of them, and no other block touches those rows.
__global__ void k_rows_times_inplace(float* Y, const float* __restrict__ T, int64_t n, int l,
                                     int ld) {
  extern __shared__ float sh[];
  float* ts = sh;              // [l][l]
  float* ys = sh + l * l;      // [rows_per_block][l]
  const int rows = blockDim.x / l;  // blockDim.x = rows * l
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) ts[e] = T[e];
  const int rr = threadIdx.x / l, c = threadIdx.x - rr * l;
  for (int64_t base = (int64_t)blockIdx.x * rows; base < n; base += (int64_t)gridDim.x * rows) {
    __syncthreads();
    const int64_t row = base + rr;
    if (rr < rows && row < n) ys[rr * l + c] = Y[row * ld + c];
    __syncthreads();
    if (rr < rows && row < n) {
      float a = 0.f;
      for (int j = 0; j < l; ++j) a = fmaf(ys[rr * l + j], ts[j * l + c], a);
      Y[row * ld + c] = a;
    }
  }
}

}  // namespace

// Blocks of the masked build's tall products: one per 1024 rows, at most kTallBlocks.
static int masked_tall_blocks(int64_t n) {
  return (int)std::min<int64_t>(kTallBlocks, std::max<int64_t>(1, ceil_div(n, 1024)));
}

size_t nystrom_masked_scratch_bytes(int l, int64_t n) {
  const size_t ll = (size_t)l * l;
  // partial [tall blocks][l][l], C, Q, work (fp64); T (fp32)
  return ((size_t)masked_tall_blocks(n) * ll + 3 * ll) * sizeof(double) + ll * sizeof(float) +
         1024;
}

sgp_status nystrom_build_masked(Lattice* L, int64_t n_train, int l, int ld, uint64_t seed,
                                float noise, int kp, float* V, float* KV, float* Bh,
                                double* Minv, void* scratch, int* status_dev, cudaStream_t st) {
  const int64_t n = L->n;
  const size_t ll = (size_t)l * l;
  const int tall = masked_tall_blocks(n);
  double* partial = static_cast<double*>(scratch);
  double* C = partial + (size_t)tall * ll;
  double* Q = C + ll;
  double* work = Q + ll;
  float* T = reinterpret_cast<float*>(work + ll);
  {  // shared-memory sizes beyond the 48 KB default, once per device
    static std::atomic<bool> attrs[64];  // several host threads may arrive here at once
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    if (dev >= 0 && dev < 64 && !attrs[dev].load()) {
      const int big = 200 * 1024;
      cudaFuncSetAttribute(k_gram<true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
      cudaFuncSetAttribute(k_gram<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
      cudaFuncSetAttribute(k_rows_times_inplace, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
      attrs[dev].store(true);
    }
  }
  cudaError_t e = cudaMemsetAsync(status_dev, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_status(e, "clear Nystrom status");
  // Y = A Omega + nu Omega, kp sketch columns per lattice product, written into Bh
  const float nu = 1e-3f * noise;
  const unsigned g = (unsigned)ceil_div(n * kp, 256);
  for (int c0 = 0; c0 < ld; c0 += kp) {
    k_fill_sketch_chunk<<<g, 256, 0, st>>>(L->perm, n, n_train, l, c0, kp, seed, V);
    enqueue_mvm(L, V, kp, SGP_BLUR_SYMMETRIC, L->outputscale, 0.f, KV, st, nullptr,
                /*internal=*/true);
    k_gather_chunk<<<g, 256, 0, st>>>(L->perm, n, n_train, l, ld, c0, kp, seed, nu, KV, Bh);
    note_launches(2);
  }
  // C = Omega^T Y (masked rows of Y are zero), Cholesky C = R R^T, B = Y R^-T in place
  const size_t gram_smem = 2 * (size_t)kRowsPerStage * l * sizeof(float);
  k_gram<true, float><<<tall, 256, gram_smem, st>>>(Bh, ld, L->perm, n, l, seed, partial);
  k_sum_blocks<<<(unsigned)ceil_div(l * l, 256), 256, 0, st>>>(partial, tall, l * l, C);
  // BF16 lattice values perturb A Omega by ~2^-8 relative: a relative diagonal shift keeps
  // C positive definite (any shift leaves P = B B^T + noise I positive definite)
  const double rel = L->value_dtype == SGP_VALUES_BF16 ? 1e-2 : 0.0;
  k_cholesky<<<1, 1024, 0, st>>>(C, l, 0.0, rel, status_dev);
  k_tri_inv_t<<<1, 128, 0, st>>>(C, l, work, T);
  const int rows = std::max(1, 1024 / l);
  const size_t rt_smem = ((size_t)l * l + (size_t)rows * l) * sizeof(float);
  k_rows_times_inplace<<<tall, rows * l, rt_smem, st>>>(Bh, T, n, l, ld);
  // M = noise I + B^T B from the stored B, Cholesky M = Q Q^T, Minv = M^-1
  k_gram<false, float><<<tall, 256, gram_smem, st>>>(Bh, ld, L->perm, n, l, seed, partial);
  k_sum_blocks<<<(unsigned)ceil_div(l * l, 256), 256, 0, st>>>(partial, tall, l * l, Q);
  k_cholesky<<<1, 1024, 0, st>>>(Q, l, (double)noise, 0.0, status_dev);
  k_inv_from_cholesky<<<1, 128, 0, st>>>(Q, l, work, Minv);
  note_launches(9);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "building the masked Nystrom factor");
  return SGP_OK;
}

}  // namespace sgp
