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
// B is stored in fp32 with rows padded to a multiple of 4 columns (zeros) and B^T B is
// formed from the stored values.  All row-indexed arrays are in the lattice's locality
// order.
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
constexpr int kApplyBlocks = 8 * 152;  // blocks of the per-iteration B^T r reduction

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

// Row by row: Bh[row] = Y[row] T (T in shared memory), columns l..ld-1 zero.
__global__ void k_rows_times(const float* __restrict__ Y, const float* __restrict__ T, int64_t n,
                             int l, int ld, float* __restrict__ Bh) {
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
      Bh[row * ld + c] = a;
      if (c < ld - l) Bh[row * ld + l + c] = 0.f;
    }
  }
}

// Per-block partial of B^T r for the columns [c_off, c_off + 16) of r = rh + rl (ld x 16
// outputs, padded rows of B are zero).  Each warp takes a contiguous range of rows; lane
// `lane` owns the B columns lane, lane + 32, lane + 64, lane + 96 against all 16 r columns
// (64 accumulators), reading its row of B coalesced; lane c < 16 loads r[row][c_off + c]
// and shuffles it to the others.  The block's warps are combined in shared memory in a
// fixed order.
constexpr int kBtWarps = 8;
constexpr int kBtRows = 2;
__global__ void __launch_bounds__(kBtWarps * 32, 2) k_bt_r(const float* __restrict__ Bh, int ld,
                                                        const float* __restrict__ rh,
                                                        const float* __restrict__ rl, int64_t n,
                                                        int k, int c_off,
                                                        double* __restrict__ partial) {
  extern __shared__ float red[];  // [kBtWarps][ld][16]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kc = min(16, k - c_off);
  float acc[4][16];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[a][c] = 0.f;
  const int64_t per_warp = ceil_div(n, (int64_t)gridDim.x * kBtWarps);
  const int64_t r0 = ((int64_t)blockIdx.x * kBtWarps + warp) * per_warp;
  const int64_t r1 = std::min<int64_t>(n, r0 + per_warp);
  // kBtRows rows per step: their loads are issued before any of their FMAs
  for (int64_t row0 = r0; row0 < r1; row0 += kBtRows) {
    float b[kBtRows][4], rv[kBtRows];
#pragma unroll
    for (int q = 0; q < kBtRows; ++q) {
      const int64_t row = row0 + q;
      const bool in = row < r1;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int j = lane + 32 * a;
        b[q][a] = (in && j < ld) ? Bh[row * ld + j] : 0.f;
      }
      const int64_t e = row * k + c_off + lane;
      rv[q] = (in && lane < kc) ? __fadd_rn(rh[e], rl[e]) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kBtRows; ++q)
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const float rc = __shfl_sync(0xffffffffu, rv[q], c);  // r[row][c_off + c]
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][c] = fmaf(b[q][a], rc, acc[a][c]);
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int j = lane + 32 * a;
    if (j < ld)
#pragma unroll
      for (int c = 0; c < 16; ++c) red[(warp * ld + j) * 16 + c] = acc[a][c];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < ld * kc; o += blockDim.x) {
    const int j = o / kc, c = o - j * kc;
    double sum = 0.0;
    for (int w = 0; w < kBtWarps; ++w) sum += (double)red[(w * ld + j) * 16 + c];
    partial[(int64_t)blockIdx.x * ld * k + (int64_t)j * k + c_off + c] = sum;
  }
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

// u = Minv t (fp64, one output per thread), written as fp32 [ld][k] (rows >= l stay 0).
__global__ void k_minv_t(const double* __restrict__ Minv, const double* __restrict__ t, int l,
                         int k, float* __restrict__ u) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= l * k) return;
  const int i = o / k, c = o - i * k;
  double s = 0.0;
  for (int j = 0; j < l; ++j) s += Minv[i * l + j] * t[j * k + c];
  u[i * k + c] = (float)s;
}

// z = (r - B u) / noise for the columns [c_off, c_off + 16) and per-block column sums of
// r z.  One thread per row: it streams its row of B as float4 and reads u ([ld][16] of the
// chunk, in shared memory) as broadcasts, 64 FMAs per float4 of B.
constexpr int kZThreads = 256;
__global__ void __launch_bounds__(kZThreads) k_apply_z(const float* __restrict__ Bh, int ld,
                                                       const float* __restrict__ u,
                                                       const float* __restrict__ rh,
                                                       const float* __restrict__ rl,
                                                       float inv_noise, int64_t n, int k,
                                                       int c_off, float* __restrict__ z,
                                                       double* __restrict__ partial) {
  extern __shared__ float sh[];
  float* us = sh;                                         // [ld][16]
  double* red = reinterpret_cast<double*>(sh + ld * 16);  // [kZThreads][16]
  const int kc = min(16, k - c_off);
  for (int e = threadIdx.x; e < ld * 16; e += blockDim.x) {
    const int q = e / 16, c = e % 16;
    us[e] = c < kc ? u[q * k + c_off + c] : 0.f;
  }
  __syncthreads();
  dfloat acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = {0.f, 0.f};
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    float s[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) s[c] = 0.f;
    const float4* b4 = reinterpret_cast<const float4*>(Bh + row * ld);
    for (int q4 = 0; q4 < ld / 4; ++q4) {
      const float4 b = b4[q4];
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float4* u4 = reinterpret_cast<const float4*>(us + (q4 * 4 + a) * 16);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const float4 uu = u4[g];
          s[4 * g + 0] = fmaf(bv[a], uu.x, s[4 * g + 0]);
          s[4 * g + 1] = fmaf(bv[a], uu.y, s[4 * g + 1]);
          s[4 * g + 2] = fmaf(bv[a], uu.z, s[4 * g + 2]);
          s[4 * g + 3] = fmaf(bv[a], uu.w, s[4 * g + 3]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      if (c < kc) {
        const int64_t e = row * k + c_off + c;
        const float r = __fadd_rn(rh[e], rl[e]);
        const float zz = (r - s[c]) * inv_noise;
        z[e] = zz;
        acc[c] = df_add(acc[c], df_two_prod(r, zz));
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 16; ++c) red[threadIdx.x * 16 + c] = df_to_double(acc[c]);
  __syncthreads();
  for (int c = threadIdx.x; c < kc; c += blockDim.x) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += red[i * 16 + c];
    partial[(int64_t)blockIdx.x * k + c_off + c] = t;
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

sgp_status Nystrom::build(Lattice* L, int rank, uint64_t seed, float noise, int blur,
                          cudaStream_t st) {
  const int64_t n = L->n;
  l = rank;
  ld = (rank + 3) / 4 * 4;
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
  {  // shared-memory sizes beyond the 48 KB default, once per device
    static std::atomic<bool> attrs[64];  // several host threads may arrive here at once
    int dev = 0;
    NY_CHECK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev >= 0 && dev < 64 && !attrs[dev].load()) {
      const int big = 200 * 1024;
      cudaFuncSetAttribute(k_gram<true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
      cudaFuncSetAttribute(k_gram<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
      cudaFuncSetAttribute(k_rows_times, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
      cudaFuncSetAttribute(k_bt_r, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
      cudaFuncSetAttribute(k_apply_z, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
      attrs[dev].store(true);
    }
  }
  float* Y = nullptr;
  float* om = nullptr;
  NY_CHECK(get((void**)&Bh, (size_t)n * ld * sizeof(float)), "alloc Nystrom B");
  NY_CHECK(cudaMallocAsync((void**)&Y, (size_t)n * l * sizeof(float), st), "alloc Nystrom Y");
  NY_CHECK(cudaMallocAsync((void**)&om, (size_t)n * l * sizeof(float), st), "alloc sketch");
  NY_CHECK(get((void**)&partial,
               std::max((size_t)kTallBlocks * l * l, (size_t)kApplyBlocks * ld * kMaxK) *
                   sizeof(double)),
           "alloc partial");
  NY_CHECK(get((void**)&C, (size_t)l * l * sizeof(double)), "alloc C");
  NY_CHECK(get((void**)&Q, (size_t)l * l * sizeof(double)), "alloc Q");
  NY_CHECK(get((void**)&Minv, (size_t)l * l * sizeof(double)), "alloc Minv");
  NY_CHECK(get((void**)&T, (size_t)l * l * sizeof(float)), "alloc T");
  NY_CHECK(get((void**)&work, (size_t)std::max(l, kMaxK) * l * sizeof(double)), "alloc work");
  NY_CHECK(get((void**)&tvec, (size_t)ld * kMaxK * sizeof(double)), "alloc t");
  NY_CHECK(get((void**)&u, (size_t)ld * kMaxK * sizeof(float)), "alloc u");
  NY_CHECK(get((void**)&status, sizeof(int)), "alloc status");
  NY_CHECK(cudaMemsetAsync(status, 0, sizeof(int), st), "clear status");
  NY_CHECK(cudaMemsetAsync(u, 0, (size_t)ld * kMaxK * sizeof(float), st), "clear u");

  // Y = A Omega (one l-column product in locality order), then Y += nu Omega
  sgp_status s = ensure_lattice_values(L, l, st);
  if (s != SGP_OK) return s;
  const unsigned g1 = (unsigned)ceil_div(n * l, 256);
  k_fill_sketch<<<g1, 256, 0, st>>>(L->perm, n, l, seed, om);
  enqueue_mvm(L, om, l, blur, L->outputscale, 0.f, Y, st, nullptr, /*internal=*/true);
  NY_CHECK(cudaFreeAsync(om, st), "free sketch");
  // nu: a small shift keeps C positive definite when A Omega is rank deficient
  const float nu = 1e-3f * noise;
  k_shift<<<g1, 256, 0, st>>>(L->perm, n, l, seed, nu, Y);
  note_launches(2);
  // C = Omega^T Y, Cholesky C = R R^T
  const size_t gram_smem = 2 * (size_t)kRowsPerStage * l * sizeof(float);
  k_gram<true, float><<<kTallBlocks, 256, gram_smem, st>>>(Y, l, L->perm, n, l, seed, partial);
  k_sum_blocks<<<(unsigned)ceil_div(l * l, 256), 256, 0, st>>>(partial, kTallBlocks, l * l, C);
  k_cholesky<<<1, 1024, 0, st>>>(C, l, 0.0, 0.0, status);
  // B = Y R^-T
  k_tri_inv_t<<<1, 128, 0, st>>>(C, l, work, T);
  const int rows = std::max(1, 1024 / l);
  const size_t rt_smem = ((size_t)l * l + (size_t)rows * l) * sizeof(float);
  k_rows_times<<<kTallBlocks, rows * l, rt_smem, st>>>(Y, T, n, l, ld, (float*)Bh);
  NY_CHECK(cudaFreeAsync(Y, st), "free Nystrom Y");
  // M = noise I + B^T B from the stored B, Cholesky M = Q Q^T
  k_gram<false, float><<<kTallBlocks, 256, gram_smem, st>>>((const float*)Bh, ld, L->perm, n, l,
                                                            seed, partial);
  k_sum_blocks<<<(unsigned)ceil_div(l * l, 256), 256, 0, st>>>(partial, kTallBlocks, l * l, Q);
  k_cholesky<<<1, 1024, 0, st>>>(Q, l, (double)noise, 0.0, status);
  k_inv_from_cholesky<<<1, 128, 0, st>>>(Q, l, work, Minv);
  note_launches(9);
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
  (void)block_threads;
  const size_t bt_smem = (size_t)kBtWarps * ld * 16 * sizeof(float);
  for (int c_off = 0; c_off < k; c_off += 16)
    k_bt_r<<<kApplyBlocks, kBtWarps * 32, bt_smem, st>>>((const float*)Bh, ld, rh, rl, n, k, c_off,
                                                         partial);
  k_sum_blocks<<<(unsigned)ceil_div((int64_t)ld * k, 256), 256, 0, st>>>(partial, kApplyBlocks,
                                                                       ld * k, tvec);
  k_minv_t<<<(unsigned)ceil_div((int64_t)l * k, 128), 128, 0, st>>>(Minv, tvec, l, k, u);
  const size_t z_smem = (size_t)ld * 16 * sizeof(float) + (size_t)kZThreads * 16 * sizeof(double);
  for (int c_off = 0; c_off < k; c_off += 16)
    k_apply_z<<<(unsigned)dot_blocks, kZThreads, z_smem, st>>>((const float*)Bh, ld, u, rh, rl,
                                                               1.f / noise, n, k, c_off, z,
                                                               dot_partial);
  note_launches(2 + 2 * ceil_div(k, 16));
}

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

void Nystrom::release(cudaStream_t st) {
  for (void* p : ptrs) (void)cudaFreeAsync(p, st);
  ptrs.clear();
}

}  // namespace sgp
