// Large-rank Nystrom preconditioner for the library CG (App. A: CG pre-conditioner; the
// rank a system needs grows with its conditioning).
//
// With A = K + noise I (K = outputscale W M^T M W^T, reachable only through products):
//   Omega   n x l Rademacher sketch, entry (i, j) = sign bit of SplitMix64 at counter
//           i l + j + 1 from the seed (i = the caller's point index);
//   Q       Omega, or after q = 1 subspace iteration an orthonormal basis of K Omega
//           (Cholesky QR, twice; the approximation depends only on the subspace);
//   Y       = K Q;   C = (Q^T Y + Y^T Q) / 2 + eps I,  eps = 1e-6 max_j C_jj (raised when
//           the Cholesky of C fails);
//   B       = Y R^-T with C = R R^T, so that B B^T = Y C^-1 Y^T ~ K, rounded to bf16 and
//           stored so (P is defined by the stored values: B^T B is formed from them);
//   tau     = lambda_min(B^T B) + noise (the smallest retained eigenvalue plus the noise,
//           estimated by inverse power iteration);
//   P       = B B^T + tau I,   P^-1 r = (r - B Minv B^T r) / tau,  Minv = (tau I + B^T B)^-1.
// On the captured subspace P ~ K + tau I, elsewhere P = tau I, so the spectrum of P^-1 A
// lies in [noise / tau, ~1].  Because tau is the smallest captured eigenvalue and not the
// noise, B Minv B^T r never cancels r to more than about tau / lambda_max: the apply stays
// accurate in fp32 (with tau = noise, fp32 cancellation in the top eigen-directions breaks
// positive definiteness at large ranks).
//
// The set-up's tall n x l products (Grams Q^T Y, B^T B, Y^T Y; panel times l x l matrix)
// run on the tensor cores as m16n8k8 TF32 MMAs with a 3xTF32 split (hi hi + hi lo + lo hi,
// about fp32 accuracy), fp32 sums inside a block and fp64 sums across blocks in a fixed
// order.  The l x l factorizations (Cholesky, triangular inverse, products) run in fp64 on
// the CUDA cores in 32 x 32 blocks.  Panels are fp32 [n][ld] in the lattice's locality
// order, ld = l rounded up to 128, padding columns zero.
// Per iteration the apply reads the bf16 factor twice (B^T r, then B u): 2 n ld bytes each,
// half of an fp32 factor.  With tau well above the noise the bf16 rounding of B (a
// perturbation of order 2^-9 ||B||^2 / sqrt(l) of B B^T, small against tau) leaves the
// iteration counts unchanged (measured at n = 2M, ranks 1024 and 2048).  The MMAs there are
// m16n8k16 bf16 with B exact and r, u split in three bf16 parts (about 24 bits).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include "sgp_internal.cuh"

namespace sgp {
namespace {

constexpr int kTile = 128;     // M and N tile of the panel products
constexpr int kKc = 32;        // K chunk staged per step
constexpr int kSMN = 136;      // smem row stride (floats) of [kKc][128] tiles (MN-major use)
constexpr int kSK = 36;        // smem row stride of [128][kKc] tiles (K-major use)
constexpr int kSR = 24;        // smem row stride of [kKc][16] right-hand-side tiles
constexpr int kSketchCols = 128;  // sketch columns per lattice product
constexpr int kNB = 32;        // block size of the fp64 factorizations

// ---- TF32 MMA pieces --------------------------------------------------------------------
// Round an fp32 bit pattern to TF32 (10 explicit mantissa bits), nearest with ties away
// from zero, by integer arithmetic on the magnitude bits: adding half a TF32 unit carries
// into the kept bits (and into the exponent when the mantissa overflows), then the 13 low
// bits are cleared.  Two integer operations instead of a conversion instruction (whose
// issue rate limits the per-iteration kernels); same result as cvt.rna for finite x.
__device__ __forceinline__ uint32_t tf32_round_bits(uint32_t b) {
  return (b + 0x1000u) & 0xFFFFE000u;
}
// x = hi + lo with hi, lo TF32 (hi hi + hi lo + lo hi keeps about fp32 accuracy); x - hi is
// exact in fp32.
__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_round_bits(__float_as_uint(x));
  lo = tf32_round_bits(__float_as_uint(x - __uint_as_float(hi)));
}
// D (16 x 8) += A (16 x 8, row-major) B (8 x 8, column-major); lane = 4 g + t holds
// A[g][t], A[g + 8][t], A[g][t + 4], A[g + 8][t + 4]; B[t][g], B[t + 4][g];
// D[g][2t], D[g][2t + 1], D[g + 8][2t], D[g + 8][2t + 1].
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                    uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                     uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
  mma(d, al, bh0, bh1);
  mma(d, ah, bl0, bl1);
  mma(d, ah, bh0, bh1);
}

// ---- cp.async ---------------------------------------------------------------------------
__device__ __forceinline__ void cp16(float* smem, const float* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int bytes = valid ? 16 : 0;  // 0: the 16 bytes are zero-filled, nothing is read
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// SplitMix64 (Steele, Lea & Flood 2014) at counter i l + j + 1: one +-1 per (point, column).
__device__ __forceinline__ float sketch_sign(uint64_t seed, int64_t i, int j, int l) {
  uint64_t z = seed + ((uint64_t)(i * l + j) + 1ull) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (z >> 63) ? -1.f : 1.f;
}

// P[p][j] = Omega[perm[p]][j] for j < l, 0 for l <= j < ld.
__global__ void k_fill_sketch_panel(const int32_t* __restrict__ perm, int64_t n, int l, int ld,
                                    uint64_t seed, float* __restrict__ P) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * ld) return;
  const int64_t p = e / ld;
  const int j = (int)(e - p * ld);
  P[e] = j < l ? sketch_sign(seed, perm[p], j, l) : 0.f;
}

// dst[p][c] = src[p][c0 + c] for c < kc (to_panel = false); the reverse when to_panel.
__global__ void k_copy_cols(float* __restrict__ panel, int ld, int c0, float* __restrict__ dense,
                            int kc, int64_t n, bool to_panel) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * kc) return;
  const int64_t p = e / kc;
  const int c = (int)(e - p * kc);
  if (to_panel) panel[p * ld + c0 + c] = dense[e];
  else dense[e] = panel[p * ld + c0 + c];
}

// ---- tall products on the tensor cores ---------------------------------------------------
// partial[s] = X[rows of split s]^T Y[rows of split s], [ldp][ldp] fp32 per split, for the
// 128 x 128 output tiles on and below the diagonal (symmetric results: the Grams here are
// symmetric up to rounding), blockIdx.x = ti (ti + 1) / 2 + tj, tj <= ti.  256 threads:
// warp (wi, wj) owns the 64 x 32 sub-tile (wi = warp / 4, wj = warp % 4).  Rows are
// staged 32 at a time.
__global__ void __launch_bounds__(256, 2) k_gram_tc(const float* __restrict__ X, int ldx,
                                                    const float* __restrict__ Y, int ldy,
                                                    int64_t n, int ntile, int64_t rows_per_split,
                                                    int ldp, float* __restrict__ partial) {
  extern __shared__ __align__(16) float sm[];
  float* xs = sm;                    // [2][kKc][kSMN]
  float* ys = sm + 2 * kKc * kSMN;   // [2][kKc][kSMN]
  int ti = (int)((sqrtf(8.f * blockIdx.x + 1.f) - 1.f) * 0.5f);
  while ((ti + 1) * (ti + 2) / 2 <= (int)blockIdx.x) ++ti;
  while (ti * (ti + 1) / 2 > (int)blockIdx.x) --ti;
  const int i0 = ti * kTile, j0 = ((int)blockIdx.x - ti * (ti + 1) / 2) * kTile;
  (void)ntile;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r_end = std::min<int64_t>(n, r_begin + rows_per_split);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  const int wi = warp >> 2, wj = warp & 3;
  float acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  auto load = [&](int buf, int64_t r0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;  // 32 rows x 32 float4
      const int rr = e >> 5, c4 = (e & 31) * 4;
      const int64_t r = r0 + rr;
      const bool ok = r < r_end;
      cp16(xs + (buf * kKc + rr) * kSMN + c4, ok ? X + r * ldx + i0 + c4 : X, ok);
      cp16(ys + (buf * kKc + rr) * kSMN + c4, ok ? Y + r * ldy + j0 + c4 : Y, ok);
    }
    cp_commit();
  };
  const int64_t nchunks = r_end > r_begin ? ceil_div(r_end - r_begin, kKc) : 0;
  if (nchunks > 0) load(0, r_begin);
  for (int64_t c = 0; c < nchunks; ++c) {
    const int buf = (int)(c & 1);
    if (c + 1 < nchunks) {
      load(buf ^ 1, r_begin + (c + 1) * kKc);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const float* Xs = xs + buf * kKc * kSMN;
    const float* Ys = ys + buf * kKc * kSMN;
#pragma unroll
    for (int kk = 0; kk < kKc; kk += 8) {
      uint32_t bh[4][2], bl[4][2];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int jb = wj * 32 + nt * 8 + g;
        split(Ys[(kk + tq) * kSMN + jb], bh[nt][0], bl[nt][0]);
        split(Ys[(kk + tq + 4) * kSMN + jb], bh[nt][1], bl[nt][1]);
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int ib = wi * 64 + mt * 16 + g;
        uint32_t ah[4], al[4];
        split(Xs[(kk + tq) * kSMN + ib], ah[0], al[0]);
        split(Xs[(kk + tq) * kSMN + ib + 8], ah[1], al[1]);
        split(Xs[(kk + tq + 4) * kSMN + ib], ah[2], al[2]);
        split(Xs[(kk + tq + 4) * kSMN + ib + 8], ah[3], al[3]);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          mma3(acc[mt][nt], ah, al, bh[nt][0], bh[nt][1], bl[nt][0], bl[nt][1]);
      }
    }
    __syncthreads();
  }
  float* out = partial + (size_t)blockIdx.y * ldp * ldp;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int i = i0 + wi * 64 + mt * 16 + g;
      const int j = j0 + wj * 32 + nt * 8 + 2 * tq;
      *reinterpret_cast<float2*>(out + (size_t)i * ldp + j) =
          make_float2(acc[mt][nt][0], acc[mt][nt][1]);
      *reinterpret_cast<float2*>(out + (size_t)(i + 8) * ldp + j) =
          make_float2(acc[mt][nt][2], acc[mt][nt][3]);
    }
}

// G[i][j] = sum over splits of partial[s][i][j] (fp64, in split order) for the tiles on
// and below the diagonal, mirrored above it.
__global__ void k_sum_splits(const float* __restrict__ partial, int splits, int ldp,
                             double* __restrict__ G) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t count = (int64_t)ldp * ldp;
  if (e >= count) return;
  int i = (int)(e / ldp), j = (int)(e % ldp);
  if (j / kTile > i / kTile) {  // computed as its transpose
    const int t = i;
    i = j;
    j = t;
  }
  const int64_t src = (int64_t)i * ldp + j;
  double t = 0.0;
  for (int s = 0; s < splits; ++s) t += (double)partial[(size_t)s * count + src];
  G[e] = t;
}

// Z[r][j] = sum_i Y[r][i] Tt[j][i] for i < kdim (Tt: [ld][ld] fp32), 128 x 128 output tile
// (blockIdx.x = row tile, blockIdx.y = column tile); warp (wi, wj) owns 64 x 32.  With
// Tt lower triangular only i < 128 (column tile + 1) contributes.
__global__ void __launch_bounds__(256, 2) k_panel_tc(const float* __restrict__ Y, int ldy,
                                                     const float* __restrict__ Tt, int ldt,
                                                     int kdim, bool lower, int64_t n,
                                                     float* __restrict__ Z, int ldz) {
  extern __shared__ __align__(16) float sm[];
  float* ysm = sm;                    // [2][kTile][kSK]
  float* tsm = sm + 2 * kTile * kSK;  // [2][kTile][kSK]
  const int64_t r0 = (int64_t)blockIdx.x * kTile;
  const int j0 = blockIdx.y * kTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  const int wi = warp >> 2, wj = warp & 3;
  float acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  auto load = [&](int buf, int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;  // 128 rows x 8 float4
      const int rr = e >> 3, c4 = (e & 7) * 4;
      const int64_t r = r0 + rr;
      const bool ok = r < n;
      cp16(ysm + (buf * kTile + rr) * kSK + c4, ok ? Y + r * ldy + k0 + c4 : Y, ok);
      cp16(tsm + (buf * kTile + rr) * kSK + c4, Tt + (size_t)(j0 + rr) * ldt + k0 + c4, true);
    }
    cp_commit();
  };
  const int nchunks = (lower ? min(kdim, j0 + kTile) : kdim) / kKc;
  load(0, 0);
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    if (c + 1 < nchunks) {
      load(buf ^ 1, (c + 1) * kKc);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const float* Ys = ysm + buf * kTile * kSK;
    const float* Ts = tsm + buf * kTile * kSK;
#pragma unroll
    for (int kk = 0; kk < kKc; kk += 8) {
      uint32_t bh[4][2], bl[4][2];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int jb = wj * 32 + nt * 8 + g;
        split(Ts[jb * kSK + kk + tq], bh[nt][0], bl[nt][0]);
        split(Ts[jb * kSK + kk + tq + 4], bh[nt][1], bl[nt][1]);
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int rb = wi * 64 + mt * 16 + g;
        uint32_t ah[4], al[4];
        split(Ys[rb * kSK + kk + tq], ah[0], al[0]);
        split(Ys[(rb + 8) * kSK + kk + tq], ah[1], al[1]);
        split(Ys[rb * kSK + kk + tq + 4], ah[2], al[2]);
        split(Ys[(rb + 8) * kSK + kk + tq + 4], ah[3], al[3]);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          mma3(acc[mt][nt], ah, al, bh[nt][0], bh[nt][1], bl[nt][0], bl[nt][1]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int64_t r = r0 + wi * 64 + mt * 16 + g;
      const int j = j0 + wj * 32 + nt * 8 + 2 * tq;
      if (r < n)
        *reinterpret_cast<float2*>(Z + r * ldz + j) = make_float2(acc[mt][nt][0], acc[mt][nt][1]);
      if (r + 8 < n)
        *reinterpret_cast<float2*>(Z + (r + 8) * ldz + j) =
            make_float2(acc[mt][nt][2], acc[mt][nt][3]);
    }
}

// 4-byte cp.async (r rows of any width k are not 16-byte aligned).
__device__ __forceinline__ void cp4(float* smem, const float* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int bytes = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp16b(void* smem, const void* gmem, bool valid) {
  cp16(reinterpret_cast<float*>(smem), reinterpret_cast<const float*>(gmem), valid);
}

// ---- per-iteration apply with the bf16 factor ---------------------------------------------
// B holds bf16 values exactly, so the products B^T r and B u are formed on the tensor cores
// as m16n8k16 bf16 MMAs with B as the exact operand and r, u split in three bf16 parts
// x = x1 + x2 + x3 (about 24 bits): products are exact in fp32, sums fp32 within a block.
// A fragments of B come from shared memory by ldmatrix (transposed for B^T).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* row_addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"((unsigned)__cvta_generic_to_shared(row_addr)));
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* row_addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"((unsigned)__cvta_generic_to_shared(row_addr)));
}
// x = x1 + x2 + x3 in bf16 (each part the nearest bf16 of what is left; the differences are
// exact in fp32)
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b,
                                       __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

constexpr int kApplyStages = 4;   // chunks in flight per block in the per-iteration kernels
constexpr int kBtRowB = 136;      // bf16 per smem row of a [32 r][128 i] tile (272 B)
constexpr int kBtStageBytes = kKc * kBtRowB * 2 + 2 * kKc * kSR * 4;
constexpr int kZRowB = 40;        // bf16 per smem row of a [128 r][32 i] tile (80 B)
constexpr int kZURow = 40;        // bf16 per smem row of a [3][16 c][32 i] u tile
constexpr int kZStageBytes = kTile * kZRowB * 2 + 3 * 16 * kZURow * 2;

// Per-iteration B^T r for 16 columns [c_off, c_off + kc) of r = rh + rl:
// tpart[s][i][c] = sum over the rows of split s of B[row][i] r[row][c_off + c], for the
// 128 rows i of tile blockIdx.x (split blockIdx.y).  Warp w owns i rows 16 w .. 16 w + 15.
// Chunks of 32 rows (B: 128 columns, r: both fp32 parts) stream through kApplyStages
// shared-memory stages by cp.async.
__global__ void __launch_bounds__(256) k_bt_bf16(const __nv_bfloat16* __restrict__ B, int ld,
                                                 const float* __restrict__ rh,
                                                 const float* __restrict__ rl, int k, int c_off,
                                                 int kc, int64_t n, int64_t rows_per_split,
                                                 float* __restrict__ tpart) {
  extern __shared__ __align__(16) uint8_t smb[];  // [kApplyStages][kBtStageBytes]
  const int i0 = blockIdx.x * kTile;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r_end = std::min<int64_t>(n, r_begin + rows_per_split);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  float acc[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  auto load = [&](int slot, int64_t r0) {
    uint8_t* st = smb + slot * kBtStageBytes;
    __nv_bfloat16* bs = reinterpret_cast<__nv_bfloat16*>(st);
    float* hs = reinterpret_cast<float*>(st + kKc * kBtRowB * 2);
    float* ls = hs + kKc * kSR;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = threadIdx.x + 256 * q;  // 32 rows x 16 pieces of 16 bytes
      const int rr = e >> 4, c8 = (e & 15) * 8;
      const int64_t r = r0 + rr;
      const bool ok = r < r_end;
      cp16b(bs + rr * kBtRowB + c8, ok ? B + r * ld + i0 + c8 : B, ok);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {  // 32 rows x 16 columns of rh and of rl
      const int e = threadIdx.x + 256 * q;
      const int rr = e >> 4, c = e & 15;
      const int64_t r = r0 + rr;
      const bool ok = r < r_end && c < kc;
      const int64_t off = ok ? r * k + c_off + c : 0;
      cp4(hs + rr * kSR + c, rh + off, ok);
      cp4(ls + rr * kSR + c, rl + off, ok);
    }
  };
  const int64_t nchunks = r_end > r_begin ? ceil_div(r_end - r_begin, kKc) : 0;
#pragma unroll
  for (int s0 = 0; s0 < kApplyStages - 1; ++s0) {
    if (s0 < nchunks) load(s0, r_begin + (int64_t)s0 * kKc);
    cp_commit();
  }
  // ldmatrix.trans row addresses: matrix q = lane / 8 covers k rows 8 (q >> 1) .. + 7 and
  // i columns 8 (q & 1) .. + 7 of the warp's 16 x 16 A tile (A[i][r] = B[r][i])
  const int q = lane >> 3, j = lane & 7;
  const int lrow = 8 * (q >> 1) + j, lcol = warp * 16 + 8 * (q & 1);
  for (int64_t c = 0; c < nchunks; ++c) {
    cp_wait<kApplyStages - 2>();
    __syncthreads();  // chunk c has landed; every warp is done with chunk c - 1's stage
    if (c + kApplyStages - 1 < nchunks)
      load((int)((c + kApplyStages - 1) % kApplyStages), r_begin + (c + kApplyStages - 1) * kKc);
    cp_commit();
    const uint8_t* st = smb + (int)(c % kApplyStages) * kBtStageBytes;
    const __nv_bfloat16* Bs = reinterpret_cast<const __nv_bfloat16*>(st);
    const float* Hs = reinterpret_cast<const float*>(st + kKc * kBtRowB * 2);
    const float* Ls = Hs + kKc * kSR;
#pragma unroll
    for (int kk = 0; kk < kKc; kk += 16) {
      uint32_t a[4];
      ldsm_x4_trans(a, Bs + (kk + lrow) * kBtRowB + lcol);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        // B operand B'[k][n] = r[kk + k][nt 8 + n]: b0 = rows 2 tq, 2 tq + 1 and b1 = rows
        // 2 tq + 8, 2 tq + 9 of column g
        __nv_bfloat16 p[4][3];
#pragma unroll
        for (int e2 = 0; e2 < 4; ++e2) {
          const int kr = kk + 2 * tq + (e2 & 1) + 8 * (e2 >> 1);
          const int o = kr * kSR + nt * 8 + g;
          split3(__fadd_rn(Hs[o], Ls[o]), p[e2][0], p[e2][1], p[e2][2]);
        }
#pragma unroll
        for (int part = 2; part >= 0; --part)
          mma_bf16(acc[nt], a, pack2(p[0][part], p[1][part]), pack2(p[2][part], p[3][part]));
      }
    }
  }
  cp_wait<0>();
  float* out = tpart + (size_t)blockIdx.y * gridDim.x * kTile * 16;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    const int i = i0 + warp * 16 + g;
    const int c = nt * 8 + 2 * tq;
    *reinterpret_cast<float2*>(out + (size_t)i * 16 + c) = make_float2(acc[nt][0], acc[nt][1]);
    *reinterpret_cast<float2*>(out + (size_t)(i + 8) * 16 + c) = make_float2(acc[nt][2], acc[nt][3]);
  }
}

// t[i][c] = sum over splits of tpart[s][i][c] (fp64 in split order, stored fp32), i < ld.
__global__ void k_sum_t(const float* __restrict__ tpart, int splits, int ld,
                        float* __restrict__ t) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ld * 16) return;
  double s = 0.0;
  for (int q = 0; q < splits; ++q) s += (double)tpart[(size_t)q * ld * 16 + e];
  t[e] = (float)s;
}

// u[i][c] = sum_j Minv[i][j] t[j][c] (fp32), i < ld, c < 16; one thread per output.  Stored
// split in three bf16 parts, transposed: u3[part][c][i].
__global__ void k_minv_u(const float* __restrict__ Minv, int ld, const float* __restrict__ t,
                         __nv_bfloat16* __restrict__ u3) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ld * 16) return;
  const int i = e >> 4, c = e & 15;
  const float* row = Minv + (size_t)i * ld;
  float s = 0.f;
  for (int j = 0; j < ld; ++j) s = fmaf(row[j], t[j * 16 + c], s);
  __nv_bfloat16 a, b, d;
  split3(s, a, b, d);
  u3[(size_t)(0 * 16 + c) * ld + i] = a;
  u3[(size_t)(1 * 16 + c) * ld + i] = b;
  u3[(size_t)(2 * 16 + c) * ld + i] = d;
}

// z[r][c_off + c] = (r - B u)[r][c] * inv_tau for the 128 rows of tile blockIdx.x, and the
// tile's column sums of r z (double-float per lane, fixed butterfly over the lanes of a
// column, warps in order) into dot[blockIdx.x][c_off + c].  Warp w owns rows 16 w .. + 15.
// Chunks of 32 columns of B (and the matching 32 entries of each u part) stream through
// kApplyStages shared-memory stages by cp.async.
__global__ void __launch_bounds__(256) k_apply_z_bf16(const __nv_bfloat16* __restrict__ B,
                                                      int ld, const __nv_bfloat16* __restrict__ u3,
                                                      const float* __restrict__ rh,
                                                      const float* __restrict__ rl, int k,
                                                      int c_off, int kc, int64_t n,
                                                      float inv_tau, float* __restrict__ z,
                                                      double* __restrict__ dot) {
  extern __shared__ __align__(16) uint8_t smb[];  // [kApplyStages][kZStageBytes]
  __shared__ double red[8][16];
  const int64_t r0 = (int64_t)blockIdx.x * kTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  float acc[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  auto load = [&](int slot, int k0) {
    uint8_t* st = smb + slot * kZStageBytes;
    __nv_bfloat16* bs = reinterpret_cast<__nv_bfloat16*>(st);
    __nv_bfloat16* us = reinterpret_cast<__nv_bfloat16*>(st + kTile * kZRowB * 2);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = threadIdx.x + 256 * q;  // 128 rows x 4 pieces of 16 bytes
      const int rr = e >> 2, c8 = (e & 3) * 8;
      const int64_t r = r0 + rr;
      const bool ok = r < n;
      cp16b(bs + rr * kZRowB + c8, ok ? B + r * ld + k0 + c8 : B, ok);
    }
    if (threadIdx.x < 3 * 16 * 4) {  // u parts: 48 rows (part, c) x 4 pieces of 16 bytes
      const int row = threadIdx.x >> 2, c8 = (threadIdx.x & 3) * 8;
      cp16b(us + row * kZURow + c8, u3 + (size_t)row * ld + k0 + c8, true);
    }
  };
  const int nchunks = ld / kKc;
#pragma unroll
  for (int s0 = 0; s0 < kApplyStages - 1; ++s0) {
    if (s0 < nchunks) load(s0, s0 * kKc);
    cp_commit();
  }
  // ldmatrix row addresses: matrix q = lane / 8 covers rows 8 (q & 1) .. + 7 of the warp's
  // 16 rows and columns 8 (q >> 1) .. + 7 of the 16-column k step
  const int q = lane >> 3, j = lane & 7;
  const int lrow = warp * 16 + 8 * (q & 1) + j, lcol = 8 * (q >> 1);
  for (int c = 0; c < nchunks; ++c) {
    cp_wait<kApplyStages - 2>();
    __syncthreads();  // chunk c has landed; every warp is done with chunk c - 1's stage
    if (c + kApplyStages - 1 < nchunks)
      load((c + kApplyStages - 1) % kApplyStages, (c + kApplyStages - 1) * kKc);
    cp_commit();
    const uint8_t* st = smb + (c % kApplyStages) * kZStageBytes;
    const __nv_bfloat16* Bs = reinterpret_cast<const __nv_bfloat16*>(st);
    const __nv_bfloat16* Us = reinterpret_cast<const __nv_bfloat16*>(st + kTile * kZRowB * 2);
#pragma unroll
    for (int kk = 0; kk < kKc; kk += 16) {
      uint32_t a[4];
      ldsm_x4(a, Bs + lrow * kZRowB + kk + lcol);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int part = 2; part >= 0; --part) {
          // B operand B'[k][n] = u[kk + k][nt 8 + n]: consecutive k of column n are adjacent
          const __nv_bfloat16* ub = Us + (part * 16 + nt * 8 + g) * kZURow + kk + 2 * tq;
          const uint32_t b0 = *reinterpret_cast<const uint32_t*>(ub);
          const uint32_t b1 = *reinterpret_cast<const uint32_t*>(ub + 8);
          mma_bf16(acc[nt], a, b0, b1);
        }
    }
  }
  cp_wait<0>();
  // epilogue: this lane holds rows g, g + 8 of the warp's 16 and columns nt 8 + 2 tq (+1)
  dfloat d[2][2];
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) d[nt][0] = d[nt][1] = {0.f, 0.f};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t r = r0 + warp * 16 + g + 8 * h;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int q2 = 0; q2 < 2; ++q2) {
        const int c = nt * 8 + 2 * tq + q2;
        if (r < n && c < kc) {
          const int64_t e = r * k + c_off + c;
          const float rv = __fadd_rn(rh[e], rl[e]);
          const float zz = (rv - acc[nt][2 * h + q2]) * inv_tau;
          z[e] = zz;
          d[nt][q2] = df_add(d[nt][q2], df_two_prod(rv, zz));
        }
      }
  }
  // lanes with the same tq hold the same columns: combine over g (xor 4, 8, 16)
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int q2 = 0; q2 < 2; ++q2) {
      double v = df_to_double(d[nt][q2]);
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      if (g == 0) red[warp][nt * 8 + 2 * tq + q2] = v;
    }
  __syncthreads();
  if (threadIdx.x < 16 && (int)threadIdx.x < kc) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
    dot[(int64_t)blockIdx.x * k + c_off + threadIdx.x] = s;
  }
}

// ---- l x l fp64 factorizations (row-major, leading dimension lda, size l) ---------------
// (A + A^T) / 2 into the lower triangle, plus `shift` + rel * max_j A[j][j] on the
// diagonal; the strict upper triangle is zeroed.  One block.
__global__ void k_prepare_spd(double* __restrict__ A, int l, int lda, double shift,
                              double rel) {
  __shared__ double dmax;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int j = 0; j < l; ++j) m = fmax(m, A[(size_t)j * lda + j]);
    dmax = m;
  }
  __syncthreads();
  const double sh = shift + rel * dmax;
  for (int64_t e = threadIdx.x; e < (int64_t)l * l; e += blockDim.x) {
    const int i = (int)(e / l), j = (int)(e % l);
    if (i > j) A[(size_t)i * lda + j] = 0.5 * (A[(size_t)i * lda + j] + A[(size_t)j * lda + i]);
    else if (i == j) A[(size_t)i * lda + j] += sh;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)l * l; e += blockDim.x) {
    const int i = (int)(e / l), j = (int)(e % l);
    if (j > i) A[(size_t)i * lda + j] = 0.0;
  }
}

// Cholesky of the diagonal block [kb, kb + nb): unblocked, in shared memory; *status = 1
// when a pivot is not positive (the pivot is then taken as 1 so that nothing overflows).
__global__ void k_potrf_diag(double* __restrict__ A, int lda, int kb, int nb,
                             int* __restrict__ status) {
  __shared__ double a[kNB][kNB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    a[i][j] = j <= i ? A[(size_t)(kb + i) * lda + kb + j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      const double d = a[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        *status = 1;
        a[j][j] = 1.0;
      } else {
        a[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] /= a[j][j];
    __syncthreads();
    const int rem = nb - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e / rem, c = j + 1 + e % rem;
      if (c <= i) a[i][c] -= a[i][j] * a[c][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    if (j <= i) A[(size_t)(kb + i) * lda + kb + j] = a[i][j];
  }
}

// Panel below the diagonal block: rows i >= kb + nb, A[i][kb .. kb + nb) <- solve of
// x L_kk^T = A[i][kb ..]; one thread per row.
__global__ void k_trsm_panel(double* __restrict__ A, int lda, int l, int kb, int nb) {
  __shared__ double Lk[kNB][kNB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    Lk[i][j] = j <= i ? A[(size_t)(kb + i) * lda + kb + j] : 0.0;
  }
  __syncthreads();
  const int i = kb + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= l) return;
  double x[kNB];
  double* row = A + (size_t)i * lda + kb;
#pragma unroll
  for (int c = 0; c < kNB; ++c) x[c] = c < nb ? row[c] : 0.0;
#pragma unroll
  for (int c = 0; c < kNB; ++c) {
    if (c < nb) {
      double s = x[c];
#pragma unroll
      for (int t = 0; t < kNB; ++t)
        if (t < c) s -= x[t] * Lk[c][t];
      x[c] = s / Lk[c][c];
    }
  }
#pragma unroll
  for (int c = 0; c < kNB; ++c)
    if (c < nb) row[c] = x[c];
}

// Lower triangle of the trailing matrix: A[i][j] -= sum_t A[i][kb + t] A[j][kb + t] for
// s <= j <= i < l, s = kb + nb; one 32 x 32 tile (I >= J) per block, 4 outputs per thread.
__global__ void __launch_bounds__(256) k_syrk_trailing(double* __restrict__ A, int lda, int l,
                                                        int kb, int nb) {
  __shared__ double pi[kNB][kNB + 1], pj[kNB][kNB + 1];
  const int s = kb + nb;
  const int b = blockIdx.x;
  int I = (int)((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= b) ++I;
  while (I * (I + 1) / 2 > b) --I;
  const int J = b - I * (I + 1) / 2;
  const int ib = s + I * kNB, jb = s + J * kNB;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, t = e % kNB;
    pi[r][t] = (ib + r < l && t < nb) ? A[(size_t)(ib + r) * lda + kb + t] : 0.0;
    pj[r][t] = (jb + r < l && t < nb) ? A[(size_t)(jb + r) * lda + kb + t] : 0.0;
  }
  __syncthreads();
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + 256 * q;
    const int r = e / kNB, c = e % kNB;
    const int i = ib + r, j = jb + c;
    if (i < l && j <= i) {
      double acc = 0.0;
      for (int t = 0; t < nb; ++t) acc += pi[r][t] * pj[c][t];
      A[(size_t)i * lda + j] -= acc;
    }
  }
}

// Inverse of each 32 x 32 lower diagonal block of L into X (forward substitution per
// column in shared memory); the strict upper part of the block is zero.
__global__ void k_trtri_diag(const double* __restrict__ L, double* __restrict__ X, int lda,
                             int l) {
  __shared__ double a[kNB][kNB + 1], x[kNB][kNB + 1];
  const int b0 = blockIdx.x * kNB;
  const int nb = min(kNB, l - b0);
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int i = e / kNB, j = e % kNB;
    a[i][j] = (i < nb && j <= i) ? L[(size_t)(b0 + i) * lda + b0 + j] : 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < nb) {
    for (int i = 0; i < nb; ++i) {
      if (i < c) {
        x[i][c] = 0.0;
      } else if (i == c) {
        x[i][c] = 1.0 / a[i][i];
      } else {
        double s = 0.0;
        for (int t = c; t < i; ++t) s += a[i][t] * x[t][c];
        x[i][c] = -s / a[i][i];
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    X[(size_t)(b0 + i) * lda + b0 + j] = x[i][j];
  }
}

// Block row I of X = L^-1: X[I][J] = -X[I][I] sum_{K = J}^{I - 1} L[I][K] X[K][J] for every
// J < I (blockIdx.x = J); rows I of the blocks before it are final.
__global__ void __launch_bounds__(256) k_trtri_row(const double* __restrict__ L,
                                                    double* __restrict__ X, int lda, int l,
                                                    int I) {
  __shared__ double lt[kNB][kNB + 1], xt[kNB][kNB + 1], sacc[kNB][kNB + 1];
  const int J = blockIdx.x;
  const int ib = I * kNB, jb = J * kNB;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int K = J; K < I; ++K) {
    const int kbk = K * kNB;
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
      const int r = e / kNB, c = e % kNB;
      lt[r][c] = (ib + r < l) ? L[(size_t)(ib + r) * lda + kbk + c] : 0.0;
      xt[r][c] = X[(size_t)(kbk + r) * lda + jb + c];
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int r = e / kNB, c = e % kNB;
      double s = 0.0;
      for (int t = 0; t < kNB; ++t) s += lt[r][t] * xt[t][c];
      acc[q] += s;
    }
    __syncthreads();
  }
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + 256 * q;
    sacc[e / kNB][e % kNB] = acc[q];
  }
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, c = e % kNB;
    lt[r][c] = (ib + r < l && ib + c < l) ? X[(size_t)(ib + r) * lda + ib + c] : 0.0;
  }
  __syncthreads();
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + 256 * q;
    const int r = e / kNB, c = e % kNB;
    if (ib + r < l) {
      double s = 0.0;
      for (int t = 0; t < kNB; ++t) s += lt[r][t] * sacc[t][c];
      X[(size_t)(ib + r) * lda + jb + c] = -s;
    }
  }
}

// M = X^T X for lower-triangular X (l x l), both triangles written; one 32 x 32 tile of the
// lower triangle per block (mirrored).  Rows of X below the tiles' columns only.
__global__ void __launch_bounds__(256) k_xtx(const double* __restrict__ X, int lda, int l,
                                             double* __restrict__ M) {
  __shared__ double xa[kNB][kNB + 1], xb[kNB][kNB + 1];
  const int b = blockIdx.x;
  int A = (int)((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
  while ((A + 1) * (A + 2) / 2 <= b) ++A;
  while (A * (A + 1) / 2 > b) --A;
  const int Bt = b - A * (A + 1) / 2;
  const int ab = A * kNB, bb = Bt * kNB;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int nblk = (l + kNB - 1) / kNB;
  for (int K = A; K < nblk; ++K) {  // X[i][a] = 0 for i < a
    const int kb = K * kNB;
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
      const int r = e / kNB, c = e % kNB;
      const bool in = kb + r < l;
      xa[r][c] = (in && ab + c < l) ? X[(size_t)(kb + r) * lda + ab + c] : 0.0;
      xb[r][c] = (in && bb + c < l) ? X[(size_t)(kb + r) * lda + bb + c] : 0.0;
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int r = e / kNB, c = e % kNB;
      double s = 0.0;
      for (int t = 0; t < kNB; ++t) s += xa[t][r] * xb[t][c];
      acc[q] += s;
    }
    __syncthreads();
  }
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + 256 * q;
    const int r = e / kNB, c = e % kNB;
    const int i = ab + r, j = bb + c;
    if (i < l && j < l) {
      M[(size_t)i * lda + j] = acc[q];
      M[(size_t)j * lda + i] = acc[q];
    }
  }
}

// y = M v (M symmetric l x l, fp64): one warp per row.
__global__ void k_symv(const double* __restrict__ M, int lda, int l, const double* __restrict__ v,
                       double* __restrict__ y) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= l) return;
  double s = 0.0;
  for (int j = lane; j < l; j += 32) s += M[(size_t)row * lda + j] * v[j];
  for (int o = 16; o >= 1; o /= 2) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

// Power-iteration step for the largest eigenvalue of M (v unit): rq = v^T y, v <- y / |y|.
// One block of 1024 threads; v0 != 0 on entry.
__global__ void k_power_step(double* __restrict__ v, const double* __restrict__ y, int l,
                             double* __restrict__ rq) {
  __shared__ double s1[1024], s2[1024];
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < l; j += blockDim.x) {
    a += v[j] * y[j];
    b += y[j] * y[j];
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int h = blockDim.x / 2; h >= 1; h /= 2) {
    if ((int)threadIdx.x < h) {
      s1[threadIdx.x] += s1[threadIdx.x + h];
      s2[threadIdx.x] += s2[threadIdx.x + h];
    }
    __syncthreads();
  }
  const double inv = s2[0] > 0.0 ? 1.0 / sqrt(s2[0]) : 0.0;
  for (int j = threadIdx.x; j < l; j += blockDim.x) v[j] = y[j] * inv;
  if (threadIdx.x == 0) *rq = s1[0];
}

__global__ void k_init_unit(double* __restrict__ v, int l) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < l) v[j] = 1.0 / sqrt((double)l) * (1.0 + 0.25 * sin(0.7 * j));
}

// Round a panel to bf16 in place (the fp32 copy then holds the bf16 values exactly) and
// write the bf16 copy.
__global__ void k_round_bf16(float* __restrict__ P, int64_t count, __nv_bfloat16* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const __nv_bfloat16 b = __float2bfloat16_rn(P[e]);
  out[e] = b;
  P[e] = __bfloat162float(b);
}

// out[i][j] = (float)A[i][j] for i, j < l, 0 elsewhere in [ld][ld].
__global__ void k_to_f32_pad(const double* __restrict__ A, int lda, int l, int ld,
                             float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ld * ld) return;
  const int i = (int)(e / ld), j = (int)(e % ld);
  out[e] = (i < l && j < l) ? (float)A[(size_t)i * lda + j] : 0.f;
}

// A[i][j] = src[i][j] + d (i == j) on the l x l block.
__global__ void k_copy_shift(const double* __restrict__ src, double* __restrict__ A, int lda,
                             int l, double d) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)l * l) return;
  const int i = (int)(e / l), j = (int)(e % l);
  A[(size_t)i * lda + j] = src[(size_t)i * lda + j] + (i == j ? d : 0.0);
}

}  // namespace

// ---- host side ----------------------------------------------------------------------------
namespace {

struct Dense {
  int l, lda;
  cudaStream_t st;
  int* status;  // device
  // In-place lower Cholesky of A (already symmetrised); returns false on a failed pivot.
  bool chol(double* A, bool& ok_out, cudaError_t& err) {
    err = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (err != cudaSuccess) return false;
    for (int kb = 0; kb < l; kb += kNB) {
      const int nb = std::min(kNB, l - kb);
      k_potrf_diag<<<1, 256, 0, st>>>(A, lda, kb, nb, status);
      note_launches(1);
      const int rest = l - kb - nb;
      if (rest > 0) {
        k_trsm_panel<<<(unsigned)ceil_div(rest, 128), 128, 0, st>>>(A, lda, l, kb, nb);
        const int64_t T = ceil_div(rest, kNB);
        k_syrk_trailing<<<(unsigned)(T * (T + 1) / 2), 256, 0, st>>>(A, lda, l, kb, nb);
        note_launches(2);
      }
    }
    int hs = 0;
    err = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    ok_out = hs == 0;
    return err == cudaSuccess;
  }
  // X = L^-1 (lower), X zero above the diagonal.
  cudaError_t trtri(const double* L, double* X) {
    cudaError_t e = cudaMemsetAsync(X, 0, (size_t)lda * lda * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const int nblk = (l + kNB - 1) / kNB;
    k_trtri_diag<<<nblk, kNB, 0, st>>>(L, X, lda, l);
    note_launches(1);
    for (int I = 1; I < nblk; ++I) {
      k_trtri_row<<<I, 256, 0, st>>>(L, X, lda, l, I);
      note_launches(1);
    }
    return cudaGetLastError();
  }
  cudaError_t xtx(const double* X, double* M) {
    const int64_t nblk = (l + kNB - 1) / kNB;
    k_xtx<<<(unsigned)(nblk * (nblk + 1) / 2), 256, 0, st>>>(X, lda, l, M);
    note_launches(1);
    return cudaGetLastError();
  }
};

}  // namespace

sgp_status ShiftedNystrom::build(Lattice* L, int rank, uint64_t seed, float noise, int blur,
                                 int power_iters, cudaStream_t st) {
  const int64_t n = L->n;
  l = rank;
  ld = (int)ceil_div(rank, kTile) * kTile;
  this->n = n;
  ok = false;
#define PC_CHECK(expr, what)                                  \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return cuda_status(e_, what);      \
  } while (0)
  std::vector<void*> temps;
  struct Free {
    std::vector<void*>& t;
    cudaStream_t st;
    ~Free() {
      for (void* p : t) (void)cudaFreeAsync(p, st);
    }
  } free_temps{temps, st};
  auto keep = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  };
  auto temp = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) temps.push_back(*p);
    return e;
  };
  {  // dynamic shared memory above 48 KB, once per device
    static std::atomic<bool> attrs[64];
    int dev = 0;
    PC_CHECK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev >= 0 && dev < 64 && !attrs[dev].load()) {
      PC_CHECK(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    4 * kKc * kSMN * (int)sizeof(float)),
               "k_gram_tc smem");
      PC_CHECK(cudaFuncSetAttribute(k_panel_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    4 * kTile * kSK * (int)sizeof(float)),
               "k_panel_tc smem");
      PC_CHECK(cudaFuncSetAttribute(k_bt_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kApplyStages * kBtStageBytes),
               "k_bt_bf16 smem");
      PC_CHECK(cudaFuncSetAttribute(k_apply_z_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kApplyStages * kZStageBytes),
               "k_apply_z_bf16 smem");
      attrs[dev].store(true);
    }
  }
  const size_t panel = (size_t)n * ld * sizeof(float);
  float *P1 = nullptr, *P2 = nullptr, *Vc = nullptr, *KVc = nullptr, *gpart = nullptr,
        *Tt = nullptr;
  double *G = nullptr, *G0 = nullptr, *Xi = nullptr, *M = nullptr, *pv = nullptr, *py = nullptr,
         *prq = nullptr;
  int* status = nullptr;
  PC_CHECK(keep((void**)&B, (size_t)n * ld * sizeof(__nv_bfloat16)),
           "alloc preconditioner B");
  PC_CHECK(temp((void**)&P1, panel), "alloc preconditioner panel");
  PC_CHECK(temp((void**)&P2, panel), "alloc preconditioner panel");
  PC_CHECK(temp((void**)&Vc, (size_t)n * kSketchCols * sizeof(float)), "alloc sketch chunk");
  PC_CHECK(temp((void**)&KVc, (size_t)n * kSketchCols * sizeof(float)), "alloc sketch chunk");
  const int ntile = ld / kTile;
  // row splits of the Grams: at most 64 k rows per split, at least 2 waves of blocks
  int splits = (int)std::max<int64_t>(ceil_div(n, 65536),
                                      ceil_div(2 * 2 * 152, ntile * (ntile + 1) / 2));
  splits = (int)std::min<int64_t>(splits, std::max<int64_t>(1, ceil_div(n, kKc)));
  const int64_t rows_per_split = ceil_div(ceil_div(n, splits), kKc) * kKc;
  splits = (int)ceil_div(n, rows_per_split);
  const size_t ll = (size_t)ld * ld;
  PC_CHECK(temp((void**)&gpart, (size_t)splits * ll * sizeof(float)), "alloc Gram partials");
  PC_CHECK(temp((void**)&Tt, ll * sizeof(float)), "alloc l x l");
  PC_CHECK(temp((void**)&G, ll * sizeof(double)), "alloc l x l");
  PC_CHECK(temp((void**)&G0, ll * sizeof(double)), "alloc l x l");
  PC_CHECK(temp((void**)&Xi, ll * sizeof(double)), "alloc l x l");
  PC_CHECK(temp((void**)&M, ll * sizeof(double)), "alloc l x l");
  PC_CHECK(temp((void**)&pv, ld * sizeof(double)), "alloc power vectors");
  PC_CHECK(temp((void**)&py, ld * sizeof(double)), "alloc power vectors");
  PC_CHECK(temp((void**)&prq, sizeof(double)), "alloc power vectors");
  PC_CHECK(temp((void**)&status, sizeof(int)), "alloc status");
  // per-iteration buffers
  // B^T r: one wave of the blocks the device keeps resident (i tiles x row splits)
  int bt_per_sm = 0, sms = 0, dev_now = 0;
  PC_CHECK(cudaGetDevice(&dev_now), "cudaGetDevice");
  PC_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_now), "SM count");
  PC_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
               &bt_per_sm, k_bt_bf16, 256, kApplyStages * kBtStageBytes),
           "occupancy");
  bt_splits = (int)std::max<int64_t>(
      1, std::min<int64_t>(std::max(1, bt_per_sm) * (int64_t)sms / ntile, ceil_div(n, kKc)));
  bt_rows = ceil_div(ceil_div(n, bt_splits), kKc) * kKc;
  bt_splits = (int)ceil_div(n, bt_rows);
  PC_CHECK(keep((void**)&tpart, (size_t)bt_splits * ld * 16 * sizeof(float)), "alloc B^T r");
  PC_CHECK(keep((void**)&tvec, (size_t)ld * 16 * sizeof(float)), "alloc t");
  PC_CHECK(keep((void**)&u, (size_t)3 * 16 * ld * sizeof(__nv_bfloat16)), "alloc u");
  PC_CHECK(keep((void**)&Minv, ll * sizeof(float)), "alloc Minv");
  sgp_status s = ensure_lattice_values(L, kSketchCols, st);
  if (s != SGP_OK) return s;

  Dense dn{l, ld, st, status};
  const unsigned g_panel = (unsigned)ceil_div((int64_t)n * ld, 256);
  const unsigned g_chunk = (unsigned)ceil_div((int64_t)n * kSketchCols, 256);
  // dst = outputscale K src, column chunk by chunk (padding columns of dst: zero)
  auto product = [&](const float* src, float* dst) -> sgp_status {
    for (int c0 = 0; c0 < ld; c0 += kSketchCols) {
      k_copy_cols<<<g_chunk, 256, 0, st>>>(const_cast<float*>(src), ld, c0, Vc, kSketchCols, n,
                                           false);
      enqueue_mvm(L, Vc, kSketchCols, blur, L->outputscale, 0.f, KVc, st, nullptr,
                  /*internal=*/true);
      k_copy_cols<<<g_chunk, 256, 0, st>>>(dst, ld, c0, KVc, kSketchCols, n, true);
      note_launches(2);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SGP_OK : cuda_status(e, "sketch products");
  };
  // G = X^T Y (fp64 [ld][ld])
  auto gram = [&](const float* X, const float* Y, double* out) {
    k_gram_tc<<<dim3(ntile * (ntile + 1) / 2, splits), 256, 4 * kKc * kSMN * sizeof(float),
                st>>>(X, ld, Y, ld, n, ntile, rows_per_split, ld, gpart);
    k_sum_splits<<<(unsigned)ceil_div((int64_t)ll, 256), 256, 0, st>>>(gpart, splits, ld, out);
    note_launches(2);
  };
  // Z = Y X^T for the fp64 lower-triangular X (Z[r][j] = sum_i Y[r][i] X[j][i])
  auto panel_times = [&](const float* Y, const double* X, float* Z) {
    k_to_f32_pad<<<(unsigned)ceil_div((int64_t)ll, 256), 256, 0, st>>>(X, ld, l, ld, Tt);
    k_panel_tc<<<dim3((unsigned)ceil_div(n, kTile), ntile), 256, 4 * kTile * kSK * sizeof(float),
                 st>>>(Y, ld, Tt, ld, ld, /*lower=*/true, n, Z, ld);
    note_launches(2);
  };
  // Cholesky of the symmetrised out-of-place copy of src with a relative diagonal shift,
  // raised 100-fold (at most 4 times) while a pivot fails; the factor lands in dst.
  auto robust_chol = [&](const double* src, double* dst, double rel, bool& good) -> sgp_status {
    good = false;
    for (int attempt = 0; attempt < 4 && !good; ++attempt, rel *= 100.0) {
      PC_CHECK(cudaMemcpyAsync(dst, src, ll * sizeof(double), cudaMemcpyDeviceToDevice, st),
               "copy l x l");
      k_prepare_spd<<<1, 1024, 0, st>>>(dst, l, ld, 0.0, rel);
      note_launches(1);
      cudaError_t err = cudaSuccess;
      if (!dn.chol(dst, good, err)) return cuda_status(err, "Cholesky");
    }
    return SGP_OK;
  };

  // 1. Q: the sketch, or an orthonormal basis of K Omega (Cholesky QR twice)
  k_fill_sketch_panel<<<g_panel, 256, 0, st>>>(L->perm, n, l, ld, seed, P1);
  note_launches(1);
  float* Q = P1;
  float* Y = P2;
  if (power_iters > 0) {
    if ((s = product(P1, P2)) != SGP_OK) return s;  // P2 = K Omega
    float* src = P2;
    float* dst = P1;
    for (int pass = 0; pass < 2; ++pass) {
      bool good = false;
      gram(src, src, G0);
      if ((s = robust_chol(G0, G, 1e-7, good)) != SGP_OK) return s;
      if (!good) return SGP_OK;  // ok stays false: the solve runs unpreconditioned
      PC_CHECK(dn.trtri(G, Xi), "triangular inverse");
      panel_times(src, Xi, dst);  // dst = src R^-T
      std::swap(src, dst);
    }
    Q = src;   // orthonormal basis (P2 after two passes)
    Y = dst;
    if ((s = product(Q, Y)) != SGP_OK) return s;
  } else {
    if ((s = product(P1, P2)) != SGP_OK) return s;
  }
  // 2. C = Q^T Y, C = R R^T, B = Y R^-T
  {
    bool good = false;
    gram(Q, Y, G0);
    if ((s = robust_chol(G0, G, 1e-6, good)) != SGP_OK) return s;
    if (!good) return SGP_OK;
    PC_CHECK(dn.trtri(G, Xi), "triangular inverse");
    // the factor in fp32 in Q's panel (Q is no longer needed), then rounded to bf16: the
    // stored values define P, and B^T B below is formed from them
    panel_times(Y, Xi, Q);
    k_round_bf16<<<g_panel, 256, 0, st>>>(Q, (int64_t)n * ld, static_cast<__nv_bfloat16*>(B));
    note_launches(1);
  }
  // 3. G = B^T B; lambda_min(G) by power iteration on G^-1; tau = lambda_min + noise
  double lam_min = 0.0;
  {
    gram(Q, Q, G0);
    bool good = false;
    if ((s = robust_chol(G0, G, 1e-9, good)) != SGP_OK) return s;
    if (!good) return SGP_OK;
    PC_CHECK(dn.trtri(G, Xi), "triangular inverse");
    PC_CHECK(dn.xtx(Xi, M), "inverse");
    k_init_unit<<<(unsigned)ceil_div(l, 256), 256, 0, st>>>(pv, l);
    note_launches(1);
    constexpr int kPowerSteps = 30;
    for (int it = 0; it < kPowerSteps; ++it) {
      k_symv<<<(unsigned)ceil_div(l, 8), 256, 0, st>>>(M, ld, l, pv, py);
      k_power_step<<<1, 1024, 0, st>>>(pv, py, l, prq);
      note_launches(2);
    }
    double rq = 0.0;
    PC_CHECK(cudaMemcpyAsync(&rq, prq, sizeof(double), cudaMemcpyDeviceToHost, st), "read rq");
    PC_CHECK(cudaStreamSynchronize(st), "sync power iteration");
    lam_min = rq > 0.0 ? 1.0 / rq : 0.0;
  }
  tau = (float)(lam_min + (double)noise);
  // 4. Minv = (tau I + G)^-1 (fp64 Cholesky, inverse factor, product), stored fp32
  {
    k_copy_shift<<<(unsigned)ceil_div((int64_t)l * l, 256), 256, 0, st>>>(G0, M, ld, l,
                                                                          (double)tau);
    note_launches(1);
    bool good = false;
    if ((s = robust_chol(M, G, 0.0, good)) != SGP_OK) return s;
    if (!good) return SGP_OK;
    PC_CHECK(dn.trtri(G, Xi), "triangular inverse");
    PC_CHECK(dn.xtx(Xi, M), "inverse");
    k_to_f32_pad<<<(unsigned)ceil_div((int64_t)ll, 256), 256, 0, st>>>(M, ld, l, ld, Minv);
    note_launches(1);
  }
  PC_CHECK(cudaGetLastError(), "building the preconditioner");
  PC_CHECK(cudaStreamSynchronize(st), "sync preconditioner");
  ok = true;
  return SGP_OK;
#undef PC_CHECK
}

int64_t ShiftedNystrom::dot_blocks() const { return ceil_div(n, kTile); }

void ShiftedNystrom::apply(const float* rh, const float* rl, int k, float* z, double* dot,
                           cudaStream_t st, cudaEvent_t* ev) const {
  const int ntile = ld / kTile;
  for (int c_off = 0; c_off < k; c_off += 16) {
    const int kc = std::min(16, k - c_off);
    // with ev (inside a capture: external record nodes) the first 16-column chunk's
    // B^T r and z kernels are bracketed for the stage timings
    const bool mark = ev && c_off == 0;
    if (mark) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
    k_bt_bf16<<<dim3(ntile, bt_splits), 256, kApplyStages * kBtStageBytes, st>>>(
        static_cast<const __nv_bfloat16*>(B), ld, rh, rl, k, c_off, kc, n, bt_rows, tpart);
    if (mark) cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
    k_sum_t<<<(unsigned)ceil_div(ld * 16, 256), 256, 0, st>>>(tpart, bt_splits, ld, tvec);
    k_minv_u<<<(unsigned)ceil_div(ld * 16, 256), 256, 0, st>>>(
        Minv, ld, tvec, static_cast<__nv_bfloat16*>(u));
    if (mark) cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal);
    k_apply_z_bf16<<<(unsigned)ceil_div(n, kTile), 256, kApplyStages * kZStageBytes, st>>>(
        static_cast<const __nv_bfloat16*>(B), ld, static_cast<const __nv_bfloat16*>(u), rh, rl,
        k, c_off, kc, n, 1.f / tau, z, dot);
    if (mark) cudaEventRecordWithFlags(ev[3], st, cudaEventRecordExternal);
    note_launches(4);
  }
}

void ShiftedNystrom::release(cudaStream_t st) {
  for (void* p : ptrs) (void)cudaFreeAsync(p, st);
  ptrs.clear();
}

}  // namespace sgp
