// Large-rank Nystrom preconditioner for the library CG (App. A: CG pre-conditioner; the
// rank a system needs grows with its conditioning).
//
// With A = K + noise I (K = outputscale W M^T M W^T, reachable only through products):
//   Omega   n x l Rademacher sketch, entry (i, j) = sign bit of SplitMix64 at counter
//           i l + j + 1 from the seed (i = the caller's point index);
//   Q       Omega, or after q = 1 subspace iteration a basis of the range of K Omega
//           (Cholesky QR; the approximation depends only on the subspace, so a second
//           pass runs only when the first Gram's Cholesky needed a raised shift, and the
//           product K Omega runs on bf16 lattice values);
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
// All tall n x l products run on the fifth-generation tensor cores (tcgen05.mma, kind::f16,
// fp32 accumulators in tensor memory, operands staged by TMA; see tc05.cuh):
//   - set-up: the panels are kept as three bf16 planes (x = x1 + x2 + x3, about 24 bits);
//     the Grams Q^T Y, Y^T Y and the panel products Y X^T take the six plane products
//     x_a y_b with a + b <= 2; B^T B of the stored bf16 factor is one exact product;
//     fp32 sums inside a block, fp64 sums across blocks in a fixed order;
//   - per iteration: B^T r and B u with the exact bf16 B and r, u split in three bf16
//     parts.  The apply reads the bf16 factor twice, 2 n ld bytes each (half of an fp32
//     factor).  With tau well above the noise the bf16 rounding of B (a perturbation of
//     order 2^-9 ||B||^2 / sqrt(l) of B B^T, small against tau) leaves the iteration counts
//     unchanged (measured at n = 2M, ranks 1024 and 2048).
// The l x l factorizations (Cholesky, triangular inverse, products) run in fp64 on the CUDA
// cores in 32 x 32 blocks; the triangular inverse joins inverted diagonal blocks pairwise,
// level by level, so its dependent chain is O(l / 32) tile products instead of O((l / 32)^2).  Panels are [n][ld] in the lattice's locality order, ld = l
// rounded up to 128, padding columns zero.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include "sgp_internal.cuh"
#include "tc05.cuh"
#include "values.cuh"

namespace sgp {
namespace {

constexpr int kTile = 128;     // M and N tile of the tensor-core products
constexpr int kSketchCols = 128;  // sketch columns per lattice product
constexpr int kNB = 32;        // block size of the fp64 factorizations

// SplitMix64 (Steele, Lea & Flood 2014) at counter i l + j + 1: one +-1 per (point, column).
__device__ __forceinline__ float sketch_sign(uint64_t seed, int64_t i, int j, int l) {
  uint64_t z = seed + ((uint64_t)(i * l + j) + 1ull) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (z >> 63) ? -1.f : 1.f;
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

// ---- per-iteration apply on the fifth-generation tensor cores ----------------------------
// B holds bf16 values exactly, so B^T r and B u are tcgen05 MMAs (kind::f16, bf16 operands,
// fp32 accumulators in tensor memory) with B as the exact operand and r, u split in three
// bf16 parts x = x1 + x2 + x3 (about 24 bits), stacked along N: the 16 columns of each part
// make N = 48, and the epilogue adds the three 16-column blocks (x3 + x2 first, then x1).
// Operand tiles arrive by TMA (128-byte swizzle) in a ring of kTcStages stages; one thread
// issues the loads and the MMAs, four warps run the epilogue from tensor memory.
//
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

constexpr int kTcStages = 4;
constexpr int kTcRows = 64;                   // K rows (bt) or K columns (z) per stage
constexpr int kTcBoxA = 128 * 128;            // bytes of a 128 x 64 bf16 operand tile
constexpr int kTcBoxU = 48 * 128;             // bytes of the 48 x 64 bf16 parts of u
constexpr int kTcBoxR = 64 * 128;             // bytes of 64 rows of the split r ([n][64])
constexpr int kTcStage = kTcBoxA + kTcBoxU;   // z: 22 KB (a multiple of the 1 KB atom)
constexpr int kBtStage = kTcBoxA + kTcBoxR;   // B^T r: 24 KB
constexpr long long kTcSpin = 1ll << 20;      // polls per bounded wait
constexpr int kTcThreads = 160;               // warp 0: issue; warps 1-4: epilogue

// r3[row][part * 16 + c] = part `part` of (rh + rl)[row][c_off + c] for c < kc (else 0):
// the split right-hand side as rows of 64 bf16 (columns 48..63 stay zero), MN-major for
// the B^T r MMAs.  One row per thread, 16-byte stores.  (The CG's x, r update writes the
// first 16 columns' split itself; this kernel serves the CG start and further chunks.)
__global__ void k_split_r(const float* __restrict__ rh, const float* __restrict__ rl, int k,
                          int c_off, int kc, int64_t n, __nv_bfloat16* __restrict__ r3) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  uint32_t w[3][8];
#pragma unroll
  for (int c2 = 0; c2 < 8; ++c2) {
    __nv_bfloat16 p[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = 2 * c2 + h;
      float x = 0.f;
      if (c < kc) {
        const int64_t e = row * k + c_off + c;
        x = __fadd_rn(rh[e], rl[e]);
      }
      split3(x, p[h][0], p[h][1], p[h][2]);
    }
#pragma unroll
    for (int part = 0; part < 3; ++part) w[part][c2] = pack2(p[0][part], p[1][part]);
  }
  uint4* o = reinterpret_cast<uint4*>(r3 + row * 64);
#pragma unroll
  for (int part = 0; part < 3; ++part) {
    o[2 * part] = make_uint4(w[part][0], w[part][1], w[part][2], w[part][3]);
    o[2 * part + 1] = make_uint4(w[part][4], w[part][5], w[part][6], w[part][7]);
  }
}

// t[i][c] = sum over splits of tpart[s][i][c] (fp64 in split order, stored fp32), i < ld.
// The loads of eight splits are issued together (they are independent) before their sums.
__global__ void k_sum_t(const float* __restrict__ tpart, int splits, int ld,
                        float* __restrict__ t) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ld * 16) return;
  const size_t stride = (size_t)ld * 16;
  double s = 0.0;
  for (int q0 = 0; q0 < splits; q0 += 8) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = q0 + j < splits ? tpart[(q0 + j) * stride + e] : 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += (double)v[j];
  }
  t[e] = (float)s;
}

// u[i][c] = sum_j Minv[i][j] t[j][c] (fp32), i < ld, c < 16: one warp per row i, lane q
// takes j = 32 q' + q (coalesced reads of the row), then a fixed butterfly over the lanes.
// Stored split in three bf16 parts, transposed: u3[part][c][i] (the K-major [48][ld]
// operand).
__global__ void __launch_bounds__(256) k_minv_u(const float* __restrict__ Minv, int ld,
                                                const float* __restrict__ t,
                                                __nv_bfloat16* __restrict__ u3) {
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= ld) return;
  const float* row = Minv + (size_t)i * ld;
  float acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.f;
  for (int j = lane; j < ld; j += 32) {
    const float m = row[j];
    const float4* tj = reinterpret_cast<const float4*>(t + (size_t)j * 16);
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
      const float4 v = tj[c4];
      acc[4 * c4] = fmaf(m, v.x, acc[4 * c4]);
      acc[4 * c4 + 1] = fmaf(m, v.y, acc[4 * c4 + 1]);
      acc[4 * c4 + 2] = fmaf(m, v.z, acc[4 * c4 + 2]);
      acc[4 * c4 + 3] = fmaf(m, v.w, acc[4 * c4 + 3]);
    }
  }
#pragma unroll
  for (int c = 0; c < 16; ++c)
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
  if (lane < 16) {
    float sum = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c)
      if (c == lane) sum = acc[c];
    __nv_bfloat16 a, b, d;
    split3(sum, a, b, d);
    u3[(size_t)(0 * 16 + lane) * ld + i] = a;
    u3[(size_t)(1 * 16 + lane) * ld + i] = b;
    u3[(size_t)(2 * 16 + lane) * ld + i] = d;
  }
}

// Block-wide pieces shared by the two kernels: barrier set-up, tensor-memory allocation and
// the AND over the four epilogue warps (named barrier 1).
__device__ __forceinline__ bool epilogue_and(bool v) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbarrier.red.and.pred q, 1, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"((uint32_t)v)
      : "memory");
  return out != 0;
}
__device__ __forceinline__ void epilogue_sync() {
  asm volatile("bar.sync 1, 128;" ::: "memory");
}
// A ring of S shared-memory stages of SB bytes (1 KB aligned) with its mbarriers, the
// tensor-memory slot and the block's abort word.
template <int S, int SB>
struct TcRing {
  static constexpr int kStages = S;
  static constexpr int kStageBytes = SB;
  static constexpr int kSmem = S * SB + 1024 /* alignment */ + 256 /* barriers */;
  uint8_t* stage;   // S x SB bytes
  uint64_t* full;   // [S] TMA -> MMA
  uint64_t* empty;  // [S] MMA -> TMA
  uint64_t* accf;   // [2] MMAs of an accumulator done -> epilogue
  uint64_t* acce;   // [2] epilogue done with an accumulator -> MMA (128 arrivals)
  uint32_t* tslot;
  int* abort;
  __device__ uint8_t* at(int64_t g) const { return stage + (int)(g % S) * SB; }
  __device__ uint64_t* full_of(int64_t g) const { return &full[g % S]; }
  __device__ uint64_t* empty_of(int64_t g) const { return &empty[g % S]; }
  __device__ static uint32_t parity(int64_t g) { return (uint32_t)(g / S) & 1u; }
};
template <class Ring>
__device__ __forceinline__ Ring tc_ring(uint8_t* raw) {
  Ring R;
  R.stage = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) &
                                       ~static_cast<uintptr_t>(1023));
  R.full = reinterpret_cast<uint64_t*>(R.stage + Ring::kStages * Ring::kStageBytes);
  R.empty = R.full + Ring::kStages;
  R.accf = R.empty + Ring::kStages;
  R.acce = R.accf + 2;
  R.tslot = reinterpret_cast<uint32_t*>(R.acce + 2);
  R.abort = reinterpret_cast<int*>(R.tslot + 1);
  return R;
}
template <class Ring>
__device__ __forceinline__ void tc_setup(const Ring& R, uint32_t tmem_cols) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < Ring::kStages; ++s) {
      tc05::mbar_init(&R.full[s], 1);
      tc05::mbar_init(&R.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc05::mbar_init(&R.accf[b], 1);
      tc05::mbar_init(&R.acce[b], 128);
    }
    *R.abort = 0;
    tc05::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc05::tmem_alloc(R.tslot, tmem_cols);
  tc05::fence_before_sync();
  __syncthreads();
  tc05::fence_after_sync();
}
// The issuing thread after a wait gave up (or the epilogue aborted): wait, bounded and
// without the abort check, for the loads still in flight and for the last committed MMAs,
// so that nothing lands in shared or tensor memory after the block exits.
template <class Ring>
__device__ __forceinline__ void tc_drain(const Ring& R, int64_t landed, int64_t issued,
                                         int64_t committed) {
  for (int64_t g = landed; g < issued; ++g)
    (void)tc05::mbar_wait(R.full_of(g), Ring::parity(g), kTcSpin);
  if (committed >= 0)
    (void)tc05::mbar_wait(R.empty_of(committed), Ring::parity(committed), kTcSpin);
}
using ApplyRing = TcRing<kTcStages, kTcStage>;  // z
using BtRing = TcRing<kTcStages, kBtStage>;       // B^T r

// Per-iteration B^T r for 16 columns of r (split in r3): tpart[s][i][c] = sum over the rows
// of split s (blockIdx.y) of B[row][i] r[row][c], i in the 128-column tile blockIdx.x.
// Both operands are MN-major: the TMA boxes of B are 64 rows (K) x 64 columns (M), two per
// stage (columns i0 .. + 63, i0 + 64 .. + 127: leading offset 8 KB); the box of r3 is 64
// rows x its 64 columns (N = 64: the three 16-column parts and 16 zero columns).
// rows_per_split is a multiple of 64; rows >= n read as zero.
__global__ void __launch_bounds__(kTcThreads, 1)
    k_bt_tc(const __grid_constant__ CUtensorMap mapBt, const __grid_constant__ CUtensorMap mapR,
            int64_t n, int64_t rows_per_split, float* __restrict__ tpart, int* __restrict__ err) {
  extern __shared__ uint8_t tc_raw[];
  const BtRing R = tc_ring<BtRing>(tc_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * 128;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r_end = std::min<int64_t>(n, r_begin + rows_per_split);
  const int64_t total = r_end > r_begin ? ceil_div(r_end - r_begin, kTcRows) : 0;
  constexpr uint32_t kIdesc = tc05::idesc_bf16(128, 64, /*a_mn=*/true, /*b_mn=*/true);
  if (*reinterpret_cast<volatile int*>(err)) return;  // an earlier launch gave up: skip
  if (threadIdx.x == 0) {
    tc05::prefetch_map(&mapBt);
    tc05::prefetch_map(&mapR);
  }
  tc_setup(R, 64);
  const uint32_t tmem = *R.tslot;
  volatile int* abort = R.abort;
  if (warp == 0) {
    if (lane == 0) {
      int64_t issued = 0, landed = 0, committed = -1;
      auto issue = [&](int64_t g) {
        uint8_t* st = R.at(g);
        const int row0 = (int)(r_begin + g * kTcRows);
        tc05::mbar_expect_tx(R.full_of(g), kBtStage);
        tc05::tma_load_2d(st, &mapBt, i0, row0, R.full_of(g));
        tc05::tma_load_2d(st + kTcBoxA / 2, &mapBt, i0 + 64, row0, R.full_of(g));
        tc05::tma_load_2d(st + kTcBoxA, &mapR, 0, row0, R.full_of(g));
        issued = g + 1;
      };
      for (int64_t g = 0; g < total && g < kTcStages; ++g) issue(g);
      bool ok = true;
      for (int64_t g = 0; g < total; ++g) {
        if (!tc05::mbar_wait(R.full_of(g), BtRing::parity(g), kTcSpin, abort)) {
          ok = false;
          break;
        }
        landed = g + 1;
        tc05::fence_after_sync();
        const uint32_t a0 = tc05::smem_u32(R.at(g)), b0 = a0 + kTcBoxA;
#pragma unroll
        for (int kk = 0; kk < kTcRows / 16; ++kk)
          tc05::mma_bf16(tmem, tc05::desc_sw128(a0 + kk * 2048, kTcBoxA / 2, 1024),
                         tc05::desc_sw128(b0 + kk * 2048, kTcBoxR, 1024), kIdesc,
                         (g | kk) ? 1u : 0u);
        tc05::mma_commit(R.empty_of(g));
        committed = g;
        // refill the previous chunk's stage once its MMAs are done
        if (g >= 1 && g - 1 + kTcStages < total) {
          const int64_t p = g - 1;
          if (!tc05::mbar_wait(R.empty_of(p), BtRing::parity(p), kTcSpin, abort)) {
            ok = false;
            break;
          }
          issue(p + kTcStages);
        }
      }
      if (ok) {
        tc05::mma_commit(&R.accf[0]);
      } else {
        *abort = 1;
        atomicExch(err, 1);
        tc_drain(R, landed, issued, committed);
      }
    }
  } else {
    const int q = warp & 3;  // tensor-memory lanes 32 q .. + 31 = rows i0 + 32 q + lane
    bool ok = true;
    if (total > 0) {
      ok = tc05::mbar_wait(&R.accf[0], 0u, kTcSpin, abort);
      ok = epilogue_and(ok);
    }
    if (!ok) {
      if (threadIdx.x == 32) {
        *abort = 1;
        atomicExch(err, 1);
      }
    } else {
      float t[16];
      if (total > 0) {
        tc05::fence_after_sync();
        float d1[16], d2[16], d3[16];
        const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16);
        tc05::tmem_ld16(ta, d1);
        tc05::tmem_ld16(ta + 16, d2);
        tc05::tmem_ld16(ta + 32, d3);
        tc05::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) t[c] = d1[c] + (d2[c] + d3[c]);
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) t[c] = 0.f;
      }
      float4* out = reinterpret_cast<float4*>(
          tpart + ((size_t)blockIdx.y * gridDim.x * 128 + i0 + 32 * q + lane) * 16);
#pragma unroll
      for (int c = 0; c < 4; ++c)
        out[c] = make_float4(t[4 * c], t[4 * c + 1], t[4 * c + 2], t[4 * c + 3]);
    }
  }
  tc05::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, 64);
}

// z[r][c_off + c] = (r - B u)[r][c] * inv_tau over 128-row tiles (tile t: rows 128 t ..),
// and the column sums of r z (fp64; the products are exact in fp64) over each block's
// tiles, in tile order, into dot[blockIdx.x][c_off + c].  Persistent: block b takes tiles b, b + gridDim.x, ..., with two
// accumulators in tensor memory so that the MMAs of one tile overlap the epilogue of the
// previous.  A = B is K-major (boxes 128 rows x 64 columns); u3 ([48][ld], the three parts
// of u = Minv B^T r) is K-major (boxes 48 x 64).  r enters rounded to fp32, which is the
// high word rh of the CG's double-float residual: the CG keeps its pairs normalised (each
// update ends in a FastTwoSum, so fl(hi + lo) = hi), and the low words are not read.
__global__ void __launch_bounds__(kTcThreads, 1)
    k_z_tc(const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapU,
           const float* __restrict__ rh, int k, int c_off, int kc, int64_t n, int ld,
           float inv_tau, float* __restrict__ z, double* __restrict__ dot,
           int* __restrict__ err) {
  extern __shared__ uint8_t tc_raw[];
  __shared__ double red[2][4][16];
  const ApplyRing R = tc_ring<ApplyRing>(tc_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = ceil_div(n, 128);
  const int nk = ld / kTcRows;
  const int64_t my_tiles =
      (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = my_tiles * nk;
  constexpr uint32_t kIdesc = tc05::idesc_bf16(128, 48, /*a_mn=*/false, /*b_mn=*/false);
  if (*reinterpret_cast<volatile int*>(err)) return;  // an earlier launch gave up: skip
  if (threadIdx.x == 0) {
    tc05::prefetch_map(&mapB);
    tc05::prefetch_map(&mapU);
  }
  tc_setup(R, 128);
  const uint32_t tmem = *R.tslot;
  volatile int* abort = R.abort;
  if (warp == 0) {
    if (lane == 0) {
      int64_t issued = 0, landed = 0, committed = -1;
      auto issue = [&](int64_t g) {
        uint8_t* st = R.stage + (g % kTcStages) * kTcStage;
        const int64_t tile = blockIdx.x + (g / nk) * (int64_t)gridDim.x;
        const int kq = (int)(g % nk);
        tc05::mbar_expect_tx(&R.full[g % kTcStages], kTcStage);
        tc05::tma_load_2d(st, &mapB, kq * kTcRows, (int)(tile * 128), &R.full[g % kTcStages]);
        tc05::tma_load_2d(st + kTcBoxA, &mapU, kq * kTcRows, 0, &R.full[g % kTcStages]);
        issued = g + 1;
      };
      for (int64_t g = 0; g < total && g < kTcStages; ++g) issue(g);
      bool ok = true;
      for (int64_t j = 0; j < my_tiles && ok; ++j) {
        const int b = (int)(j & 1);
        if (j >= 2 && !tc05::mbar_wait(&R.acce[b], (uint32_t)((j - 2) >> 1) & 1u, kTcSpin,
                                       abort)) {
          ok = false;
          break;
        }
        tc05::fence_after_sync();
        for (int kq = 0; kq < nk; ++kq) {
          const int64_t g = j * nk + kq;
          const int s = (int)(g % kTcStages);
          if (!tc05::mbar_wait(&R.full[s], (uint32_t)(g / kTcStages) & 1u, kTcSpin, abort)) {
            ok = false;
            break;
          }
          landed = g + 1;
          tc05::fence_after_sync();
          const uint32_t a0 = tc05::smem_u32(R.stage + s * kTcStage), b0 = a0 + kTcBoxA;
#pragma unroll
          for (int kk = 0; kk < kTcRows / 16; ++kk)
            tc05::mma_bf16(tmem + 64 * b, tc05::desc_sw128(a0 + kk * 32, 16, 1024),
                           tc05::desc_sw128(b0 + kk * 32, 16, 1024), kIdesc,
                           (kq | kk) ? 1u : 0u);
          tc05::mma_commit(&R.empty[s]);
          committed = g;
          if (kq == nk - 1) tc05::mma_commit(&R.accf[b]);
          if (g >= 1 && g - 1 + kTcStages < total) {
            const int64_t p = g - 1;
            if (!tc05::mbar_wait(&R.empty[p % kTcStages], (uint32_t)(p / kTcStages) & 1u,
                                 kTcSpin, abort)) {
              ok = false;
              break;
            }
            issue(p + kTcStages);
          }
        }
      }
      if (!ok) {
        *abort = 1;
        atomicExch(err, 1);
        tc_drain(R, landed, issued, committed);
      }
    }
  } else {
    const int q = warp & 3;  // tensor-memory lanes 32 q .. + 31
    const bool vec = (k & 3) == 0 && (c_off & 3) == 0;
    double blk = 0.0;  // warp 1, lane c: the block's column sum over its tiles, in order
    for (int64_t j = 0; j < my_tiles; ++j) {
      const int b = (int)(j & 1);
      const int64_t tile = blockIdx.x + j * (int64_t)gridDim.x;
      bool ok = tc05::mbar_wait(&R.accf[b], (uint32_t)(j >> 1) & 1u, kTcSpin, abort);
      ok = epilogue_and(ok);
      if (!ok) {
        if (threadIdx.x == 32) {
          *abort = 1;
          atomicExch(err, 1);
        }
        break;
      }
      tc05::fence_after_sync();
      float d1[16], d2[16], d3[16];
      const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + 64u * b;
      tc05::tmem_ld16(ta, d1);
      tc05::tmem_ld16(ta + 16, d2);
      tc05::tmem_ld16(ta + 32, d3);
      tc05::tmem_wait_ld();
      tc05::fence_before_sync();
      tc05::mbar_arrive(&R.acce[b]);
      const int64_t row = tile * 128 + 32 * q + lane;
      double pr[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) pr[c] = 0.0;
      if (row < n) {
        float rv[16];
        const int64_t e0 = row * k + c_off;
        if (vec) {
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4)
            if (4 * c4 < kc) {
              const float4 h = *reinterpret_cast<const float4*>(rh + e0 + 4 * c4);
              rv[4 * c4] = h.x;
              rv[4 * c4 + 1] = h.y;
              rv[4 * c4 + 2] = h.z;
              rv[4 * c4 + 3] = h.w;
            }
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (c < kc) rv[c] = rh[e0 + c];
        }
        float zz[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          zz[c] = 0.f;
          if (c < kc) {
            zz[c] = (rv[c] - (d1[c] + (d2[c] + d3[c]))) * inv_tau;
            pr[c] = (double)rv[c] * (double)zz[c];
          }
        }
        if (vec) {
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4)
            if (4 * c4 < kc)
              *reinterpret_cast<float4*>(z + e0 + 4 * c4) =
                  make_float4(zz[4 * c4], zz[4 * c4 + 1], zz[4 * c4 + 2], zz[4 * c4 + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (c < kc) z[e0 + c] = zz[c];
        }
      }
      // column sums over the tile's rows: butterfly within each warp, then the four
      // quarters in row order
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        double v = pr[c];
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        if (lane == 0) red[b][q][c] = v;
      }
      epilogue_sync();
      if (warp == 1 && lane < kc)
        blk += ((red[b][0][lane] + red[b][1][lane]) + red[b][2][lane]) + red[b][3][lane];
    }
    if (warp == 1 && lane < kc) dot[(int64_t)blockIdx.x * k + c_off + lane] = blk;
  }
  tc05::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, 128);
}

// ---- set-up panels on the fifth-generation tensor cores ----------------------------------
// The set-up's n x ld panels are kept as three bf16 planes [3][n][ld] holding the parts of
// an fp32 value x = x1 + x2 + x3 (split3: about 24 significant bits, as fp32).  The Grams
// X^T Y and the panel products Y T^T then run as tcgen05 MMAs over plane pairs: the six
// products x_a y_b with a + b <= 2 (the dropped ones are below 2^-24 relative), smallest
// first, all accumulated in one fp32 tensor-memory accumulator.  Operand tiles arrive by
// 3D TMA loads (one box per operand tile covers all planes).

// P3[.][p][j]: plane 0 = Omega[perm[p]][j] for j < l, 0 for l <= j < ld; planes 1, 2 = 0.
// Eight columns per thread (16-byte stores).
__global__ void k_fill_sketch3(const int32_t* __restrict__ perm, int64_t n, int l, int ld,
                               uint64_t seed, __nv_bfloat16* __restrict__ P3) {
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
  const int64_t plane = n * ld;
  if (e >= plane) return;
  const int64_t p = e / ld;
  const int j0 = (int)(e - p * ld);
  const int64_t ip = perm[p];
  uint32_t w[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = j0 + 2 * c;
    w[c] = pack2(__float2bfloat16_rn(j < l ? sketch_sign(seed, ip, j, l) : 0.f),
                 __float2bfloat16_rn(j + 1 < l ? sketch_sign(seed, ip, j + 1, l) : 0.f));
  }
  *reinterpret_cast<uint4*>(P3 + e) = make_uint4(w[0], w[1], w[2], w[3]);
  *reinterpret_cast<uint4*>(P3 + plane + e) = make_uint4(0u, 0u, 0u, 0u);
  *reinterpret_cast<uint4*>(P3 + 2 * plane + e) = make_uint4(0u, 0u, 0u, 0u);
}

// dense[p][c] = (x3 + x2) + x1 of panel column c0 + c (to_panel = false), or the split of
// dense[p][c] into the panel's planes (to_panel = true); c < kc (a multiple of 8).  Eight
// columns per thread (16-byte plane accesses, two float4 of dense).
__global__ void k_cols3(__nv_bfloat16* __restrict__ P3, int ld, int c0, float* __restrict__ dense,
                        int kc, int64_t n, bool to_panel) {
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
  if (e >= n * kc) return;
  const int64_t p = e / kc;
  const int c = (int)(e - p * kc);
  const int64_t plane = n * ld, q = p * ld + c0 + c;
  float4* d4 = reinterpret_cast<float4*>(dense + e);
  if (to_panel) {
    const float4 x0 = d4[0], x1 = d4[1];
    const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
    uint32_t w[3][4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      __nv_bfloat16 a0, b0, g0, a1, b1, g1;
      split3(x[2 * t], a0, b0, g0);
      split3(x[2 * t + 1], a1, b1, g1);
      w[0][t] = pack2(a0, a1);
      w[1][t] = pack2(b0, b1);
      w[2][t] = pack2(g0, g1);
    }
#pragma unroll
    for (int pl = 0; pl < 3; ++pl)
      *reinterpret_cast<uint4*>(P3 + pl * plane + q) =
          make_uint4(w[pl][0], w[pl][1], w[pl][2], w[pl][3]);
  } else {
    const uint4 u0 = *reinterpret_cast<const uint4*>(P3 + q);
    const uint4 u1 = *reinterpret_cast<const uint4*>(P3 + plane + q);
    const uint4 u2 = *reinterpret_cast<const uint4*>(P3 + 2 * plane + q);
    const uint32_t a[4] = {u0.x, u0.y, u0.z, u0.w}, b[4] = {u1.x, u1.y, u1.z, u1.w},
                   g[4] = {u2.x, u2.y, u2.z, u2.w};
    float x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int sh = (t & 1) * 16;
      const float x1 = __uint_as_float(((a[t >> 1] >> sh) & 0xFFFFu) << 16);
      const float x2 = __uint_as_float(((b[t >> 1] >> sh) & 0xFFFFu) << 16);
      const float x3 = __uint_as_float(((g[t >> 1] >> sh) & 0xFFFFu) << 16);
      x[t] = (x3 + x2) + x1;
    }
    d4[0] = make_float4(x[0], x[1], x[2], x[3]);
    d4[1] = make_float4(x[4], x[5], x[6], x[7]);
  }
}

// T3 = the three planes of (float)A for the l x l block of A (fp64, leading dimension lda),
// zero elsewhere in [ld][ld].
__global__ void k_split3_pad(const double* __restrict__ A, int lda, int l, int ld,
                             __nv_bfloat16* __restrict__ T3) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t plane = (int64_t)ld * ld;
  if (e >= plane) return;
  const int i = (int)(e / ld), j = (int)(e % ld);
  __nv_bfloat16 a, b, d;
  split3((i < l && j < l) ? (float)A[(size_t)i * lda + j] : 0.f, a, b, d);
  T3[e] = a;
  T3[plane + e] = b;
  T3[2 * plane + e] = d;
}

// The plane pairs (a, b) of the products, smallest first: (2,0) (0,2) (1,1) (1,0) (0,1)
// (0,0).
__host__ __device__ constexpr int pair_a(int q) { return q == 0 ? 2 : (q == 2 || q == 3) ? 1 : 0; }
__host__ __device__ constexpr int pair_b(int q) { return q == 1 ? 2 : (q == 2 || q == 4) ? 1 : 0; }

// Gram partials: partial[s][i][j] = sum over the rows of split s (blockIdx.y) of X[r][i]
// Y[r][j] for the 128 x 128 tile blockIdx.x = ti (ti + 1) / 2 + tj, tj <= ti (the results
// are symmetric up to rounding; k_sum_splits mirrors them).  X and Y are P-plane panels
// (P = 3: six plane products; P = 1: bf16 values, one exact product); both are MN-major
// operands: per stage, 32 rows of each 64-column half as one box over the P planes
// (leading offset = one half's bytes).  rows_per_split is a multiple of 32.
template <int P>
struct GramCfg {
  static constexpr int kBox = 32 * 128;        // one plane of a half: 32 rows x 64 bf16
  static constexpr int kHalf = P * kBox;
  static constexpr int kStage = 4 * kHalf;     // X halves 0, 1, then Y halves 0, 1
  using Ring = TcRing<P == 3 ? 4 : 8, kStage>;
};
template <int P>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gram5(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
            int64_t n, int64_t rows_per_split, int ldp, float* __restrict__ partial,
            int* __restrict__ err) {
  using Cfg = GramCfg<P>;
  using Ring = typename Cfg::Ring;
  extern __shared__ uint8_t tc_raw[];
  const Ring R = tc_ring<Ring>(tc_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ti = (int)((sqrtf(8.f * blockIdx.x + 1.f) - 1.f) * 0.5f);
  while ((ti + 1) * (ti + 2) / 2 <= (int)blockIdx.x) ++ti;
  while (ti * (ti + 1) / 2 > (int)blockIdx.x) --ti;
  const int i0 = ti * 128, j0 = ((int)blockIdx.x - ti * (ti + 1) / 2) * 128;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r_end = std::min<int64_t>(n, r_begin + rows_per_split);
  const int64_t total = r_end > r_begin ? ceil_div(r_end - r_begin, 32) : 0;
  constexpr uint32_t kIdesc = tc05::idesc_bf16(128, 128, /*a_mn=*/true, /*b_mn=*/true);
  if (*reinterpret_cast<volatile int*>(err)) return;
  if (threadIdx.x == 0) {
    tc05::prefetch_map(&mapX);
    tc05::prefetch_map(&mapY);
  }
  tc_setup(R, 128);
  const uint32_t tmem = *R.tslot;
  volatile int* abort = R.abort;
  if (warp == 0) {
    if (lane == 0) {
      int64_t issued = 0, landed = 0, committed = -1;
      auto issue = [&](int64_t g) {
        uint8_t* st = R.at(g);
        const int row0 = (int)(r_begin + g * 32);
        tc05::mbar_expect_tx(R.full_of(g), Cfg::kStage);
        tc05::tma_load_3d(st, &mapX, i0, row0, 0, R.full_of(g));
        tc05::tma_load_3d(st + Cfg::kHalf, &mapX, i0 + 64, row0, 0, R.full_of(g));
        tc05::tma_load_3d(st + 2 * Cfg::kHalf, &mapY, j0, row0, 0, R.full_of(g));
        tc05::tma_load_3d(st + 3 * Cfg::kHalf, &mapY, j0 + 64, row0, 0, R.full_of(g));
        issued = g + 1;
      };
      for (int64_t g = 0; g < total && g < Ring::kStages; ++g) issue(g);
      bool ok = true;
      for (int64_t g = 0; g < total; ++g) {
        if (!tc05::mbar_wait(R.full_of(g), Ring::parity(g), kTcSpin, abort)) {
          ok = false;
          break;
        }
        landed = g + 1;
        tc05::fence_after_sync();
        const uint32_t xa = tc05::smem_u32(R.at(g)), ya = xa + 2 * Cfg::kHalf;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
#pragma unroll
          for (int q = 0; q < (P == 3 ? 6 : 1); ++q) {
            const int pa = P == 3 ? pair_a(q) : 0, pb = P == 3 ? pair_b(q) : 0;
            tc05::mma_bf16(tmem,
                           tc05::desc_sw128(xa + pa * Cfg::kBox + kk * 2048, Cfg::kHalf, 1024),
                           tc05::desc_sw128(ya + pb * Cfg::kBox + kk * 2048, Cfg::kHalf, 1024),
                           kIdesc, (g | kk | q) ? 1u : 0u);
          }
        tc05::mma_commit(R.empty_of(g));
        committed = g;
        if (g >= 1 && g - 1 + Ring::kStages < total) {
          if (!tc05::mbar_wait(R.empty_of(g - 1), Ring::parity(g - 1), kTcSpin, abort)) {
            ok = false;
            break;
          }
          issue(g - 1 + Ring::kStages);
        }
      }
      if (ok) {
        tc05::mma_commit(&R.accf[0]);
      } else {
        *abort = 1;
        atomicExch(err, 1);
        tc_drain(R, landed, issued, committed);
      }
    }
  } else {
    const int q = warp & 3;
    bool ok = true;
    if (total > 0) ok = epilogue_and(tc05::mbar_wait(&R.accf[0], 0u, kTcSpin, abort));
    if (!ok) {
      if (threadIdx.x == 32) {
        *abort = 1;
        atomicExch(err, 1);
      }
    } else {
      float4* out = reinterpret_cast<float4*>(
          partial + ((size_t)blockIdx.y * ldp + i0 + 32 * q + lane) * ldp + j0);
      if (total > 0) tc05::fence_after_sync();
#pragma unroll 1
      for (int cb = 0; cb < 8; ++cb) {
        float v[16];
        if (total > 0) {
          tc05::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + 16u * cb, v);
          tc05::tmem_wait_ld();
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c) v[c] = 0.f;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
          out[4 * cb + c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
      }
    }
  }
  tc05::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, 128);
}

// Panel product Z[r][j] = sum_i Y[r][i] T[j][i] for i < kdim (with `lower`, T is lower
// triangular and only i < j0 + 128 contributes), on the 128 x 128 tile (column tile
// blockIdx.x, row tile blockIdx.y; the two swapped when the row tiles exceed a grid's y
// extent).  Y ([3][n][ld]) and T ([3][ld][ld]) are 3-plane,
// both K-major (boxes 128 rows x 64 columns over the 3 planes).  ROUND = false: Z is
// stored as 3 planes [3][n][ld]; ROUND = true: Z is stored rounded to bf16 [n][ld].
struct PanelCfg {
  static constexpr int kBox = 128 * 128;   // one plane: 128 rows x 64 bf16
  static constexpr int kStage = 6 * kBox;  // Y planes, then T planes
  using Ring = TcRing<2, kStage>;
};
template <bool ROUND>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_panel5(const __grid_constant__ CUtensorMap mapY, const __grid_constant__ CUtensorMap mapT,
             int64_t n, int ld, int kdim, bool lower, bool rows_in_y,
             __nv_bfloat16* __restrict__ Z, int* __restrict__ err) {
  using Ring = PanelCfg::Ring;
  extern __shared__ uint8_t tc_raw[];
  const Ring R = tc_ring<Ring>(tc_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)(rows_in_y ? blockIdx.y : blockIdx.x) * 128;
  const int j0 = (int)(rows_in_y ? blockIdx.x : blockIdx.y) * 128;
  const int64_t total = (lower ? min(kdim, j0 + 128) : kdim) / 64;
  constexpr uint32_t kIdesc = tc05::idesc_bf16(128, 128, /*a_mn=*/false, /*b_mn=*/false);
  if (*reinterpret_cast<volatile int*>(err)) return;
  if (threadIdx.x == 0) {
    tc05::prefetch_map(&mapY);
    tc05::prefetch_map(&mapT);
  }
  tc_setup(R, 128);
  const uint32_t tmem = *R.tslot;
  volatile int* abort = R.abort;
  if (warp == 0) {
    if (lane == 0) {
      int64_t issued = 0, landed = 0, committed = -1;
      auto issue = [&](int64_t g) {
        uint8_t* st = R.at(g);
        tc05::mbar_expect_tx(R.full_of(g), PanelCfg::kStage);
        tc05::tma_load_3d(st, &mapY, (int)(g * 64), (int)r0, 0, R.full_of(g));
        tc05::tma_load_3d(st + 3 * PanelCfg::kBox, &mapT, (int)(g * 64), j0, 0, R.full_of(g));
        issued = g + 1;
      };
      for (int64_t g = 0; g < total && g < Ring::kStages; ++g) issue(g);
      bool ok = true;
      for (int64_t g = 0; g < total; ++g) {
        if (!tc05::mbar_wait(R.full_of(g), Ring::parity(g), kTcSpin, abort)) {
          ok = false;
          break;
        }
        landed = g + 1;
        tc05::fence_after_sync();
        const uint32_t ya = tc05::smem_u32(R.at(g)), ta = ya + 3 * PanelCfg::kBox;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
          for (int q = 0; q < 6; ++q)
            tc05::mma_bf16(tmem, tc05::desc_sw128(ya + pair_a(q) * PanelCfg::kBox + kk * 32, 16, 1024),
                           tc05::desc_sw128(ta + pair_b(q) * PanelCfg::kBox + kk * 32, 16, 1024),
                           kIdesc, (g | kk | q) ? 1u : 0u);
        tc05::mma_commit(R.empty_of(g));
        committed = g;
        if (g >= 1 && g - 1 + Ring::kStages < total) {
          if (!tc05::mbar_wait(R.empty_of(g - 1), Ring::parity(g - 1), kTcSpin, abort)) {
            ok = false;
            break;
          }
          issue(g - 1 + Ring::kStages);
        }
      }
      if (ok) {
        tc05::mma_commit(&R.accf[0]);
      } else {
        *abort = 1;
        atomicExch(err, 1);
        tc_drain(R, landed, issued, committed);
      }
    }
  } else {
    const int q = warp & 3;
    bool ok = true;
    if (total > 0) ok = epilogue_and(tc05::mbar_wait(&R.accf[0], 0u, kTcSpin, abort));
    if (!ok) {
      if (threadIdx.x == 32) {
        *abort = 1;
        atomicExch(err, 1);
      }
    } else {
      const int64_t r = r0 + 32 * q + lane;
      const int64_t plane = n * ld;
      if (total > 0) tc05::fence_after_sync();
#pragma unroll 1
      for (int cb = 0; cb < 8; ++cb) {
        float v[16];
        if (total > 0) {
          tc05::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + 16u * cb, v);
          tc05::tmem_wait_ld();
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c) v[c] = 0.f;
        }
        if (r < n) {
          const int64_t e = r * ld + j0 + 16 * cb;
          if (ROUND) {
            uint32_t w[8];
#pragma unroll
            for (int c = 0; c < 8; ++c)
              w[c] = pack2(__float2bfloat16_rn(v[2 * c]), __float2bfloat16_rn(v[2 * c + 1]));
            uint4* o = reinterpret_cast<uint4*>(Z + e);
            o[0] = make_uint4(w[0], w[1], w[2], w[3]);
            o[1] = make_uint4(w[4], w[5], w[6], w[7]);
          } else {
            uint32_t w[3][8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              __nv_bfloat16 a0, b0, d0, a1, b1, d1;
              split3(v[2 * c], a0, b0, d0);
              split3(v[2 * c + 1], a1, b1, d1);
              w[0][c] = pack2(a0, a1);
              w[1][c] = pack2(b0, b1);
              w[2][c] = pack2(d0, d1);
            }
#pragma unroll
            for (int pl = 0; pl < 3; ++pl) {
              uint4* o = reinterpret_cast<uint4*>(Z + pl * plane + e);
              o[0] = make_uint4(w[pl][0], w[pl][1], w[pl][2], w[pl][3]);
              o[1] = make_uint4(w[pl][4], w[pl][5], w[pl][6], w[pl][7]);
            }
          }
        }
      }
    }
  }
  tc05::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, 128);
}

// dst = the lower triangle of (src + src^T) / 2 plus `shift` + rel * max_j src[j][j] on
// the diagonal, strict upper triangle zero (l x l, leading dimension lda), and zero in the
// rest of the lda x lda array; out of place, any grid (each block reads the diagonal for
// the maximum).
__global__ void __launch_bounds__(256) k_prepare_spd(const double* __restrict__ src,
                                                     double* __restrict__ dst, int l, int lda,
                                                     double shift, double rel) {
  __shared__ double red[256];
  double m = 0.0;
  for (int j = threadIdx.x; j < l; j += blockDim.x) m = fmax(m, src[(size_t)j * lda + j]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int h = blockDim.x / 2; h >= 1; h /= 2) {
    if ((int)threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  const double sh = shift + rel * red[0];
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)lda * lda) return;
  const int i = (int)(e / lda), j = (int)(e % lda);
  if (i >= l || j >= l) {
    dst[e] = 0.0;
    return;
  }
  dst[e] = i > j ? 0.5 * (src[e] + src[(size_t)j * lda + i]) : (i == j ? src[e] + sh : 0.0);
}

// Cholesky of the diagonal block [kb, kb + nb): unblocked, in shared memory; *status = 1
// when a pivot is not positive (the pivot is then taken as 1 so that nothing overflows).
// Per column j: thread 0 takes the pivot and its reciprocal, one warp scales the column,
// then the 32 x 8 threads update the trailing lower triangle (thread (c, t) owns column
// c, rows c + t, c + t + 8, ...).
__global__ void __launch_bounds__(256) k_potrf_diag(double* __restrict__ A, int lda, int kb,
                                                    int nb, int* __restrict__ status) {
  __shared__ double a[kNB][kNB + 1];
  __shared__ double rinv;
  const int tx = (int)threadIdx.x % kNB, ty = (int)threadIdx.x / kNB;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int i = e / kNB, j = e % kNB;
    a[i][j] = (i < nb && j <= i) ? A[(size_t)(kb + i) * lda + kb + j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      const double d = a[j][j];
      double piv = 1.0;
      if (!(d > 0.0) || !isfinite(d)) *status = 1;
      else piv = sqrt(d);
      a[j][j] = piv;
      rinv = 1.0 / piv;
    }
    __syncthreads();
    if (ty == 0 && j + 1 + tx < nb) a[j + 1 + tx][j] *= rinv;
    __syncthreads();
    if (tx > j && tx < nb) {
      const double lcj = a[tx][j];
      for (int i = tx + ty; i < nb; i += 8) a[i][tx] -= a[i][j] * lcj;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    if (j <= i) A[(size_t)(kb + i) * lda + kb + j] = a[i][j];
  }
}

// Panel below the diagonal block: rows i >= kb + nb, A[i][kb .. kb + nb) <- solve of
// x L_kk^T = A[i][kb ..]; one thread per row, one warp per block (an SM's fp64 pipe is
// narrow: the rows are spread over as many SMs as possible).  Column c is final once the
// updates of columns t < c have reached it (in increasing t, as a row-by-row substitution
// orders them); it then updates the columns after it, which are independent of each other.
__global__ void __launch_bounds__(32) k_trsm_panel(double* __restrict__ A, int lda, int l,
                                                   int kb, int nb) {
  __shared__ double Lk[kNB][kNB + 1];
  __shared__ double rd[kNB];
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int i = e / kNB, j = e % kNB;
    Lk[i][j] = (i < nb && j <= i) ? A[(size_t)(kb + i) * lda + kb + j] : 0.0;
  }
  __syncwarp();
  if ((int)threadIdx.x < nb) rd[threadIdx.x] = 1.0 / Lk[threadIdx.x][threadIdx.x];
  __syncwarp();
  const int i = kb + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= l) return;
  double x[kNB];
  double* row = A + (size_t)i * lda + kb;
#pragma unroll
  for (int c = 0; c < kNB; ++c) x[c] = c < nb ? row[c] : 0.0;
#pragma unroll
  for (int c = 0; c < kNB; ++c) {
    if (c < nb) {
      x[c] *= rd[c];
#pragma unroll
      for (int q = c + 1; q < kNB; ++q) x[q] -= x[c] * Lk[q][c];
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

// One level of the recursive triangular inverse.  With the inverses X11, X22 of two
// consecutive diagonal blocks of size b, at [i0, i0 + b) and [i0 + b, i0 + b + b2),
// b2 = min(b, l - i0 - b), the inverse of their union is
//   inv([[L11, 0], [L21, L22]]) = [[X11, 0], [-X22 L21 X11, X22]],
// computed in two launches per level:
//   MODE 0: S21 = L21 X11   (X11 lower triangular: column tile c needs row tiles >= c)
//   MODE 1: X21 = -X22 S21  (X22 lower triangular: row tile r needs column tiles <= r)
// Every pair of the level at once; one 32 x 32 tile of the b2 x b result per block
// (blockIdx.x = pair, row tile, column tile), 4 outputs per thread.  Reads beyond l are
// zero.
template <int MODE>
__global__ void __launch_bounds__(256) k_trtri_level(const double* __restrict__ L,
                                                      double* __restrict__ X,
                                                      double* __restrict__ S, int lda, int l,
                                                      int b) {
  __shared__ double at[kNB][kNB + 1], bt[kNB][kNB + 1];
  const int tb = b / kNB;
  const int pair = (int)(blockIdx.x / (unsigned)(tb * tb));
  const int t = (int)(blockIdx.x % (unsigned)(tb * tb));
  const int rt = t / tb, ct = t % tb;
  const int i0 = pair * 2 * b;
  const int r0 = i0 + b + rt * kNB;  // first row of the tile (in the second block)
  const int c0 = i0 + ct * kNB;      // first column of the tile (in the first block)
  if (i0 + b >= l || r0 >= l) return;  // uniform per block
  const double* A = MODE == 0 ? L : X;
  const double* Bm = MODE == 0 ? X : S;
  const int k_base = MODE == 0 ? i0 : i0 + b;
  const int kt0 = MODE == 0 ? ct : 0, kt1 = MODE == 0 ? tb - 1 : rt;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int kt = kt0; kt <= kt1; ++kt) {
    const int kb = k_base + kt * kNB;
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
      const int r = e / kNB, c = e % kNB;
      at[r][c] = (r0 + r < l && kb + c < l) ? A[(size_t)(r0 + r) * lda + kb + c] : 0.0;
      bt[r][c] = (kb + r < l) ? Bm[(size_t)(kb + r) * lda + c0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int r = e / kNB, c = e % kNB;
      double s = 0.0;
#pragma unroll 8
      for (int k = 0; k < kNB; ++k) s += at[r][k] * bt[k][c];
      acc[q] += s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + 256 * q;
    const int r = e / kNB, c = e % kNB;
    if (r0 + r < l) {
      if (MODE == 0) S[(size_t)(r0 + r) * lda + c0 + c] = acc[q];
      else X[(size_t)(r0 + r) * lda + c0 + c] = -acc[q];
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
// Blocks of `func` (threads per block, dynamic shared bytes) that one SM holds at once,
// from its registers, its static and dynamic shared memory (plus the per-block reserve)
// and the SM's limits; at least 1.  (The runtime's occupancy query may assume a smaller
// shared-memory carve-out than the one a launch gets.)
static cudaError_t resident_blocks(const void* func, int threads, int dyn_smem, int dev,
                                   int* out) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, func);
  int smem_sm = 0, reserve = 0, regs_sm = 0, threads_sm = 0;
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  if (e != cudaSuccess) return e;
  const int warps = (threads + 31) / 32;
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;  // allocation unit: 256
  const int by_regs = regs_sm / std::max(1, regs_warp * warps);
  const int by_smem = smem_sm / std::max(1, (int)fa.sharedSizeBytes + dyn_smem + reserve);
  const int by_threads = threads_sm / std::max(1, threads);
  *out = std::max(1, std::min(std::min(by_regs, by_smem), std::min(by_threads, 32)));
  return cudaSuccess;
}

namespace {

struct Dense {
  int l, lda;
  cudaStream_t st;
  int* status;  // device
  double* S;    // l x l scratch of the triangular inverse
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
        k_trsm_panel<<<(unsigned)ceil_div(rest, 32), 32, 0, st>>>(A, lda, l, kb, nb);
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
  // X = L^-1 (lower), X zero above the diagonal: the 32 x 32 diagonal blocks inverted,
  // then pairs of inverted blocks joined level by level (b = 32, 64, ...); S: l x l scratch.
  cudaError_t trtri(const double* L, double* X) {
    cudaError_t e = cudaMemsetAsync(X, 0, (size_t)lda * lda * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const int nblk = (l + kNB - 1) / kNB;
    k_trtri_diag<<<nblk, kNB, 0, st>>>(L, X, lda, l);
    note_launches(1);
    for (int b = kNB; b < l; b *= 2) {
      const int tb = b / kNB;
      const unsigned grid = (unsigned)(ceil_div(l - b, 2 * b) * tb * tb);
      k_trtri_level<0><<<grid, 256, 0, st>>>(L, X, S, lda, l, b);
      k_trtri_level<1><<<grid, 256, 0, st>>>(L, X, S, lda, l, b);
      note_launches(2);
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
#define PC_MAP(expr)                                                   \
  do {                                                                 \
    if (!(expr)) {                                                     \
      set_error("encoding a preconditioner tensor map failed");        \
      return SGP_ERR_CUDA;                                             \
    }                                                                  \
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
    cudaError_t e = dev_malloc(p, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  };
  auto temp = [&](void** p, size_t bytes) {
    cudaError_t e = dev_malloc(p, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) temps.push_back(*p);
    return e;
  };
  {  // dynamic shared memory above 48 KB, once per device
    static std::atomic<bool> attrs[64];
    int dev = 0;
    PC_CHECK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev >= 0 && dev < 64 && !attrs[dev].load()) {
      PC_CHECK(cudaFuncSetAttribute(k_gram5<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    GramCfg<3>::Ring::kSmem),
               "k_gram5 smem");
      PC_CHECK(cudaFuncSetAttribute(k_gram5<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    GramCfg<1>::Ring::kSmem),
               "k_gram5 smem");
      PC_CHECK(cudaFuncSetAttribute(k_panel5<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    PanelCfg::Ring::kSmem),
               "k_panel5 smem");
      PC_CHECK(cudaFuncSetAttribute(k_panel5<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    PanelCfg::Ring::kSmem),
               "k_panel5 smem");
      PC_CHECK(cudaFuncSetAttribute(k_bt_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    BtRing::kSmem),
               "k_bt_tc smem");
      PC_CHECK(cudaFuncSetAttribute(k_z_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    ApplyRing::kSmem),
               "k_z_tc smem");
      // the largest shared-memory carve-out, so that two apply blocks share an SM
      PC_CHECK(cudaFuncSetAttribute(k_bt_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    cudaSharedmemCarveoutMaxShared),
               "k_bt_tc carve-out");
      PC_CHECK(cudaFuncSetAttribute(k_z_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    cudaSharedmemCarveoutMaxShared),
               "k_z_tc carve-out");
      attrs[dev].store(true);
    }
  }
  int sms = 0, dev_now = 0;
  PC_CHECK(cudaGetDevice(&dev_now), "cudaGetDevice");
  PC_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_now), "SM count");
  const size_t panel3 = (size_t)3 * n * ld * sizeof(__nv_bfloat16);
  __nv_bfloat16 *P1 = nullptr, *P2 = nullptr, *T3 = nullptr;
  float *Vc = nullptr, *KVc = nullptr, *gpart = nullptr;
  double *G = nullptr, *G0 = nullptr, *Xi = nullptr, *M = nullptr, *Sx = nullptr, *pv = nullptr,
         *py = nullptr, *prq = nullptr;
  int* status = nullptr;
  PC_CHECK(keep((void**)&B, (size_t)n * ld * sizeof(__nv_bfloat16)),
           "alloc preconditioner B");
  PC_CHECK(keep((void**)&err, sizeof(int)), "alloc error flag");
  PC_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st), "clear error flag");
  PC_CHECK(temp((void**)&P1, panel3), "alloc preconditioner panel");
  PC_CHECK(temp((void**)&P2, panel3), "alloc preconditioner panel");
  PC_CHECK(temp((void**)&Vc, (size_t)n * kSketchCols * sizeof(float)), "alloc sketch chunk");
  PC_CHECK(temp((void**)&KVc, (size_t)n * kSketchCols * sizeof(float)), "alloc sketch chunk");
  const int ntile = ld / kTile;
  // row splits of the Grams (multiples of 32 rows): the count whose blocks fill the last
  // of their waves best, between 1 and 8 waves (one block per SM), at least 2048 rows each
  const int tiles = ntile * (ntile + 1) / 2;
  int splits = 1;
  {
    const int64_t lo = std::max<int64_t>(1, ceil_div(sms, tiles));
    const int64_t hi = std::max<int64_t>(lo, std::min<int64_t>(ceil_div(8 * (int64_t)sms, tiles),
                                                               ceil_div(n, 2048)));
    double best = -1.0;
    for (int64_t sp = lo; sp <= hi; ++sp) {
      const int64_t blocks = sp * tiles, waves = ceil_div(blocks, sms);
      const double eff = (double)blocks / (double)(waves * sms);
      if (eff > best + 1e-9) {
        best = eff;
        splits = (int)sp;
      }
    }
  }
  const int64_t rows_per_split = ceil_div(ceil_div(n, splits), 32) * 32;
  splits = (int)ceil_div(n, rows_per_split);
  const size_t ll = (size_t)ld * ld;
  PC_CHECK(temp((void**)&gpart, (size_t)splits * ll * sizeof(float)), "alloc Gram partials");
  PC_CHECK(temp((void**)&T3, 3 * ll * sizeof(__nv_bfloat16)), "alloc l x l");
  PC_CHECK(temp((void**)&G, ll * sizeof(double)), "alloc l x l");
  PC_CHECK(temp((void**)&G0, ll * sizeof(double)), "alloc l x l");
  PC_CHECK(temp((void**)&Xi, ll * sizeof(double)), "alloc l x l");
  PC_CHECK(temp((void**)&M, ll * sizeof(double)), "alloc l x l");
  PC_CHECK(temp((void**)&Sx, ll * sizeof(double)), "alloc l x l");
  PC_CHECK(temp((void**)&pv, ld * sizeof(double)), "alloc power vectors");
  PC_CHECK(temp((void**)&py, ld * sizeof(double)), "alloc power vectors");
  PC_CHECK(temp((void**)&prq, sizeof(double)), "alloc power vectors");
  PC_CHECK(temp((void**)&status, sizeof(int)), "alloc status");
  // per-iteration buffers.  B^T r: one wave of the blocks the device keeps resident (i
  // tiles x row splits of a multiple of 64 rows); z: one persistent block per resident slot
  int tc_per_sm = 0;
  PC_CHECK(resident_blocks(reinterpret_cast<const void*>(k_bt_tc), kTcThreads, BtRing::kSmem,
                           dev_now, &tc_per_sm),
           "occupancy");
  bt_splits = (int)std::max<int64_t>(
      1, std::min<int64_t>(tc_per_sm * (int64_t)sms / ntile, ceil_div(n, kTcRows)));
  bt_rows = ceil_div(ceil_div(n, bt_splits), kTcRows) * kTcRows;
  bt_splits = (int)ceil_div(n, bt_rows);
  PC_CHECK(resident_blocks(reinterpret_cast<const void*>(k_z_tc), kTcThreads, ApplyRing::kSmem,
                           dev_now, &tc_per_sm),
           "occupancy");
  z_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(tc_per_sm * (int64_t)sms,
                                                         ceil_div(n, kTile)));
  ldr = ceil_div(n, kTcRows) * kTcRows;
  PC_CHECK(keep((void**)&tpart, (size_t)bt_splits * ld * 16 * sizeof(float)), "alloc B^T r");
  PC_CHECK(keep((void**)&tvec, (size_t)ld * 16 * sizeof(float)), "alloc t");
  PC_CHECK(keep((void**)&u, (size_t)3 * 16 * ld * sizeof(__nv_bfloat16)), "alloc u");
  PC_CHECK(keep((void**)&r3, (size_t)ldr * 64 * sizeof(__nv_bfloat16)), "alloc split r");
  PC_CHECK(cudaMemsetAsync(r3, 0, (size_t)ldr * 64 * sizeof(__nv_bfloat16), st), "clear split r");
  PC_CHECK(keep((void**)&Minv, ll * sizeof(float)), "alloc Minv");
  {  // TMA maps of the factor (as the K-major A of B u and the MN-major A of B^T r), of u
     // and of the split r
    const CUtensorMapDataType bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    PC_MAP(tc05::make_map_2d(&map_b_k, bf, B, (uint64_t)n, (uint64_t)ld, (uint64_t)ld * 2, 128,
                             kTcRows));
    PC_MAP(tc05::make_map_2d(&map_b_mn, bf, B, (uint64_t)n, (uint64_t)ld, (uint64_t)ld * 2,
                             kTcRows, kTcRows));
    PC_MAP(tc05::make_map_2d(&map_u, bf, u, 48, (uint64_t)ld, (uint64_t)ld * 2, 48, kTcRows));
    PC_MAP(tc05::make_map_2d(&map_r, bf, r3, (uint64_t)n, 64, 128, kTcRows, 64));
  }
  sgp_status s = ensure_lattice_values(L, kSketchCols, st);
  if (s != SGP_OK) return s;

  Dense dn{l, ld, st, status, Sx};
  const unsigned g_plane = (unsigned)ceil_div((int64_t)n * ld / 8, 256);
  const unsigned g_chunk = (unsigned)ceil_div((int64_t)n * kSketchCols / 8, 256);
  // dst = outputscale K src, column chunk by chunk (3-plane panels; padding columns of dst:
  // zero).  bf16_values: lattice values held in bf16 (the subspace product, whose result
  // only fixes the subspace)
  auto product = [&](__nv_bfloat16* src, __nv_bfloat16* dst, bool bf16_values) -> sgp_status {
    for (int c0 = 0; c0 < ld; c0 += kSketchCols) {
      k_cols3<<<g_chunk, 256, 0, st>>>(src, ld, c0, Vc, kSketchCols, n, false);
      if (bf16_values)
        enqueue_mvm_bf16_values(L, Vc, kSketchCols, blur, L->outputscale, KVc, st);
      else
        enqueue_mvm(L, Vc, kSketchCols, blur, L->outputscale, 0.f, KVc, st, nullptr,
                    /*internal=*/true);
      k_cols3<<<g_chunk, 256, 0, st>>>(dst, ld, c0, KVc, kSketchCols, n, true);
      note_launches(2);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SGP_OK : cuda_status(e, "sketch products");
  };
  // G = X^T Y (fp64 [ld][ld]) of two 3-plane panels, or (planes = 1) of bf16 panels
  auto gram = [&](const void* X, const void* Y, int planes, double* out) -> sgp_status {
    CUtensorMap mx, my;
    PC_MAP(tc05::make_map_planes(&mx, X, planes, n, ld, ld, planes, 32));
    PC_MAP(tc05::make_map_planes(&my, Y, planes, n, ld, ld, planes, 32));
    if (planes == 3)
      k_gram5<3><<<dim3(tiles, splits), kTcThreads, GramCfg<3>::Ring::kSmem, st>>>(
          mx, my, n, rows_per_split, ld, gpart, err);
    else
      k_gram5<1><<<dim3(tiles, splits), kTcThreads, GramCfg<1>::Ring::kSmem, st>>>(
          mx, my, n, rows_per_split, ld, gpart, err);
    k_sum_splits<<<(unsigned)ceil_div((int64_t)ll, 256), 256, 0, st>>>(gpart, splits, ld, out);
    note_launches(2);
    return SGP_OK;
  };
  // Z = Y X^T for the fp64 lower-triangular X (Z[r][j] = sum_i Y[r][i] X[j][i]): Y 3-plane,
  // Z 3-plane, or rounded to bf16 when `round`
  auto panel_times = [&](const __nv_bfloat16* Y, const double* X, void* Z, bool round)
      -> sgp_status {
    k_split3_pad<<<(unsigned)ceil_div((int64_t)ll, 256), 256, 0, st>>>(X, ld, l, ld, T3);
    CUtensorMap my, mt;
    PC_MAP(tc05::make_map_planes(&my, Y, 3, n, ld, ld, 3, 128));
    PC_MAP(tc05::make_map_planes(&mt, T3, 3, ld, ld, ld, 3, 128));
    // column tiles fastest: the tiles of one row block run together and read its rows
    // of Y from L2 after the first
    const int64_t row_tiles = ceil_div(n, kTile);
    const dim3 grid = row_tiles <= 65535 ? dim3(ntile, (unsigned)row_tiles)
                                         : dim3((unsigned)row_tiles, ntile);
    const bool rows_in_y = row_tiles <= 65535;
    if (round)
      k_panel5<true><<<grid, kTcThreads, PanelCfg::Ring::kSmem, st>>>(
          my, mt, n, ld, ld, /*lower=*/true, rows_in_y, static_cast<__nv_bfloat16*>(Z), err);
    else
      k_panel5<false><<<grid, kTcThreads, PanelCfg::Ring::kSmem, st>>>(
          my, mt, n, ld, ld, /*lower=*/true, rows_in_y, static_cast<__nv_bfloat16*>(Z), err);
    note_launches(2);
    return SGP_OK;
  };
  // Cholesky of the symmetrised out-of-place copy of src with a relative diagonal shift,
  // raised 100-fold (at most 4 times) while a pivot fails; the factor lands in dst, and
  // `raised` tells whether the first shift failed.
  bool raised = false;
  auto robust_chol = [&](const double* src, double* dst, double rel, bool& good) -> sgp_status {
    good = false;
    raised = false;
    for (int attempt = 0; attempt < 4 && !good; ++attempt, rel *= 100.0) {
      raised = attempt > 0;
      k_prepare_spd<<<(unsigned)ceil_div((int64_t)ll, 256), 256, 0, st>>>(src, dst, l, ld, 0.0,
                                                                          rel);
      note_launches(1);
      cudaError_t err_ = cudaSuccess;
      if (!dn.chol(dst, good, err_)) return cuda_status(err_, "Cholesky");
    }
    return SGP_OK;
  };

  // 1. Q: the sketch, or a basis of the range of K Omega by Cholesky QR.  The Nystrom
  // approximation depends only on that range, so one pass suffices while the Gram's first
  // Cholesky succeeds; a second pass restores the orthogonality when its shift had to be
  // raised.
  k_fill_sketch3<<<g_plane, 256, 0, st>>>(L->perm, n, l, ld, seed, P1);
  note_launches(1);
  __nv_bfloat16* Q = P1;
  __nv_bfloat16* Y = P2;
  // P2 = K Omega.  With the subspace iteration this product only fixes the subspace (Q's
  // range): it runs on bf16 lattice values, whose ~2.5e-3 relative error perturbs the
  // captured directions negligibly, while Y = K Q below, which defines B, stays fp32.
  if ((s = product(P1, P2, power_iters > 0)) != SGP_OK) return s;
  if (power_iters > 0) {
    __nv_bfloat16* src = P2;
    __nv_bfloat16* dst = P1;
    for (int pass = 0; pass < 2; ++pass) {
      bool good = false;
      if ((s = gram(src, src, 3, G0)) != SGP_OK) return s;
      if ((s = robust_chol(G0, G, 1e-7, good)) != SGP_OK) return s;
      if (!good) return SGP_OK;  // ok stays false: the solve runs unpreconditioned
      PC_CHECK(dn.trtri(G, Xi), "triangular inverse");
      if ((s = panel_times(src, Xi, dst, false)) != SGP_OK) return s;  // dst = src R^-T
      std::swap(src, dst);
      if (!raised) break;
    }
    Q = src;  // the basis (P1 after one pass, P2 after two)
    Y = dst;
    if ((s = product(Q, Y, false)) != SGP_OK) return s;
  }
  // 2. C = Q^T Y, C = R R^T, B = Y R^-T rounded to bf16 (the stored values define P)
  {
    bool good = false;
    if ((s = gram(Q, Y, 3, G0)) != SGP_OK) return s;
    if ((s = robust_chol(G0, G, 1e-6, good)) != SGP_OK) return s;
    if (!good) return SGP_OK;
    PC_CHECK(dn.trtri(G, Xi), "triangular inverse");
    if ((s = panel_times(Y, Xi, B, true)) != SGP_OK) return s;
  }
  // 3. G = B^T B (exact products of the bf16 values); lambda_min(G) by power iteration on
  // G^-1; tau = lambda_min + noise
  double lam_min = 0.0;
  {
    if ((s = gram(B, B, 1, G0)) != SGP_OK) return s;
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
  if ((s = check(st)) != SGP_OK) return s;
  ok = true;
  return SGP_OK;
#undef PC_CHECK
#undef PC_MAP
}

int64_t ShiftedNystrom::dot_blocks() const { return z_blocks; }

void ShiftedNystrom::apply(const float* rh, const float* rl, int k, float* z, double* dot,
                           cudaStream_t st, cudaEvent_t* ev, bool split_ready) const {
  const int ntile = ld / kTile;
  for (int c_off = 0; c_off < k; c_off += 16) {
    const int kc = std::min(16, k - c_off);
    // with ev (inside a capture: external record nodes) the first 16-column chunk's
    // B^T r and z kernels are bracketed for the stage timings
    const bool mark = ev && c_off == 0;
    if (mark) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
    if (!(split_ready && c_off == 0)) {
      k_split_r<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(rh, rl, k, c_off, kc, n,
                                                           static_cast<__nv_bfloat16*>(r3));
      note_launches(1);
    }
    k_bt_tc<<<dim3(ntile, bt_splits), kTcThreads, BtRing::kSmem, st>>>(map_b_mn, map_r, n, bt_rows,
                                                                  tpart, err);
    if (mark) cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
    k_sum_t<<<(unsigned)ceil_div(ld * 16, 256), 256, 0, st>>>(tpart, bt_splits, ld, tvec);
    k_minv_u<<<(unsigned)ceil_div(ld, 8), 256, 0, st>>>(Minv, ld, tvec,
                                                         static_cast<__nv_bfloat16*>(u));
    if (mark) cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal);
    k_z_tc<<<z_blocks, kTcThreads, ApplyRing::kSmem, st>>>(map_b_k, map_u, rh, k, c_off, kc, n, ld,
                                                  1.f / tau, z, dot, err);
    if (mark) cudaEventRecordWithFlags(ev[3], st, cudaEventRecordExternal);
    note_launches(4);
  }
}

sgp_status ShiftedNystrom::check(cudaStream_t st) const {
  if (!err) return SGP_OK;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "reading the preconditioner's error flag");
  if (h) {
    set_error("a preconditioner kernel gave up waiting for its tensor-memory copies");
    return SGP_ERR_CUDA;
  }
  return SGP_OK;
}

void ShiftedNystrom::release(cudaStream_t st) {
  for (void* p : ptrs) (void)cudaFreeAsync(p, st);
  ptrs.clear();
}

}  // namespace sgp
