// Continuous-batching server of GP posterior requests (Sec. 2: Eq. gp_pred_mean and
// Eq. gp_pred_cov, solved with CG that touches the kernel only through lattice MVMs).
//
// Per request: one lattice over the joint point set [X; Xs] (Sec. 3.2), so that the
// cross-covariances K*X and KX* are the same operator sliced at test or training rows.
// The CG system is (outputscale K~ + noise I) restricted to the training rows: the
// slice writes zero at test rows, and the right-hand sides are zero there, so every CG
// vector stays in the training subspace.  Right-hand sides: column 0 = y, columns
// 1..S = KX* z_s for Rademacher probes z_s over the test points; after the solve one
// product sliced at the test rows gives the mean (column 0) and the probe estimate of
// diag(K*X A^-1 KX*) (columns 1..S).  The probe product also carries a ones column over
// the training rows (column kp - 1): its largest entry is the Gershgorin bound behind
// the request's condition estimate, which decides whether its CG is preconditioned with
// the rank-l Nystrom factor of App. A.
//
// Batching: one CG iteration of every active request is a fixed sequence of kernels
// (splat, two fix-ups, 2 Dmax blur passes, slice with <p, Ap>, alpha, x/r update; for
// preconditioned requests B^T r, its two ordered sums, Minv B^T r and z = P^-1 r; then
// convergence check and beta, p update) with fixed grids.  Each kernel walks "virtual
// blocks" over a device table of the active requests; a request's virtual blocks cover
// its own rows in a partition fixed by its own sizes, so its results (and reduction
// order) do not depend on the other requests in the batch.  Requests that have stopped
// are skipped by a device flag; blur pass t touches only requests with t < 2 (d + 1).
// Requests are grouped into lanes of similar dimension and per-iteration work; each lane
// is such a batch with its own table, stream and CUDA graph of one iteration (captured
// once per Dmax, sparse blur and preconditioning, then replayed), rewritten
// (stream-ordered) when requests join or leave, and the lanes run concurrently.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <mutex>
#include <string>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <vector>

#include "sgp_internal.cuh"
#include "values.cuh"
#include "../../include/sgp_serve.h"

namespace sgp {
namespace {

constexpr int kMaxSlots = 64;       // requests in one batch
constexpr int kMaxServeK = 32;      // columns per request (1 + probes, padded to 4)
constexpr int kST = 256;            // threads of the table-driven kernels
constexpr int kGrid = 4 * 152;      // their fixed grid (4 blocks per SM)
constexpr int kBlurU = 2;           // blur rows per thread
constexpr int kVecRows = 4;         // vector-kernel rows per thread
constexpr int kMaxLd = kMaxRank;    // preconditioner: B row stride bound
constexpr int kBtVbRows = 512;      // rows of one B^T r virtual block
constexpr int kBtSeg = 16;          // B^T r partials per first-level sum
constexpr int kZVbRows = 576;       // rows of one z virtual block
constexpr int kStages = 3;          // bulk-copied chunks in flight per block
constexpr int kRingBytes = 192 * 1024;  // shared memory of the chunk ring
constexpr int kRingRowsMax = 96;    // rows of one chunk at most
constexpr int kRingGrid = 152;      // persistent grid of the ring kernels (one block per SM)
constexpr int kSpinLimit = 1 << 20; // bounded mbarrier waits (about a second at most)
constexpr double kBf16MaxKappa = 100.0;  // BF16 server: larger condition estimates use fp32
constexpr uint64_t kPrecondSeedXor = 0x6A09E667F3BCC909ull;  // sketch seed = seed ^ this

enum { U_SPLAT = 0, U_MED, U_HUGE, U_BLUR, U_VEC, U_VERT, U_BT, U_BTS, U_BTT, U_MINV, U_Z,
       U_KINDS };

// One active request as the kernels see it.  Row-indexed arrays are in the lattice's
// locality order p; perm[p] < n_train marks a training row.
struct SlotDev {
  int64_t n, n_train, m;
  int D, r;
  int64_t nseg, nmed, nhuge;
  const int32_t* perm;
  const int32_t* idx;
  const float* w;
  const int2* items;
  const int4* seg;
  const int4* med;
  const int4* huge;
  const int32_t* nbr;
  float taps[kMaxOrder + 1];  // symmetric-blur (half-kernel) taps
  float outputscale, noise;
  void* lat0;
  void* lat1;
  float* spart;  // splat partials
  float *xh, *xl, *rh, *rl, *p, *ap;  // [n][kp]
  double* dpart;                      // [virtual blocks][kp]
  double *rho, *bnorm, *relres, *alpha, *beta;  // [kp]
  int* active;                        // [kp]
  int* state;                         // [0] request still iterating, [1] iterations done
  int max_iter;
  float tol;
  // sparse lattices: direction lists, per-vertex epochs and the pass buffer (the values
  // stay in lat0 with lazy centre-tap factors g0pow, as in the library's sparse blur)
  int sparse;
  const int32_t* act;
  const int64_t* act_off;  // [D + 1]
  int32_t* epoch;
  void* stmp;
  const float* g0pow;
  // rank-l Nystrom preconditioner (l = 0: plain CG): P = B B^T + noise I
  int l, ld;
  float inv_noise;
  const float* Bh;      // [n][ld] fp32, locality order, zero at test rows
  const double* Minv;   // [l][l] (noise I + B^T B)^-1
  float* btpart;        // [U_BT virtual blocks][ld][kp] fp32 partials of B^T r
  float* bt2;           // [segments][ld][kp] sums of kBtSeg partials
  double* tvec;         // [ld][kp] B^T r
  float* u;             // [ld][kp] Minv B^T r (rows >= l zero)
  double* dpart2;       // [U_Z virtual blocks][kp] partials of <r, z>
};

struct Table {
  int nslots;
  int kp;
  int* flags;  // [kMaxSlots][2]: state copied by the check kernel, read by the host
  int* err;    // set to 1 when a bulk-copy wait gave up (the round's results are void)
  int wait_limit;  // try_wait polls of the ring's chunk waits (kSpinLimit; 0 under SGP_FAULT)
  int64_t pre[U_KINDS][kMaxSlots + 1];  // prefix sums of virtual blocks per unit kind
  SlotDev s[kMaxSlots];
};

__host__ __device__ inline int groups_of(int kp) { return kST / (kp / 4); }

__device__ __forceinline__ int find_slot(const int64_t* pre, int ns, int64_t vb) {
  int lo = 0, hi = ns - 1;  // largest q with pre[q] <= vb
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= vb) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Walk this block's virtual blocks of one unit kind: q = request, local = its block index.
#define SLOT_LOOP(KIND)                                                            \
  const int ns_ = T->nslots;                                                       \
  const int64_t total_ = T->pre[KIND][ns_];                                        \
  for (int64_t vb_ = blockIdx.x; vb_ < total_; vb_ += gridDim.x) {                 \
    const int q = find_slot(T->pre[KIND], ns_, vb_);                               \
    const SlotDev& s = T->s[q];                                                    \
    const int64_t local = vb_ - T->pre[KIND][q];

#define SLOT_LOOP_END }

// SplitMix64 (Steele, Lea & Flood 2014) sign at counter i l + j + 1.
__device__ __forceinline__ float rademacher_pm(uint64_t seed, int64_t i, int j, int l) {
  uint64_t z = seed + ((uint64_t)(i * l + j) + 1ull) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (z >> 63) ? -1.f : 1.f;
}

// Per-column sums of the block's per-thread partials (thread t owns columns (t % G) 4 ..
// + 3 of block row t / G), fixed order; out[0..kp).  Uniform call, trailing barrier.
__device__ __forceinline__ void vb_column_sums(const dfloat (&d)[4], int kp, double* out,
                                               double* sh) {
#pragma unroll
  for (int j = 0; j < 4; ++j) sh[threadIdx.x * 4 + j] = df_to_double(d[j]);
  __syncthreads();
  const int G = kp / 4, rows = kST / G;
  for (int col = threadIdx.x; col < kp; col += blockDim.x) {
    const int chunk = col / 4, lane = col % 4;
    double t = 0.0;
    for (int r = 0; r < rows; ++r) t += sh[(r * G + chunk) * 4 + lane];
    out[col] = t;
  }
  __syncthreads();
}

// Totals of all kp columns over a request's nvb virtual-block partials part[b][c], in one
// coalesced pass: thread t < R kp (R = kST / kp) owns column t % kp and the blocks
// t / kp, t / kp + R, ... (summed in order), then thread c < kp adds the R sums of its
// column in order.  out (shared, kp entries); uniform call, trailing barrier.
__device__ __forceinline__ void slot_cols_total(const double* part, int64_t nvb, int kp,
                                                double* red, double* out) {
  const int R = kST / kp;
  const int t = threadIdx.x;
  double acc = 0.0;
  if (t < R * kp)
    for (int64_t b = t / kp; b < nvb; b += R) acc += part[b * kp + t % kp];
  red[t] = acc;
  __syncthreads();
  if (t < kp) {
    double v = 0.0;
    for (int r = 0; r < R; ++r) v += red[r * kp + t];
    out[t] = v;
  }
  __syncthreads();
}

__device__ __forceinline__ float4 f4_fma(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 f4_ld(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void f4_st(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// ---- one CG iteration over the table --------------------------------------------------
// Splat W^T p into lat0: one thread-group per segment of a vertex's incidence list.
template <class S>
__global__ void __launch_bounds__(kST) kb_splat(const Table* __restrict__ T) {
  const int kp = T->kp, G = kp / 4, groups = kST / G;
  const int g = threadIdx.x / G, col = (int)(threadIdx.x % G) * 4;
  SLOT_LOOP(U_SPLAT)
  if (*s.state == 0 || g >= groups) continue;
  const int64_t sidx = local * groups + g;
  if (sidx >= s.nseg) continue;
  const int4 sg = s.seg[sidx];
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int it = sg.y; it < sg.z; ++it) {
    const int2 e = s.items[it];
    acc = f4_fma(__int_as_float(e.y), f4_ld(s.p + (int64_t)e.x * kp + col), acc);
  }
  if (sg.w < 0) {
    Store<S>::st4(static_cast<S*>(s.lat0) + (int64_t)sg.x * kp + col, acc);
    if (s.sparse && col == 0) s.epoch[sg.x] = 0;
  } else {
    f4_st(s.spart + (int64_t)sg.w * kp + col, acc);
  }
  SLOT_LOOP_END
}

// Vertices with 2..kSplatMedSegs segments: one thread-group sums the partials in order.
template <class S>
__global__ void __launch_bounds__(kST) kb_splat_med(const Table* __restrict__ T) {
  const int kp = T->kp, G = kp / 4, groups = kST / G;
  const int g = threadIdx.x / G, col = (int)(threadIdx.x % G) * 4;
  SLOT_LOOP(U_MED)
  if (*s.state == 0 || g >= groups) continue;
  const int64_t ridx = local * groups + g;
  if (ridx >= s.nmed) continue;
  const int4 rw = s.med[ridx];
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int j = 0; j < rw.z; ++j) {
    const float4 v = f4_ld(s.spart + (int64_t)(rw.y + j) * kp + col);
    acc = make_float4(acc.x + v.x, acc.y + v.y, acc.z + v.z, acc.w + v.w);
  }
  Store<S>::st4(static_cast<S*>(s.lat0) + (int64_t)rw.x * kp + col, acc);
  if (s.sparse && col == 0) s.epoch[rw.x] = 0;
  SLOT_LOOP_END
}

// Vertices with more segments: one virtual block per vertex, strided partials per group
// and a fixed shared-memory tree over the groups.
template <class S>
__global__ void __launch_bounds__(kST) kb_splat_huge(const Table* __restrict__ T) {
  __shared__ float4 red[kST];
  const int kp = T->kp, G = kp / 4, groups = kST / G;
  const int g = threadIdx.x / G, col = (int)(threadIdx.x % G) * 4;
  int pow2 = 1;
  while (pow2 * 2 <= groups) pow2 *= 2;
  SLOT_LOOP(U_HUGE)
  if (*s.state == 0) continue;  // uniform over the block
  const int4 rw = s.huge[local];
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (g < pow2)
    for (int j = g; j < rw.z; j += pow2) {
      const float4 v = f4_ld(s.spart + (int64_t)(rw.y + j) * kp + col);
      acc = make_float4(acc.x + v.x, acc.y + v.y, acc.z + v.z, acc.w + v.w);
    }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int half = pow2 / 2; half >= 1; half /= 2) {
    if (g < half) {
      const float4 a = red[threadIdx.x], b = red[threadIdx.x + half * G];
      red[threadIdx.x] = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
    }
    __syncthreads();
  }
  if (g == 0) Store<S>::st4(static_cast<S*>(s.lat0) + (int64_t)rw.x * kp + col, red[threadIdx.x]);
  if (s.sparse && threadIdx.x == 0) s.epoch[rw.x] = 0;
  __syncthreads();
  SLOT_LOOP_END
}

// Blur pass t of the symmetric operator: direction t for t < D, then 2D - 1 - t; pass t
// reads lat[t % 2] and writes lat[(t + 1) % 2], so after 2D passes the values are back
// in lat0.  Each thread owns 4 columns of kBlurU rows (ids first, then rows).
template <int R, class S>
__global__ void __launch_bounds__(kST) kb_blur(const Table* __restrict__ T, int t) {
  const int kp = T->kp, G = kp / 4, groups = kST / G;
  const int g = threadIdx.x / G, col = (int)(threadIdx.x % G) * 4;
  SLOT_LOOP(U_BLUR)
  if (*s.state == 0 || t >= 2 * s.D || g >= groups) continue;
  const int j = t < s.D ? t : 2 * s.D - 1 - t;
  if (s.sparse) {  // the vertices of list j: new rows into stmp, lazy factors on reads
    const int64_t base = s.act_off[j], count = s.act_off[j + 1] - base;
    const S* lat = static_cast<const S*>(s.lat0);
    const int32_t* nbr = s.nbr + (int64_t)j * R * 2 * s.m;
    for (int u = 0; u < kBlurU; ++u) {
      const int64_t e = (local * kBlurU + u) * groups + g;
      if (e >= count) break;
      const int64_t v = s.act[base + e];
      const float4 own = Store<S>::ldg4(lat + v * kp + col);
      const float fo = s.g0pow[t - s.epoch[v]];
      float4 acc = make_float4(s.taps[0] * fo * own.x, s.taps[0] * fo * own.y,
                               s.taps[0] * fo * own.z, s.taps[0] * fo * own.w);
#pragma unroll
      for (int tt = 0; tt < R; ++tt) {
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
        const int ia = nbr[(int64_t)(2 * tt) * s.m + v];
        const int ic = nbr[(int64_t)(2 * tt + 1) * s.m + v];
        if (ia >= 0) {
          const float f = s.g0pow[t - s.epoch[ia]];
          const float4 x = Store<S>::ldg4(lat + (int64_t)ia * kp + col);
          sum = make_float4(f * x.x, f * x.y, f * x.z, f * x.w);
        }
        if (ic >= 0) {
          const float f = s.g0pow[t - s.epoch[ic]];
          const float4 x = Store<S>::ldg4(lat + (int64_t)ic * kp + col);
          sum = make_float4(sum.x + f * x.x, sum.y + f * x.y, sum.z + f * x.z, sum.w + f * x.w);
        }
        const float wt = s.taps[tt + 1];
        acc = make_float4(fmaf(wt, sum.x, acc.x), fmaf(wt, sum.y, acc.y), fmaf(wt, sum.z, acc.z),
                          fmaf(wt, sum.w, acc.w));
      }
      Store<S>::st4(static_cast<S*>(s.stmp) + e * kp + col, acc);
    }
    continue;
  }
  const S* in = static_cast<const S*>((t & 1) ? s.lat1 : s.lat0);
  S* out = static_cast<S*>((t & 1) ? s.lat0 : s.lat1);
  const int64_t m = s.m;
  const int32_t* nbr = s.nbr + (int64_t)j * R * 2 * m;
  int64_t v[kBlurU];
  int ia[kBlurU][R], ic[kBlurU][R];
#pragma unroll
  for (int u = 0; u < kBlurU; ++u) {
    v[u] = (local * kBlurU + u) * groups + g;
#pragma unroll
    for (int tt = 0; tt < R; ++tt) {
      ia[u][tt] = v[u] < m ? __ldg(nbr + (int64_t)(2 * tt) * m + v[u]) : -1;
      ic[u][tt] = v[u] < m ? __ldg(nbr + (int64_t)(2 * tt + 1) * m + v[u]) : -1;
    }
  }
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 own[kBlurU], sa[kBlurU][R], sc[kBlurU][R];
#pragma unroll
  for (int u = 0; u < kBlurU; ++u) {
    own[u] = v[u] < m ? Store<S>::ldg4(in + v[u] * kp + col) : zero;
#pragma unroll
    for (int tt = 0; tt < R; ++tt) {
      sa[u][tt] = ia[u][tt] >= 0 ? Store<S>::ldg4(in + (int64_t)ia[u][tt] * kp + col) : zero;
      sc[u][tt] = ic[u][tt] >= 0 ? Store<S>::ldg4(in + (int64_t)ic[u][tt] * kp + col) : zero;
    }
  }
#pragma unroll
  for (int u = 0; u < kBlurU; ++u) {
    if (v[u] >= m) continue;
    const float c0 = s.taps[0];
    float4 acc = make_float4(c0 * own[u].x, c0 * own[u].y, c0 * own[u].z, c0 * own[u].w);
#pragma unroll
    for (int tt = 0; tt < R; ++tt) {
      const float wt = s.taps[tt + 1];
      acc.x = fmaf(wt, sa[u][tt].x + sc[u][tt].x, acc.x);
      acc.y = fmaf(wt, sa[u][tt].y + sc[u][tt].y, acc.y);
      acc.z = fmaf(wt, sa[u][tt].z + sc[u][tt].z, acc.z);
      acc.w = fmaf(wt, sa[u][tt].w + sc[u][tt].w, acc.w);
    }
    Store<S>::st4(out + v[u] * kp + col, acc);
  }
  SLOT_LOOP_END
}

// Sparse requests, after kb_blur pass t: list rows back into lat0, epoch t + 1.
template <class S>
__global__ void __launch_bounds__(kST) kb_sparse_store(const Table* __restrict__ T, int t) {
  const int kp = T->kp, G = kp / 4, groups = kST / G;
  const int g = threadIdx.x / G, col = (int)(threadIdx.x % G) * 4;
  SLOT_LOOP(U_BLUR)
  if (!s.sparse || *s.state == 0 || t >= 2 * s.D || g >= groups) continue;
  const int j = t < s.D ? t : 2 * s.D - 1 - t;
  const int64_t base = s.act_off[j], count = s.act_off[j + 1] - base;
  for (int u = 0; u < kBlurU; ++u) {
    const int64_t e = (local * kBlurU + u) * groups + g;
    if (e >= count) break;
    const int64_t v = s.act[base + e];
    Store<S>::st4(static_cast<S*>(s.lat0) + v * kp + col,
                  Store<S>::ld4(static_cast<const S*>(s.stmp) + e * kp + col));
    if (col == 0) s.epoch[v] = t + 1;
  }
  SLOT_LOOP_END
}

// Sparse requests, after their 2D passes: the remaining centre-tap factors.
template <class S>
__global__ void __launch_bounds__(kST) kb_sparse_finish(const Table* __restrict__ T) {
  const int kp = T->kp, G = kp / 4, groups = kST / G;
  const int g = threadIdx.x / G, col = (int)(threadIdx.x % G) * 4;
  SLOT_LOOP(U_VERT)
  if (!s.sparse || *s.state == 0 || g >= groups) continue;
  const int P = 2 * s.D;
  for (int u = 0; u < kBlurU; ++u) {
    const int64_t v = (local * kBlurU + u) * groups + g;
    if (v >= s.m) break;
    const int e = s.epoch[v];
    if (e == P) continue;
    S* row = static_cast<S*>(s.lat0) + v * kp + col;
    const float f = s.g0pow[P - e];
    const float4 x = Store<S>::ld4(row);
    Store<S>::st4(row, make_float4(f * x.x, f * x.y, f * x.z, f * x.w));
  }
  SLOT_LOOP_END
}

// A p = outputscale W lat0 + noise p on training rows, 0 on test rows; partials of <p, Ap>.
template <class S>
__global__ void __launch_bounds__(kST) kb_slice_dot(const Table* __restrict__ T) {
  __shared__ double sh[kST * 4];
  const int kp = T->kp, G = kp / 4, groups = kST / G;
  const int g = threadIdx.x / G, col = (int)(threadIdx.x % G) * 4;
  SLOT_LOOP(U_VEC)
  if (*s.state == 0) continue;  // uniform over the block
  dfloat d[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  const S* lat = static_cast<const S*>(s.lat0);
  if (g < groups) {
    for (int i = 0; i < kVecRows; ++i) {
      const int64_t row = (local * kVecRows + i) * groups + g;
      if (row >= s.n) break;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int c = 0; c < s.D; ++c) {
        const int64_t e = row * s.D + c;
        acc = f4_fma(s.w[e], Store<S>::ld4(lat + (int64_t)s.idx[e] * kp + col), acc);
      }
      const float4 pv = f4_ld(s.p + row * kp + col);
      float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
      if (s.perm[row] < s.n_train) {
        const float a = s.outputscale, b = s.noise;
        res = make_float4(fmaf(b, pv.x, a * acc.x), fmaf(b, pv.y, a * acc.y),
                          fmaf(b, pv.z, a * acc.z), fmaf(b, pv.w, a * acc.w));
      }
      f4_st(s.ap + row * kp + col, res);
      d[0] = df_add(d[0], df_two_prod(pv.x, res.x));
      d[1] = df_add(d[1], df_two_prod(pv.y, res.y));
      d[2] = df_add(d[2], df_two_prod(pv.z, res.z));
      d[3] = df_add(d[3], df_two_prod(pv.w, res.w));
    }
  }
  vb_column_sums(d, kp, s.dpart + local * kp, sh);
  SLOT_LOOP_END
}

// alpha = rho / <p, A p> per active column (a non-positive <p, A p> stops the column).
__global__ void __launch_bounds__(kST) kb_alpha(const Table* __restrict__ T) {
  __shared__ double red[kST], tot[kMaxServeK];
  const int q = blockIdx.x;
  if (q >= T->nslots) return;
  const SlotDev& s = T->s[q];
  if (*s.state == 0) return;
  const int kp = T->kp;
  const int64_t nvb = T->pre[U_VEC][q + 1] - T->pre[U_VEC][q];
  slot_cols_total(s.dpart, nvb, kp, red, tot);
  const int c = threadIdx.x;
  if (c < kp) {
    const double pap = tot[c];
    double a = 0.0;
    if (s.active[c]) {
      if (pap > 0.0 && isfinite(pap)) a = s.rho[c] / pap;
      else s.active[c] = 0;
    }
    s.alpha[c] = a;
  }
}

// x += alpha p, r -= alpha A p on active columns (double-float); partials of <r, r>.
__device__ __forceinline__ void xr_row(const SlotDev& s, int64_t e, const bool (&on)[4],
                                       const dfloat (&a)[4], const dfloat (&na)[4], dfloat (&d)[4]) {
  const float4 p4 = f4_ld(s.p + e), q4 = f4_ld(s.ap + e);
  float4 xh = f4_ld(s.xh + e), xl = f4_ld(s.xl + e), rh = f4_ld(s.rh + e), rl = f4_ld(s.rl + e);
  float* pv = reinterpret_cast<float*>(const_cast<float4*>(&p4));
  float* qv = reinterpret_cast<float*>(const_cast<float4*>(&q4));
  float* xhv = reinterpret_cast<float*>(&xh);
  float* xlv = reinterpret_cast<float*>(&xl);
  float* rhv = reinterpret_cast<float*>(&rh);
  float* rlv = reinterpret_cast<float*>(&rl);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (on[j]) {
      const dfloat x = df_add({xhv[j], xlv[j]}, df_mul_f(a[j], pv[j]));
      const dfloat r = df_add({rhv[j], rlv[j]}, df_mul_f(na[j], qv[j]));
      xhv[j] = x.hi, xlv[j] = x.lo, rhv[j] = r.hi, rlv[j] = r.lo;
    }
    dfloat sq = df_two_prod(rhv[j], rhv[j]);
    sq = df_fast_two_sum(sq.hi, __fmaf_rn(2.f * rhv[j], rlv[j], sq.lo));
    d[j] = df_add(d[j], sq);
  }
  f4_st(s.xh + e, xh);
  f4_st(s.xl + e, xl);
  f4_st(s.rh + e, rh);
  f4_st(s.rl + e, rl);
}

__global__ void __launch_bounds__(kST) kb_update_xr(const Table* __restrict__ T) {
  __shared__ double sh[kST * 4];
  const int kp = T->kp, G = kp / 4, groups = kST / G;
  const int g = threadIdx.x / G, col = (int)(threadIdx.x % G) * 4;
  SLOT_LOOP(U_VEC)
  if (*s.state == 0) continue;
  bool on[4];
  dfloat a[4], na[4];
  dfloat d[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    on[j] = s.active[col + j] != 0;
    a[j] = df_from_double(s.alpha[col + j]);
    na[j] = {-a[j].hi, -a[j].lo};
  }
  if (g < groups) {
    for (int i = 0; i < kVecRows; ++i) {
      const int64_t row = (local * kVecRows + i) * groups + g;
      if (row >= s.n) break;
      xr_row(s, row * kp + col, on, a, na, d);
    }
  }
  vb_column_sums(d, kp, s.dpart + local * kp, sh);
  SLOT_LOOP_END
}

// Convergence check and beta = <r, r>_new / <r, r>_old per active column; the request
// stops when no column is active.  Its state is copied to the host-read flags.
__global__ void __launch_bounds__(kST) kb_check_beta(const Table* __restrict__ T) {
  __shared__ double red[kST], trr[kMaxServeK], trz[kMaxServeK];
  const int q = blockIdx.x;
  if (q >= T->nslots) return;
  const SlotDev& s = T->s[q];
  if (*s.state == 0) {
    if (threadIdx.x == 0) {
      T->flags[2 * q] = 0;
      T->flags[2 * q + 1] = s.state[1];
    }
    return;
  }
  const int kp = T->kp;
  const int64_t nvb = T->pre[U_VEC][q + 1] - T->pre[U_VEC][q];
  const int64_t nvz = T->pre[U_Z][q + 1] - T->pre[U_Z][q];
  const int it = s.state[1] + 1;
  slot_cols_total(s.dpart, nvb, kp, red, trr);
  // preconditioned: beta = <r, z>_new / <r, z>_old; the stopping rule stays on ||r||
  if (s.l) slot_cols_total(s.dpart2, nvz, kp, red, trz);
  const int c = threadIdx.x;
  int go = 0;
  if (c < kp && s.active[c]) {
    const double rr = trr[c], rz = s.l ? trz[c] : rr;
    const double rel = sqrt(rr) / s.bnorm[c];
    s.relres[c] = rel;
    if (rel <= (double)s.tol || it >= s.max_iter || !isfinite(rel)) {
      s.active[c] = 0;
    } else {
      s.beta[c] = rz / s.rho[c];
      s.rho[c] = rz;
      go = 1;
    }
  }
  const int any = __syncthreads_or(go);
  if (threadIdx.x == 0) {
    s.state[1] = it;
    s.state[0] = any;
    T->flags[2 * q] = any;
    T->flags[2 * q + 1] = it;
  }
}

// p = r + beta p on active columns (double-float sum rounded to fp32); p = z + beta p for
// preconditioned requests (z in ap).
__global__ void __launch_bounds__(kST) kb_update_p(const Table* __restrict__ T) {
  const int kp = T->kp, G = kp / 4, groups = kST / G;
  const int g = threadIdx.x / G, col = (int)(threadIdx.x % G) * 4;
  SLOT_LOOP(U_VEC)
  if (*s.state == 0 || g >= groups) continue;
  const bool pre = s.l > 0;
  bool on[4];
  dfloat b[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    on[j] = s.active[col + j] != 0;
    b[j] = df_from_double(s.beta[col + j]);
  }
  for (int i = 0; i < kVecRows; ++i) {
    const int64_t row = (local * kVecRows + i) * groups + g;
    if (row >= s.n) break;
    const int64_t e = row * kp + col;
    float4 p4 = f4_ld(s.p + e);
    const float4 rh = pre ? f4_ld(s.ap + e) : f4_ld(s.rh + e);
    const float4 rl = pre ? make_float4(0.f, 0.f, 0.f, 0.f) : f4_ld(s.rl + e);
    float* pv = reinterpret_cast<float*>(&p4);
    const float* rhv = reinterpret_cast<const float*>(&rh);
    const float* rlv = reinterpret_cast<const float*>(&rl);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (on[j]) {
        const dfloat t = df_add({rhv[j], rlv[j]}, df_mul_f(b[j], pv[j]));
        pv[j] = __fadd_rn(t.hi, t.lo);
      }
    }
    f4_st(s.p + e, p4);
  }
  SLOT_LOOP_END
}

// ---- bulk copies (TMA) into a shared-memory ring, completed on mbarriers -------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
               ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// One contiguous global -> shared copy (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false when `limit` polls fail.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          int limit = kSpinLimit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Rows of one stage of the chunk ring for kp columns: a stage holds rows x (kMaxLd + 2 kp)
// floats, kStages stages in kRingBytes.
__host__ __device__ inline int ring_rows_cap(int kp) {
  const int r = kRingBytes / kStages / ((kMaxLd + 2 * kp) * 4);
  return r < kRingRowsMax ? r : kRingRowsMax;
}

// Chunks of rows [r0, r1) of one request: B ([rows][ld]), rh and, with `lo`, rl ([rows][kp]
// each) land in stage st of the ring, back to back.
struct ChunkRing {
  float* base;       // dynamic shared memory, kStages stages
  int stage_floats;  // ring_rows_cap(kp) (kMaxLd + 2 kp)
  int rows;          // rows per chunk (<= ring_rows_cap(kp))
  bool lo;           // rl is copied too
  uint64_t* bar;     // [kStages]
  uint32_t phase;    // bit st: parity of stage st's next completion
  __device__ float* B(int st) const { return base + (size_t)st * stage_floats; }
};

// Issue chunk k of rows [r0, r1) into stage st (one thread).
__device__ __forceinline__ void ring_issue(const ChunkRing& ring, int st, const SlotDev& s,
                                           int kp, int64_t r0, int64_t r1, int k) {
  const int64_t a = r0 + (int64_t)k * ring.rows;
  const int rows = (int)(r1 - a < ring.rows ? r1 - a : ring.rows);
  const uint32_t bB = (uint32_t)rows * s.ld * 4, bR = (uint32_t)rows * kp * 4;
  float* dst = ring.B(st);
  mbar_expect_tx(&ring.bar[st], bB + (ring.lo ? 2 : 1) * bR);
  bulk_g2s(dst, s.Bh + a * s.ld, bB, &ring.bar[st]);
  bulk_g2s(dst + rows * s.ld, s.rh + a * kp, bR, &ring.bar[st]);
  if (ring.lo) bulk_g2s(dst + rows * s.ld + rows * kp, s.rl + a * kp, bR, &ring.bar[st]);
}

// After a failed wait on chunk k0: record the error, then wait (bounded) for this block's
// chunks k0 .. k1 - 1 still in flight, so that no copy lands after the block has exited.
__device__ void ring_abort(ChunkRing& ring, const Table* T, int k0, int k1) {
  if (threadIdx.x == 0) atomicExch(T->err, 1);
  for (int k = k0; k < k1; ++k) {
    const int st = k % kStages;
    (void)mbar_wait(&ring.bar[st], (ring.phase >> st) & 1u);
    ring.phase ^= 1u << st;
  }
}

__device__ __forceinline__ void ring_init(ChunkRing& ring, float* base, uint64_t* bar, int kp,
                                          bool lo) {
  ring.base = base;
  ring.stage_floats = ring_rows_cap(kp) * (kMaxLd + 2 * kp);
  ring.rows = ring_rows_cap(kp);
  ring.lo = lo;
  ring.bar = bar;
  ring.phase = 0;
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(&bar[st], 1);
    mbar_fence_init();
  }
  __syncthreads();
}

// ---- preconditioner apply z = P^-1 r (requests with l > 0) ----------------------------
// P^-1 r = (r - B Minv B^T r) / noise (Woodbury), in five table-driven kernels: B^T r
// partials, two ordered sums, Minv (B^T r), and z with the <r, z> partials.

// Per-virtual-block partial of B^T r over kBtVbRows rows, with r taken as its fp32 part
// rh (the low part rl is below the preconditioner's own rounding): the rows stream through
// the chunk ring (bulk copies, kStages chunks in flight); warp w takes rows w, w + 8, ...
// of each chunk, lane owns the B columns 4 lane .. 4 lane + 3 (one float4 of the row)
// against KC columns of r broadcast from shared memory (fp32 sums).  The warps are added in
// a fixed order in shared memory and the block writes btpart[local][ld][kp].  kp > KC: one
// pass per KC columns (B streamed again).
template <int KC>
__global__ void __launch_bounds__(kST, 1) kb_bt(const Table* __restrict__ T) {
  extern __shared__ __align__(128) float dsm[];
  __shared__ __align__(8) uint64_t bar[kStages];
  __shared__ __align__(16) float red[KC * kMaxLd];  // [c][j]
  constexpr int kWarps = kST / 32;
  const int kp = T->kp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ChunkRing ring;
  ring_init(ring, dsm, bar, kp, false);
  SLOT_LOOP(U_BT)
  if (*s.state == 0 || s.l == 0) continue;  // uniform over the block
  const int ld = s.ld;
  const int64_t r0 = local * kBtVbRows;
  const int64_t r1 = r0 + kBtVbRows < s.n ? r0 + kBtVbRows : s.n;
  const int nch = (int)ceil_div(r1 - r0, ring.rows);
  const bool mine = 4 * lane < ld;
  for (int c_off = 0; c_off < kp; c_off += KC) {
    const int kc = kp - c_off < KC ? kp - c_off : KC;
    float acc[4][KC];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < KC; ++c) acc[a][c] = 0.f;
    if (threadIdx.x == 0)
      for (int k = 0; k < nch && k < kStages; ++k) ring_issue(ring, k, s, kp, r0, r1, k);
    for (int k = 0; k < nch; ++k) {
      const int st = k % kStages;
      const bool ok =
          __syncthreads_and(mbar_wait(&ring.bar[st], (ring.phase >> st) & 1u, T->wait_limit));
      if (!ok) {
        ring_abort(ring, T, k, k + kStages < nch ? k + kStages : nch);
        return;
      }
      ring.phase ^= 1u << st;
      const int64_t a0 = r0 + (int64_t)k * ring.rows;
      const int rows = (int)(r1 - a0 < ring.rows ? r1 - a0 : ring.rows);
      const float* Bs = ring.B(st);
      const float* Hs = Bs + rows * ld;
#pragma unroll 2
      for (int rr = warp; rr < rows; rr += kWarps) {
        const float4 b = mine ? *reinterpret_cast<const float4*>(Bs + rr * ld + 4 * lane)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        float rv[KC];
#pragma unroll
        for (int g = 0; g < KC / 4; ++g) {
          const float4 h = 4 * g < kc
                               ? *reinterpret_cast<const float4*>(Hs + rr * kp + c_off + 4 * g)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
          rv[4 * g + 0] = h.x;
          rv[4 * g + 1] = h.y;
          rv[4 * g + 2] = h.z;
          rv[4 * g + 3] = h.w;
        }
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          acc[0][c] = fmaf(b.x, rv[c], acc[0][c]);
          acc[1][c] = fmaf(b.y, rv[c], acc[1][c]);
          acc[2][c] = fmaf(b.z, rv[c], acc[2][c]);
          acc[3][c] = fmaf(b.w, rv[c], acc[3][c]);
        }
      }
      __syncthreads();  // stage st is free again
      if (threadIdx.x == 0 && k + kStages < nch) ring_issue(ring, st, s, kp, r0, r1, k + kStages);
    }
    for (int w = 0; w < kWarps; ++w) {
      if (warp == w && mine)
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          float4* dst = reinterpret_cast<float4*>(red + c * kMaxLd + 4 * lane);
          const float4 prev = w == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : *dst;
          *dst = make_float4(prev.x + acc[0][c], prev.y + acc[1][c], prev.z + acc[2][c],
                             prev.w + acc[3][c]);
        }
      __syncthreads();
    }
    for (int o = threadIdx.x; o < ld * kc; o += kST) {
      const int j = o / kc, c = o - j * kc;
      s.btpart[(local * ld + j) * kp + c_off + c] = red[c * kMaxLd + j];
    }
    __syncthreads();
  }
  SLOT_LOOP_END
}

// First-level sums of the B^T r partials: virtual block (segment g, chunk h) adds the
// partials g kBtSeg .. g kBtSeg + kBtSeg - 1 of outputs h kST .. h kST + kST - 1 in order.
__global__ void __launch_bounds__(kST) kb_bt_seg(const Table* __restrict__ T) {
  const int kp = T->kp;
  SLOT_LOOP(U_BTS)
  if (*s.state == 0 || s.l == 0) continue;
  const int cnt = s.ld * kp;
  const int nch = (cnt + kST - 1) / kST;
  const int64_t g = local / nch;
  const int o = (int)(local - g * nch) * kST + threadIdx.x;
  if (o >= cnt) continue;
  const int64_t nvb = T->pre[U_BT][q + 1] - T->pre[U_BT][q];
  const int64_t b0 = g * kBtSeg, b1 = b0 + kBtSeg < nvb ? b0 + kBtSeg : nvb;
  float t = 0.f;
  for (int64_t b = b0; b < b1; ++b) t += s.btpart[b * cnt + o];
  s.bt2[g * cnt + o] = t;
  SLOT_LOOP_END
}

// t = B^T r: the segment sums added in order in fp64, one output per thread.
__global__ void __launch_bounds__(kST) kb_bt_total(const Table* __restrict__ T) {
  const int kp = T->kp;
  SLOT_LOOP(U_BTT)
  if (*s.state == 0 || s.l == 0) continue;
  const int cnt = s.ld * kp;
  const int o = (int)local * kST + threadIdx.x;
  if (o >= cnt) continue;
  const int64_t nseg = ceil_div(T->pre[U_BT][q + 1] - T->pre[U_BT][q], kBtSeg);
  double t = 0.0;
  for (int64_t g = 0; g < nseg; ++g) t += (double)s.bt2[g * cnt + o];
  s.tvec[o] = t;
  SLOT_LOOP_END
}

// u = Minv t (fp64) on the first l rows, 0 below; stored fp32 [ld][kp].  Four lanes per
// output, each a quarter of the dot product, combined by shuffles in a fixed order.
__global__ void __launch_bounds__(kST) kb_minv(const Table* __restrict__ T) {
  const int kp = T->kp;
  SLOT_LOOP(U_MINV)
  if (*s.state == 0 || s.l == 0) continue;  // uniform over the block
  const int o = (int)(local * kST + threadIdx.x) / 4, part = threadIdx.x & 3;
  const int cnt = s.ld * kp;
  const int j = o / kp, c = o - j * kp;
  double a = 0.0;
  if (o < cnt && j < s.l)
    for (int i = part; i < s.l; i += 4) a += s.Minv[j * s.l + i] * s.tvec[i * kp + c];
  a += __shfl_xor_sync(0xffffffffu, a, 1);
  a += __shfl_xor_sync(0xffffffffu, a, 2);
  if (o < cnt && part == 0) s.u[o] = (float)a;
  SLOT_LOOP_END
}

// TF32 tensor-core pieces: round to tf32 (nearest, ties away), the 3xTF32 split x = hi + lo
// (hi·hi + hi·lo + lo·hi keeps about fp32 accuracy), and one m16n8k8 MMA with fp32 sums.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
// D (16 x 8) += A (16 x 8, row-major) B (8 x 8, column-major); lane = 4 g + t holds
// A[g][t], A[g + 8][t], A[g][t + 4], A[g + 8][t + 4]; B[t][g], B[t + 4][g];
// D[g][2t], D[g][2t + 1], D[g + 8][2t], D[g + 8][2t + 1].
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// z = (r - B u) / noise, written into ap (free between the x, r update and the next
// product), and the virtual block's column sums of r z into dpart2.  The block's kZVbRows
// rows stream through the chunk ring; warp w takes the 16-row tiles w, w + 8, ... of each
// chunk and forms B u on the tensor cores (m16n8k8, 3xTF32 split, NT tiles of 8 columns),
// A fragments from the staged B rows, B fragments from u split once into shared memory.  The epilogue
// reads r from the stage.  The column sums of r z are double-float per lane, combined over
// the lanes of a column by a fixed butterfly and over the warps in order.  Test rows have
// zero B rows and zero r, so z = 0 there.
template <int NT>
__global__ void __launch_bounds__(kST, 1) kb_apply_z(const Table* __restrict__ T) {
  extern __shared__ __align__(128) float dsm[];
  __shared__ __align__(8) uint64_t bar[kStages];
  __shared__ double red[kST / 32][8 * NT];
  constexpr int kWarps = kST / 32;
  const int kp = T->kp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // u split once per virtual block: uh = tf32(u), ul = tf32(u - uh), [kMaxLd][kp] each
  uint32_t* uh = reinterpret_cast<uint32_t*>(dsm);
  uint32_t* ul = uh + kMaxLd * kp;
  ChunkRing ring;
  ring_init(ring, dsm + 2 * kMaxLd * kp, bar, kp, true);
  ring.rows = ring.rows / 16 * 16;
  SLOT_LOOP(U_Z)
  if (*s.state == 0 || s.l == 0) continue;  // uniform over the block
  const int ld = s.ld, ksteps = (ld + 7) / 8;
  const int64_t r0 = local * kZVbRows;
  const int64_t r1 = r0 + kZVbRows < s.n ? r0 + kZVbRows : s.n;
  const int nch = (int)ceil_div(r1 - r0, ring.rows);
  if (threadIdx.x == 0)
    for (int k = 0; k < nch && k < kStages; ++k) ring_issue(ring, k, s, kp, r0, r1, k);
  for (int e = threadIdx.x; e < ld * kp; e += kST) tf32_split(s.u[e], uh[e], ul[e]);
  dfloat acc[NT][2];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = {0.f, 0.f};
  for (int k = 0; k < nch; ++k) {
    const int st = k % kStages;
    const bool ok =
        __syncthreads_and(mbar_wait(&ring.bar[st], (ring.phase >> st) & 1u, T->wait_limit));
    if (!ok) {
      ring_abort(ring, T, k, k + kStages < nch ? k + kStages : nch);
      return;
    }
    ring.phase ^= 1u << st;
    const int64_t a0 = r0 + (int64_t)k * ring.rows;
    const int rows = (int)(r1 - a0 < ring.rows ? r1 - a0 : ring.rows);
    const float* Bs = ring.B(st);
    const float* Hs = Bs + rows * ld;
    const float* Ls = Hs + rows * kp;
    for (int rt = warp * 16; rt < rows; rt += kWarps * 16) {
      float d[NT][4];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
      // rows past the chunk read stale stage data; their outputs are not stored
      const float* ra = Bs + (rt + g) * ld;
      const float* rb = ra + 8 * ld;
      for (int ks = 0; ks < ksteps; ++ks) {
        const int j0 = ks * 8 + t, j1 = j0 + 4;
        const bool in0 = j0 < ld, in1 = j1 < ld;
        uint32_t ah[4], al[4];
        tf32_split(in0 ? ra[j0] : 0.f, ah[0], al[0]);
        tf32_split(in0 ? rb[j0] : 0.f, ah[1], al[1]);
        tf32_split(in1 ? ra[j1] : 0.f, ah[2], al[2]);
        tf32_split(in1 ? rb[j1] : 0.f, ah[3], al[3]);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int n = 8 * nt + g;
          const bool n_in = n < kp;
          const uint32_t bh0 = in0 && n_in ? uh[j0 * kp + n] : 0u;
          const uint32_t bl0 = in0 && n_in ? ul[j0 * kp + n] : 0u;
          const uint32_t bh1 = in1 && n_in ? uh[j1 * kp + n] : 0u;
          const uint32_t bl1 = in1 && n_in ? ul[j1 * kp + n] : 0u;
          mma_tf32(d[nt], ah, bh0, bh1);
          mma_tf32(d[nt], ah, bl0, bl1);
          mma_tf32(d[nt], al, bh0, bh1);
        }
      }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int c = 8 * nt + 2 * t;
        if (c >= kp) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int row = rt + g + 8 * half;
          if (row >= rows) continue;
          const float2 h = *reinterpret_cast<const float2*>(Hs + row * kp + c);
          const float2 lo = *reinterpret_cast<const float2*>(Ls + row * kp + c);
          const float x0 = __fadd_rn(h.x, lo.x), x1 = __fadd_rn(h.y, lo.y);
          const float z0 = (x0 - d[nt][2 * half]) * s.inv_noise;
          const float z1 = (x1 - d[nt][2 * half + 1]) * s.inv_noise;
          *reinterpret_cast<float2*>(s.ap + (a0 + row) * kp + c) = make_float2(z0, z1);
          acc[nt][0] = df_add(acc[nt][0], df_two_prod(x0, z0));
          acc[nt][1] = df_add(acc[nt][1], df_two_prod(x1, z1));
        }
      }
    }
    __syncthreads();  // stage st is free again
    if (threadIdx.x == 0 && k + kStages < nch) ring_issue(ring, st, s, kp, r0, r1, k + kStages);
  }
  // column sums: the 8 lanes of a column (same t) by a fixed butterfly, then the warps in order
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      double v = df_to_double(acc[nt][e]);
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      const int c = 8 * nt + 2 * t + e;
      if (g == 0 && c < kp) red[warp][c] = v;
    }
  __syncthreads();
  if ((int)threadIdx.x < kp) {
    double v = 0.0;
    for (int w = 0; w < kWarps; ++w) v += red[w][threadIdx.x];
    s.dpart2[local * kp + threadIdx.x] = v;
  }
  __syncthreads();
  SLOT_LOOP_END
}

// Dynamic shared memory of kb_bt and kb_apply_z for kp columns.
size_t ring_smem_bytes(int kp) {
  return (size_t)kStages * ring_rows_cap(kp) * (kMaxLd + 2 * kp) * 4;
}
size_t apply_z_smem_bytes(int kp) { return ring_smem_bytes(kp) + 2 * (size_t)kMaxLd * kp * 4; }

// kb_apply_z for the server's kp: NT = kp / 8 rounded up tiles of 8 columns.
void launch_apply_z(int kp, const Table* T, cudaStream_t st) {
  const size_t sm = apply_z_smem_bytes(kp);
  switch ((kp + 7) / 8) {
    case 1: kb_apply_z<1><<<kRingGrid, kST, sm, st>>>(T); break;
    case 2: kb_apply_z<2><<<kRingGrid, kST, sm, st>>>(T); break;
    case 3: kb_apply_z<3><<<kRingGrid, kST, sm, st>>>(T); break;
    default: kb_apply_z<4><<<kRingGrid, kST, sm, st>>>(T); break;
  }
}
cudaError_t apply_z_smem_attributes(int kp) {
  const int sm = (int)apply_z_smem_bytes(kp);
  cudaError_t e =
      cudaFuncSetAttribute(kb_apply_z<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_apply_z<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_apply_z<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_apply_z<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

// kb_bt for the server's kp: KC = min(kp, 16) columns per pass.
void launch_bt(int kp, const Table* T, cudaStream_t st) {
  const size_t sm = ring_smem_bytes(kp);
  switch (kp < 16 ? kp : 16) {
    case 4: kb_bt<4><<<kRingGrid, kST, sm, st>>>(T); break;
    case 8: kb_bt<8><<<kRingGrid, kST, sm, st>>>(T); break;
    case 12: kb_bt<12><<<kRingGrid, kST, sm, st>>>(T); break;
    default: kb_bt<16><<<kRingGrid, kST, sm, st>>>(T); break;
  }
}
cudaError_t bt_smem_attributes(int kp) {
  const int sm = (int)ring_smem_bytes(kp);
  cudaError_t e = cudaFuncSetAttribute(kb_bt<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_bt<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_bt<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_bt<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

// ---- per-request set-up and read-out (single-request launches) ------------------------
// Partials of <r, r> for the initial residual (the same virtual blocks as the iteration).
__global__ void __launch_bounds__(kST) kb_norm(const Table* __restrict__ T) {
  __shared__ double sh[kST * 4];
  const int kp = T->kp, G = kp / 4, groups = kST / G;
  const int g = threadIdx.x / G, col = (int)(threadIdx.x % G) * 4;
  SLOT_LOOP(U_VEC)
  dfloat d[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  if (g < groups) {
    for (int i = 0; i < kVecRows; ++i) {
      const int64_t row = (local * kVecRows + i) * groups + g;
      if (row >= s.n) break;
      const float4 rh = f4_ld(s.rh + row * kp + col);
      d[0] = df_add(d[0], df_two_prod(rh.x, rh.x));
      d[1] = df_add(d[1], df_two_prod(rh.y, rh.y));
      d[2] = df_add(d[2], df_two_prod(rh.z, rh.z));
      d[3] = df_add(d[3], df_two_prod(rh.w, rh.w));
    }
  }
  vb_column_sums(d, kp, s.dpart + local * kp, sh);
  SLOT_LOOP_END
}

__global__ void __launch_bounds__(kST) kb_init_scalars(const Table* __restrict__ T) {
  __shared__ double red[kST], trr[kMaxServeK], trz[kMaxServeK];
  const int q = blockIdx.x;
  if (q >= T->nslots) return;
  const SlotDev& s = T->s[q];
  const int kp = T->kp;
  const int64_t nvb = T->pre[U_VEC][q + 1] - T->pre[U_VEC][q];
  const int64_t nvz = T->pre[U_Z][q + 1] - T->pre[U_Z][q];
  slot_cols_total(s.dpart, nvb, kp, red, trr);
  if (s.l) slot_cols_total(s.dpart2, nvz, kp, red, trz);
  const int c = threadIdx.x;
  int on = 0;
  if (c < kp) {
    const double rr = trr[c];
    s.rho[c] = s.l ? trz[c] : rr;
    s.bnorm[c] = sqrt(rr);
    s.alpha[c] = 0.0;
    s.beta[c] = 0.0;
    on = (rr > 0.0 && 1.0 > (double)s.tol && s.max_iter > 0) ? 1 : 0;
    s.relres[c] = rr > 0.0 ? 1.0 : 0.0;
    s.active[c] = on;
  }
  const int any = __syncthreads_or(on);
  if (threadIdx.x == 0) {
    s.state[0] = any;
    s.state[1] = 0;
  }
}

// Probe right-hand sides in the caller's order: column 1 + s of test row t holds z_s[t];
// the last column (kp - 1 > S) holds 1 on the training rows, for the row sums of K~_XX.
__global__ void k_probe_fill(float* __restrict__ V, int64_t n_all, int64_t n_train, int kp,
                             int S, uint64_t seed) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_all * kp) return;
  const int64_t i = e / kp;
  const int c = (int)(e - i * kp);
  float v = 0.f;
  if (i >= n_train) {
    if (c >= 1 && c <= S) v = rademacher_pm(seed, i - n_train, c - 1, S);
  } else if (c == kp - 1) {
    v = 1.f;
  }
  V[e] = v;
}

// Largest training-row sum max_i KZ[i][kp - 1] (i < n_train) of outputscale K~_XX; the
// entries are non-negative, so the float bits order like the values (*out preset to 0).
__global__ void k_rowsum_max(const float* __restrict__ KZ, int64_t n_train, int kp,
                             int* __restrict__ out) {
  __shared__ float red[256];
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_train;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, KZ[i * kp + kp - 1]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int h = blockDim.x / 2; h >= 1; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, __float_as_int(fmaxf(red[0], 0.f)));
}

// b (locality order): training rows [y, (KX* z)_1..S, 0 ...], test rows 0; r = p = b,
// x = 0.  KZ is the probe product in the caller's order.
__global__ void k_rhs(const int32_t* __restrict__ perm, const float* __restrict__ y,
                      const float* __restrict__ KZ, int64_t n_all, int64_t n_train, int kp,
                      int S, float* __restrict__ xh, float* __restrict__ xl,
                      float* __restrict__ rh, float* __restrict__ rl, float* __restrict__ p) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_all * kp) return;
  const int64_t row = e / kp;
  const int c = (int)(e - row * kp);
  const int64_t i = perm[row];
  float b = 0.f;
  if (i < n_train) b = c == 0 ? y[i] : (c <= S ? KZ[i * kp + c] : 0.f);
  xh[e] = 0.f;
  xl[e] = 0.f;
  rh[e] = b;
  rl[e] = 0.f;
  p[e] = b;
}

__global__ void k_x_sum(const float* __restrict__ xh, const float* __restrict__ xl,
                        float* __restrict__ out, int64_t count) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) out[e] = __fadd_rn(xh[e], xl[e]);
}

// mean[t] = (K*X W)[t][0]; var[t] = outputscale - (1/S) sum_s z_s[t] (K*X W)[t][1 + s].
__global__ void k_predict(const int32_t* __restrict__ perm, const float* __restrict__ KW,
                          int64_t n_all, int64_t n_train, int kp, int S, uint64_t seed,
                          float outputscale, float* __restrict__ mean, float* __restrict__ var) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_all) return;
  const int64_t i = perm[row];
  if (i < n_train) return;
  const int64_t t = i - n_train;
  const float* o = KW + row * kp;
  mean[t] = o[0];
  double acc = 0.0;
  for (int s = 0; s < S; ++s) acc += (double)rademacher_pm(seed, t, s, S) * (double)o[1 + s];
  var[t] = S > 0 ? (float)((double)outputscale - acc / S) : 0.f;
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace sgp

using namespace sgp;

// ---- host engine ------------------------------------------------------------------------
// Requests are grouped into lanes by dimension class and per-iteration work class; each
// lane is its own batch (device table, CUDA graph, stream), so a small request never
// iterates in lockstep with one a hundred times its size, and lanes run concurrently on
// the GPU.  sgp_server_step harvests lanes whose round of iterations has finished,
// admits queued requests, relaunches idle lanes and then waits (briefly) for the next
// lane to finish.
namespace {

constexpr int kStepWaitUs = 2000;  // longest wait of one step for a lane to finish
constexpr int kSetupThreads = 3;   // concurrent request set-ups

struct Lane;

struct Request {
  long long id = 0;
  sgp_request in{};
  sgp_request_stats st{};
  unsigned long long bound = 0;
  unsigned long long held = 0;  // accounted against the budget while active
  Lattice* L = nullptr;
  float *xh = nullptr, *xl = nullptr, *rh = nullptr, *rl = nullptr, *p = nullptr, *ap = nullptr;
  double* dpart = nullptr;
  double* scal = nullptr;  // rho, bnorm, relres, alpha, beta: [5][kp]
  int* ints = nullptr;     // active [kp], state [2], bulk-copy error [1]
  float* outd = nullptr;   // mean, var: [2][ns]
  Table* dtab1 = nullptr;  // one-request table for the set-up kernels
  cudaEvent_t ready = nullptr;
  bool waited = false;     // the lane's stream has waited for `ready`
  int64_t vb[U_KINDS] = {};
  Lane* lane = nullptr;
  bool from_cache = false;  // R->L is a resident lattice owned by the server's cache
  // rank-l Nystrom preconditioner (l = 0: none) and the condition estimate behind it
  int l = 0, ld = 0;
  double kappa = 0.0;
  float* Bh = nullptr;
  double* Minv = nullptr;
  float *btpart = nullptr, *bt2 = nullptr, *u = nullptr;
  double *tvec = nullptr, *dpart2 = nullptr;
  std::vector<void*> ptrs;
  std::string setup_error;  // message of a failed set-up (set on the set-up thread)
};

struct Lane {
  int key = 0;
  int value_dtype = 0;  // SGP_VALUES_* of every request in the lane
  cudaStream_t st = nullptr;
  Table* dtab = nullptr;
  int* dflags = nullptr;
  int* hflags = nullptr;  // pinned
  cudaEvent_t ev = nullptr;
  std::unique_ptr<Table> htab;
  std::vector<Request*> active;  // the first ntab are in the launched table, in order
  int ntab = 0;
  bool in_flight = false;
  bool dirty = true;
  std::map<int, cudaGraphExec_t> graphs;  // by Dmax
  std::map<int, int> graph_kernels;
};

}  // namespace

struct sgp_server {
  sgp_server_opts o{};
  int kp = 4, S = 0;
  int device = 0;
  cudaStream_t bs = nullptr;  // stream for releasing requests that failed their set-up
  std::chrono::steady_clock::time_point t0;
  long long next_id = 1;
  std::deque<Request*> queue;
  std::map<int, std::unique_ptr<Lane>> lanes;
  std::map<long long, std::unique_ptr<Request>> reqs;
  int n_active = 0;  // admitted: in set-up or in a lane
  unsigned long long in_use = 0;
  int peak_active = 0;

  // Set-up threads (kSetupThreads, each with its own stream): admitted requests are
  // uploaded, built and given their right-hand sides there, so that the stepping thread
  // keeps relaunching lanes and several builds overlap on the GPU.
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv;
  // Resident lattices for reuse (sgp_request.lattice_key).  Set-up threads take an idle
  // one (busy = true) under mu; the stepping thread inserts, returns and evicts.
  struct Cached {
    Lattice* L = nullptr;
    unsigned long long bytes = 0;
    float outputscale = 0.f;
    bool busy = false;
    double last_us = 0.0;
  };
  std::map<unsigned long long, Cached> cache;                // guarded by mu
  unsigned long long cache_bytes = 0;                         // stepping thread
  std::deque<Request*> to_setup;                              // guarded by mu
  std::vector<std::pair<Request*, sgp_status>> setup_done;    // guarded by mu
  bool stop = false;                                          // guarded by mu
  // SGP_FAULT=ring_wait: the next lane round that applies a preconditioner runs its
  // bulk-copy waits with a limit of 0 polls (they give up at once), once
  bool inject_ring_wait = false;                              // stepping thread
};

namespace {

double now_us(const sgp_server* S) { return 1e6 * seconds_since(S->t0); }

#define SRV_CHECK(expr, what)                                \
  do {                                                       \
    cudaError_t e_ = (expr);                                 \
    if (e_ != cudaSuccess) return cuda_status(e_, what);     \
  } while (0)

bool expired(const sgp_server* S, const Request* R) {
  return R->in.timeout_us > 0.0 && now_us(S) > R->st.arrival_us + R->in.timeout_us;
}

void fill_slot(const sgp_server* S, const Request* R, SlotDev& s) {
  const Lattice* L = R->L;
  s.n = L->n;
  s.n_train = R->in.n;
  s.m = L->m;
  s.D = L->D;
  s.r = L->r;
  s.nseg = L->nseg;
  s.nmed = L->nmed;
  s.nhuge = L->nhuge;
  s.perm = L->perm;
  s.idx = L->idx;
  s.w = L->w;
  s.items = L->items;
  s.seg = L->seg;
  s.med = L->med_rows;
  s.huge = L->huge_rows;
  s.nbr = L->nbr;
  for (int t = 0; t <= kMaxOrder; ++t) s.taps[t] = t <= L->r ? (float)L->half[t] : 0.f;
  s.outputscale = L->outputscale;
  s.noise = R->in.noise;
  s.lat0 = L->lat[0];
  s.lat1 = L->lat[1];
  s.spart = L->partial;
  s.xh = R->xh;
  s.xl = R->xl;
  s.rh = R->rh;
  s.rl = R->rl;
  s.p = R->p;
  s.ap = R->ap;
  s.dpart = R->dpart;
  const int kp = S->kp;
  s.rho = R->scal;
  s.bnorm = R->scal + kp;
  s.relres = R->scal + 2 * kp;
  s.alpha = R->scal + 3 * kp;
  s.beta = R->scal + 4 * kp;
  s.active = R->ints;
  s.state = R->ints + kp;
  s.max_iter = S->o.max_iter;
  s.tol = (float)S->o.tol;
  s.sparse = L->sparse ? 1 : 0;
  s.act = L->act;
  s.act_off = L->act_off_dev;
  s.epoch = L->epoch;
  s.stmp = L->act_tmp;
  s.g0pow = L->g0pow;
  s.l = R->l;
  s.ld = R->ld;
  s.inv_noise = 1.f / R->in.noise;
  s.Bh = R->Bh;
  s.Minv = R->Minv;
  s.btpart = R->btpart;
  s.bt2 = R->bt2;
  s.tvec = R->tvec;
  s.u = R->u;
  s.dpart2 = R->dpart2;
}

void unit_counts(const sgp_server* S, const Request* R, int64_t (&vb)[U_KINDS]) {
  const Lattice* L = R->L;
  const int groups = groups_of(S->kp);
  vb[U_SPLAT] = ceil_div(L->nseg, groups);
  vb[U_MED] = ceil_div(L->nmed, groups);
  vb[U_HUGE] = L->nhuge;
  vb[U_BLUR] = ceil_div(L->sparse ? L->act_max : L->m, (int64_t)groups * kBlurU);
  vb[U_VEC] = ceil_div(L->n, (int64_t)groups * kVecRows);
  vb[U_VERT] = L->sparse ? ceil_div(L->m, (int64_t)groups * kBlurU) : 0;
  const int64_t nch = ceil_div((int64_t)R->ld * S->kp, kST);  // output chunks of B^T r
  vb[U_BT] = R->l ? ceil_div(L->n, kBtVbRows) : 0;
  vb[U_BTS] = R->l ? nch * ceil_div(vb[U_BT], kBtSeg) : 0;
  vb[U_BTT] = R->l ? nch : 0;
  vb[U_MINV] = R->l ? ceil_div((int64_t)R->ld * S->kp * 4, kST) : 0;
  vb[U_Z] = R->l ? ceil_div(L->n, kZVbRows) : 0;
}

// Lane of a built request: dimension class (D <= 4, 8, ..., 128), work class (blur,
// slice and preconditioner volume per iteration, classes a factor 8 apart) and the value
// type of its lattice (a BF16 server keeps fp32 values for ill-conditioned requests).
int lane_key(const sgp_server* S, const Request* R) {
  const Lattice* L = R->L;
  if (!S->o.lane_classes) return L->value_dtype == SGP_VALUES_BF16 ? 1 << 16 : 0;
  int dclass = 0;
  while ((4 << dclass) < L->D) ++dclass;
  const double work = ((double)L->m + (double)L->n) * L->D * S->kp + 2.0 * L->n * R->ld;
  const int wclass = std::max(0, (int)std::floor(std::log(std::max(work, 1.0)) / std::log(8.0)));
  return (L->value_dtype == SGP_VALUES_BF16 ? 1 << 16 : 0) + dclass * 64 + std::min(wclass, 63);
}

void release(sgp_server* S, Request* R, cudaStream_t st) {
  for (void* p : R->ptrs) (void)cudaFreeAsync(p, st);
  R->ptrs.clear();
  if (R->from_cache) {  // hand the resident lattice back
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->cache.find(R->in.lattice_key);
    if (it != S->cache.end()) {
      it->second.busy = false;
      it->second.last_us = now_us(S);
    }
    R->L = nullptr;
    R->from_cache = false;
  }
  if (R->L) {
    sgp_set_stream(R->L, st);
    sgp_lattice_free(R->L);
    R->L = nullptr;
  }
  if (R->ready) {
    cudaEventDestroy(R->ready);
    R->ready = nullptr;
  }
  S->in_use -= R->held;
  R->held = 0;
  clear_pending_error();
}

// Upload, build, right-hand sides and CG start of one request on the set-up stream.
sgp_status setup(sgp_server* S, Request* R, cudaStream_t st, Table& t1) {
  const sgp_request& in = R->in;
  const int64_t n_all = in.n + in.ns;
  const int d = in.d, kp = S->kp;
  auto get = [&](void** p, size_t bytes) {
    cudaError_t e = dev_malloc(p, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) R->ptrs.push_back(*p);
    return e;
  };
  struct Scratch {  // inputs and probe products, released (stream-ordered) on return
    cudaStream_t st;
    std::vector<void*> p;
    ~Scratch() {
      for (void* x : p) (void)cudaFreeAsync(x, st);
    }
    cudaError_t get(void** x, size_t bytes) {
      cudaError_t e = dev_malloc(x, std::max<size_t>(bytes, 16), st);
      if (e == cudaSuccess) p.push_back(*x);
      return e;
    }
  } tmp{st, {}};
  float* yd = nullptr;
  SRV_CHECK(tmp.get((void**)&yd, (size_t)in.n * sizeof(float)), "alloc y");
  SRV_CHECK(cudaMemcpyAsync(yd, in.y, (size_t)in.n * sizeof(float), cudaMemcpyHostToDevice, st),
            "copy y");
  if (in.lattice_key) {  // a resident lattice of the same points, if idle
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->cache.find(in.lattice_key);
    if (it != S->cache.end() && !it->second.busy && it->second.L->n == n_all &&
        it->second.L->d == d && it->second.outputscale == in.outputscale) {
      it->second.busy = true;
      R->L = it->second.L;
      R->from_cache = true;
      R->st.lattice_reused = 1;
    }
  }
  sgp_status s = SGP_OK;
  if (!R->from_cache) {
    float *Xd = nullptr, *lsd = nullptr;
    SRV_CHECK(tmp.get((void**)&Xd, (size_t)n_all * d * sizeof(float)), "alloc X");
    SRV_CHECK(tmp.get((void**)&lsd, (size_t)d * sizeof(float)), "alloc ls");
    SRV_CHECK(cudaMemcpyAsync(Xd, in.X, (size_t)in.n * d * sizeof(float), cudaMemcpyHostToDevice,
                              st),
              "copy X");
    SRV_CHECK(cudaMemcpyAsync(Xd + in.n * d, in.Xs, (size_t)in.ns * d * sizeof(float),
                              cudaMemcpyHostToDevice, st),
              "copy Xs");
    SRV_CHECK(cudaMemcpyAsync(lsd, in.lengthscales, d * sizeof(float), cudaMemcpyHostToDevice, st),
              "copy ls");
    sgp_opts lo;
    sgp_opts_init(&lo);
    lo.order_r = S->o.order_r;
    lo.kernel = S->o.kernel;
    lo.spacing_s = S->o.spacing_s;
    lo.outputscale = in.outputscale;
    lo.value_dtype = S->o.value_dtype;
    lo.stream = st;
    s = sgp_lattice_build(Xd, lsd, n_all, d, &lo, &R->L);
    if (s != SGP_OK) return s;
  }
  Lattice* L = R->L;
  R->st.m = L->m;
  s = ensure_lattice_values(L, kp, st);
  if (s != SGP_OK) return s;
  R->l = R->ld = 0;
  unit_counts(S, R, R->vb);
  const size_t vec = (size_t)n_all * kp * sizeof(float);
  float** vecs[6] = {&R->xh, &R->xl, &R->rh, &R->rl, &R->p, &R->ap};
  for (float** v : vecs) SRV_CHECK(get((void**)v, vec), "alloc CG vectors");
  SRV_CHECK(get((void**)&R->dpart, (size_t)R->vb[U_VEC] * kp * sizeof(double)), "alloc partials");
  SRV_CHECK(get((void**)&R->scal, 5 * (size_t)kp * sizeof(double)), "alloc scalars");
  SRV_CHECK(get((void**)&R->ints, ((size_t)kp + 3) * sizeof(int)), "alloc flags");
  SRV_CHECK(cudaMemsetAsync(R->ints, 0, ((size_t)kp + 3) * sizeof(int), st), "clear flags");
  SRV_CHECK(get((void**)&R->outd, 2 * (size_t)in.ns * sizeof(float)), "alloc outputs");
  SRV_CHECK(get((void**)&R->dtab1, sizeof(Table)), "alloc table");
  // right-hand sides: y and KX* z_s (one product of the probe columns, caller's order)
  float *Vz = nullptr, *KZ = nullptr;
  SRV_CHECK(tmp.get((void**)&Vz, vec), "alloc probes");
  SRV_CHECK(tmp.get((void**)&KZ, vec), "alloc probes");
  const unsigned g = (unsigned)ceil_div(n_all * kp, 256);
  k_probe_fill<<<g, 256, 0, st>>>(Vz, n_all, in.n, kp, S->S, in.seed);
  note_launches(1);
  enqueue_mvm(L, Vz, kp, SGP_BLUR_SYMMETRIC, L->outputscale, 0.f, KZ, st);
  k_rhs<<<g, 256, 0, st>>>(L->perm, yd, KZ, n_all, in.n, kp, S->S, R->xh, R->xl, R->rh, R->rl,
                           R->p);
  note_launches(1);
  // Condition estimate (Gershgorin: largest training-row sum of outputscale K~ over
  // noise), for the App. A preconditioner and for the BF16 value gate
  size_t pre_bytes = 0;
  const bool bf16 = L->value_dtype == SGP_VALUES_BF16;
  if (S->o.precond_rank > 0 || bf16) {
    int* rowmax_d = nullptr;
    SRV_CHECK(tmp.get((void**)&rowmax_d, sizeof(int)), "alloc row sum");
    SRV_CHECK(cudaMemsetAsync(rowmax_d, 0, sizeof(int), st), "clear row sum");
    k_rowsum_max<<<152, 256, 0, st>>>(KZ, in.n, kp, rowmax_d);
    note_launches(1);
    int rowmax_bits = 0;
    SRV_CHECK(cudaMemcpyAsync(&rowmax_bits, rowmax_d, sizeof(int), cudaMemcpyDeviceToHost, st),
              "read row sum");
    SRV_CHECK(cudaStreamSynchronize(st), "condition estimate");
    float rowmax = 0.f;
    std::memcpy(&rowmax, &rowmax_bits, sizeof(float));
    R->kappa = ((double)rowmax + (double)in.noise) / (double)in.noise;
  }
  if (bf16 && R->kappa > kBf16MaxKappa) {
    // the bf16 operator error (~2^-8 per product) amplified by this conditioning would
    // exceed the solver's tolerance: fp32 values on the same lattice, and the probe
    // product and right-hand sides again
    L->value_dtype = SGP_VALUES_F32;
    L->lat_elems = 0;      // reallocate the value buffers at the fp32 size,
    L->act_tmp_elems = 0;  // and a sparse lattice's pass buffer
    s = ensure_lattice_values(L, kp, st);
    if (s != SGP_OK) return s;
    enqueue_mvm(L, Vz, kp, SGP_BLUR_SYMMETRIC, L->outputscale, 0.f, KZ, st);
    k_rhs<<<g, 256, 0, st>>>(L->perm, yd, KZ, n_all, in.n, kp, S->S, R->xh, R->xl, R->rh,
                             R->rl, R->p);
    note_launches(1);
  }
  R->st.value_dtype = L->value_dtype;
  if (S->o.precond_rank > 0) {
    if (R->kappa >= S->o.precond_min_kappa) {
      const int l = (int)std::min<long long>(S->o.precond_rank, in.n);
      const int ld = (l + 3) / 4 * 4;
      R->l = l;
      R->ld = ld;
      unit_counts(S, R, R->vb);
      SRV_CHECK(get((void**)&R->Bh, (size_t)n_all * ld * sizeof(float)), "alloc Nystrom B");
      SRV_CHECK(get((void**)&R->Minv, (size_t)l * l * sizeof(double)), "alloc Nystrom Minv");
      const size_t nseg = (size_t)ceil_div(R->vb[U_BT], kBtSeg);
      SRV_CHECK(get((void**)&R->btpart, (size_t)R->vb[U_BT] * ld * kp * sizeof(float)),
                "alloc B^T r partials");
      SRV_CHECK(get((void**)&R->bt2, nseg * ld * kp * sizeof(float)), "alloc B^T r sums");
      SRV_CHECK(get((void**)&R->tvec, (size_t)ld * kp * sizeof(double)), "alloc B^T r");
      SRV_CHECK(get((void**)&R->u, (size_t)ld * kp * sizeof(float)), "alloc Minv B^T r");
      SRV_CHECK(get((void**)&R->dpart2, (size_t)R->vb[U_Z] * kp * sizeof(double)),
                "alloc <r, z> partials");
      pre_bytes = (size_t)n_all * ld * sizeof(float) + (size_t)l * l * sizeof(double) +
                  ((size_t)R->vb[U_BT] + nseg) * ld * kp * sizeof(float) +
                  (size_t)ld * kp * (sizeof(double) + sizeof(float)) +
                  (size_t)R->vb[U_Z] * kp * sizeof(double);
      void* scratch = nullptr;
      int* status_d = nullptr;
      SRV_CHECK(tmp.get(&scratch, nystrom_masked_scratch_bytes(l, n_all)),
                "alloc Nystrom scratch");
      SRV_CHECK(tmp.get((void**)&status_d, sizeof(int)), "alloc Nystrom status");
      s = nystrom_build_masked(L, in.n, l, ld, in.seed ^ kPrecondSeedXor, in.noise, kp, Vz, KZ,
                               R->Bh, R->Minv, scratch, status_d, st);
      if (s != SGP_OK) return s;
      int failed = 0;
      SRV_CHECK(cudaMemcpyAsync(&failed, status_d, sizeof(int), cudaMemcpyDeviceToHost, st),
                "read Nystrom status");
      SRV_CHECK(cudaStreamSynchronize(st), "Nystrom factor");
      if (failed) {  // a Cholesky pivot failed: plain CG (the buffers are released at the end)
        R->l = R->ld = 0;
        unit_counts(S, R, R->vb);
      }
    }
  }
  R->st.precond_rank = R->l;
  R->st.kappa_est = R->kappa;
  // initial residual norms and scalars through a one-request table
  std::memset(&t1, 0, sizeof(Table));
  t1.nslots = 1;
  t1.kp = kp;
  t1.flags = nullptr;
  t1.err = R->ints + kp + 2;
  t1.wait_limit = kSpinLimit;
  fill_slot(S, R, t1.s[0]);
  for (int u = 0; u < U_KINDS; ++u) t1.pre[u][1] = R->vb[u];
  SRV_CHECK(cudaMemcpyAsync(R->dtab1, &t1, sizeof(Table), cudaMemcpyHostToDevice, st),
            "copy table");
  kb_norm<<<kGrid, kST, 0, st>>>(R->dtab1);
  note_launches(1);
  if (R->l) {  // z_0 = P^-1 r_0 (the kernels run for a request whose state is set)
    static const int kOne = 1;
    SRV_CHECK(cudaMemcpyAsync(R->ints + kp, &kOne, sizeof(int), cudaMemcpyHostToDevice, st),
              "mark the request active");
    launch_bt(kp, R->dtab1, st);
    kb_bt_seg<<<kGrid, kST, 0, st>>>(R->dtab1);
    kb_bt_total<<<kGrid, kST, 0, st>>>(R->dtab1);
    kb_minv<<<kGrid, kST, 0, st>>>(R->dtab1);
    launch_apply_z(kp, R->dtab1, st);
    note_launches(5);
  }
  kb_init_scalars<<<1, kST, 0, st>>>(R->dtab1);
  note_launches(1);
  if (R->l)  // p_0 = z_0
    SRV_CHECK(cudaMemcpyAsync(R->p, R->ap, vec, cudaMemcpyDeviceToDevice, st), "p = z");
  SRV_CHECK(cudaGetLastError(), "request set-up");
  SRV_CHECK(cudaEventCreateWithFlags(&R->ready, cudaEventDisableTiming), "event");
  SRV_CHECK(cudaEventRecord(R->ready, st), "record");
  // a resident lattice's bytes are counted by the cache, not by the request
  R->held = (R->from_cache ? 0 : L->bytes) + 6 * vec + (size_t)R->vb[U_VEC] * kp * sizeof(double) +
            2 * (size_t)in.ns * sizeof(float) + sizeof(Table) + pre_bytes;
  return SGP_OK;
}

// Predictive slice, copy to the host, release.  Runs on the (idle) lane's stream.
sgp_status finish(sgp_server* S, Request* R, cudaStream_t st) {
  const sgp_request& in = R->in;
  Lattice* L = R->L;
  const int kp = S->kp;
  const int64_t n_all = L->n;
  const int64_t cnt = n_all * kp;
  k_x_sum<<<(unsigned)ceil_div(cnt, 256), 256, 0, st>>>(R->xh, R->xl, R->p, cnt);
  note_launches(1);
  enqueue_mvm(L, R->p, kp, SGP_BLUR_SYMMETRIC, L->outputscale, 0.f, R->ap, st, nullptr,
              /*internal=*/true);
  float* mean_d = R->outd;
  float* var_d = R->outd + in.ns;
  k_predict<<<(unsigned)ceil_div(n_all, 256), 256, 0, st>>>(L->perm, R->ap, n_all, in.n, kp,
                                                           S->S, in.seed, L->outputscale,
                                                           mean_d, var_d);
  note_launches(1);
  SRV_CHECK(cudaMemcpyAsync(in.mean, mean_d, (size_t)in.ns * sizeof(float),
                            cudaMemcpyDeviceToHost, st),
            "copy mean");
  if (in.var)
    SRV_CHECK(cudaMemcpyAsync(in.var, var_d, (size_t)in.ns * sizeof(float),
                              cudaMemcpyDeviceToHost, st),
              "copy var");
  std::vector<double> relres(kp);
  std::vector<int> ints(kp + 3);
  SRV_CHECK(cudaMemcpyAsync(relres.data(), R->scal + 2 * kp, kp * sizeof(double),
                            cudaMemcpyDeviceToHost, st),
            "copy residuals");
  SRV_CHECK(cudaMemcpyAsync(ints.data(), R->ints, (kp + 3) * sizeof(int), cudaMemcpyDeviceToHost,
                            st),
            "copy state");
  SRV_CHECK(cudaStreamSynchronize(st), "finishing a request");
  double worst = 0.0;
  for (int c = 0; c <= S->S; ++c) worst = std::max(worst, relres[c]);
  R->st.iters = ints[kp + 1];
  R->st.rel_res = worst;
  R->st.bytes = R->held;
  R->st.status = SGP_OK;
  if (ints[kp + 2]) {  // a bulk copy of its set-up never completed: the result is void
    set_error("sgp_server: a bulk-copy wait of the preconditioner gave up");
    R->st.status = SGP_ERR_CUDA;
  }
  R->st.done_us = now_us(S);
  R->st.done = 1;
  if (in.lattice_key && !R->from_cache) {  // keep the lattice resident for reuse
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->cache.find(in.lattice_key) == S->cache.end()) {
      sgp_server::Cached c;
      c.L = L;
      c.bytes = L->bytes;
      c.outputscale = in.outputscale;
      c.last_us = now_us(S);
      S->cache[in.lattice_key] = c;
      S->cache_bytes += c.bytes;
      // the lattice's bytes stay in in_use, now counted by the cache rather than the request
      R->held -= std::min<unsigned long long>(R->held, c.bytes);
      R->L = nullptr;
    }
  }
  release(S, R, st);
  return SGP_OK;
}

// Free the least recently used idle resident lattice; false when none is idle.
bool evict_one(sgp_server* S, unsigned long long keep_key) {
  Lattice* victim = nullptr;
  unsigned long long bytes = 0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto best = S->cache.end();
    for (auto it = S->cache.begin(); it != S->cache.end(); ++it)
      if (!it->second.busy && it->first != keep_key &&
          (best == S->cache.end() || it->second.last_us < best->second.last_us))
        best = it;
    if (best == S->cache.end()) return false;
    victim = best->second.L;
    bytes = best->second.bytes;
    S->cache.erase(best);
  }
  S->cache_bytes -= bytes;
  S->in_use -= bytes;
  sgp_set_stream(victim, S->bs);
  sgp_lattice_free(victim);
  return true;
}

template <int Rr, class Sv>
int enqueue_iteration_t(Lane* ln, int dmax, bool sparse, bool pre) {
  cudaStream_t st = ln->st;
  const Table* T = ln->dtab;
  kb_splat<Sv><<<kGrid, kST, 0, st>>>(T);
  kb_splat_med<Sv><<<kGrid, kST, 0, st>>>(T);
  kb_splat_huge<Sv><<<kGrid, kST, 0, st>>>(T);
  for (int t = 0; t < 2 * dmax; ++t) {
    kb_blur<Rr, Sv><<<kGrid, kST, 0, st>>>(T, t);
    if (sparse) kb_sparse_store<Sv><<<kGrid, kST, 0, st>>>(T, t);
  }
  if (sparse) kb_sparse_finish<Sv><<<kGrid, kST, 0, st>>>(T);
  kb_slice_dot<Sv><<<kGrid, kST, 0, st>>>(T);
  kb_alpha<<<kMaxSlots, kST, 0, st>>>(T);
  kb_update_xr<<<kGrid, kST, 0, st>>>(T);
  if (pre) {
    const int kp = ln->htab->kp;
    launch_bt(kp, T, st);
    kb_bt_seg<<<kGrid, kST, 0, st>>>(T);
    kb_bt_total<<<kGrid, kST, 0, st>>>(T);
    kb_minv<<<kGrid, kST, 0, st>>>(T);
    launch_apply_z(kp, T, st);
  }
  kb_check_beta<<<kMaxSlots, kST, 0, st>>>(T);
  kb_update_p<<<kGrid, kST, 0, st>>>(T);
  return 8 + 2 * dmax + (sparse ? 2 * dmax + 1 : 0) + (pre ? 5 : 0);
}

template <class Sv>
int enqueue_iteration_s(const sgp_server* S, Lane* ln, int dmax, bool sparse, bool pre) {
  switch (S->o.order_r) {
    case 1: return enqueue_iteration_t<1, Sv>(ln, dmax, sparse, pre);
    case 2: return enqueue_iteration_t<2, Sv>(ln, dmax, sparse, pre);
    case 3: return enqueue_iteration_t<3, Sv>(ln, dmax, sparse, pre);
    default: return enqueue_iteration_t<4, Sv>(ln, dmax, sparse, pre);
  }
}

int graph_key(int dmax, bool sparse, bool pre) {
  return 4 * dmax + (pre ? 2 : 0) + (sparse ? 1 : 0);
}

// Graph of one iteration of the lane, keyed by Dmax, whether a request blurs sparsely and
// whether one is preconditioned.
sgp_status graph_for(const sgp_server* S, Lane* ln, int dmax, bool sparse, bool pre,
                     cudaGraphExec_t* out) {
  const int key = graph_key(dmax, sparse, pre);
  auto it = ln->graphs.find(key);
  if (it != ln->graphs.end()) {
    *out = it->second;
    return SGP_OK;
  }
  SRV_CHECK(cudaStreamBeginCapture(ln->st, cudaStreamCaptureModeThreadLocal), "begin capture");
  const int kernels = ln->value_dtype == SGP_VALUES_BF16
                          ? enqueue_iteration_s<bf16>(S, ln, dmax, sparse, pre)
                          : enqueue_iteration_s<float>(S, ln, dmax, sparse, pre);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(ln->st, &g);
  if (e != cudaSuccess) return cuda_status(e, "capturing the batched CG iteration");
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_status(e, "instantiating the batched CG iteration");
  ln->graphs[key] = ex;
  ln->graph_kernels[key] = kernels;
  *out = ex;
  return SGP_OK;
}

sgp_status lane_for(sgp_server* S, int key, int value_dtype, Lane** out) {
  auto it = S->lanes.find(key);
  if (it != S->lanes.end()) {
    *out = it->second.get();
    return SGP_OK;
  }
  auto ln = std::make_unique<Lane>();
  ln->key = key;
  ln->value_dtype = value_dtype;
  ln->htab = std::make_unique<Table>();
  SRV_CHECK(cudaStreamCreateWithFlags(&ln->st, cudaStreamNonBlocking), "lane stream");
  SRV_CHECK(cudaMalloc((void**)&ln->dtab, sizeof(Table)), "alloc lane table");
  SRV_CHECK(cudaMalloc((void**)&ln->dflags, (2 * kMaxSlots + 1) * sizeof(int)), "alloc lane flags");
  // on the lane's own stream: a legacy-stream memset is not ordered with the lane's kernels
  // and could land after the first round has written its flags
  SRV_CHECK(cudaMemsetAsync(ln->dflags, 0, (2 * kMaxSlots + 1) * sizeof(int), ln->st),
            "clear lane flags");
  SRV_CHECK(cudaMallocHost((void**)&ln->hflags, (2 * kMaxSlots + 1) * sizeof(int)),
            "alloc lane flags");
  SRV_CHECK(cudaEventCreateWithFlags(&ln->ev, cudaEventDisableTiming), "lane event");
  *out = ln.get();
  S->lanes[key] = std::move(ln);
  return SGP_OK;
}

void destroy_lane(Lane* ln) {
  if (ln->st) cudaStreamSynchronize(ln->st);
  for (auto& kv : ln->graphs) cudaGraphExecDestroy(kv.second);
  if (ln->dtab) cudaFree(ln->dtab);
  if (ln->dflags) cudaFree(ln->dflags);
  if (ln->hflags) cudaFreeHost(ln->hflags);
  if (ln->ev) cudaEventDestroy(ln->ev);
  if (ln->st) cudaStreamDestroy(ln->st);
}

void setup_worker(sgp_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = S->bs;
  auto t1 = std::make_unique<Table>();  // host image of the one-request tables
  for (;;) {
    Request* R = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !S->to_setup.empty(); });
      if (S->stop) break;
      R = S->to_setup.front();
      S->to_setup.pop_front();
    }
    const double t = now_us(S);
    const sgp_status status = setup(S, R, st, *t1);
    R->st.setup_us = now_us(S) - t;
    // error messages are per host thread: carry this one to the stepping thread
    if (status != SGP_OK) R->setup_error = sgp_last_error();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->setup_done.emplace_back(R, status);
    }
  }
  if (st != S->bs) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
}

// Requests whose set-up has finished join their lane (or complete with the error).
sgp_status collect_setups(sgp_server* S, int* done) {
  std::vector<std::pair<Request*, sgp_status>> ready;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    ready.swap(S->setup_done);
  }
  for (auto& rs : ready) {
    Request* R = rs.first;
    sgp_status s = rs.second;
    S->in_use -= R->bound;  // the reservation made at admission
    Lane* ln = nullptr;
    if (s == SGP_OK) s = lane_for(S, lane_key(S, R), R->L->value_dtype, &ln);
    if (s != SGP_OK) {
      if (!R->setup_error.empty()) set_error("request set-up: " + R->setup_error);
      R->st.status = s;
      R->held = 0;
      release(S, R, S->bs);
      R->st.done_us = now_us(S);
      R->st.done = 1;
      S->n_active -= 1;
      ++*done;
      if (s == SGP_ERR_CUDA) return s;  // a failed device call: report it
      continue;
    }
    S->in_use += R->held;
    R->lane = ln;
    ln->active.push_back(R);
    ln->dirty = true;
  }
  return SGP_OK;
}

sgp_status admit(sgp_server* S) {
  for (auto it = S->queue.begin(); it != S->queue.end();) {  // deadlines passed in the queue
    Request* R = *it;
    if (!expired(S, R)) {
      ++it;
      continue;
    }
    R->st.status = SGP_ERR_TIMEOUT;
    R->st.done_us = now_us(S);
    R->st.done = 1;
    it = S->queue.erase(it);
  }
  while (!S->queue.empty() && S->n_active < S->o.max_active) {
    Request* R = S->queue.front();
    while (S->in_use + R->bound > S->o.hbm_budget && evict_one(S, R->in.lattice_key)) {
    }
    if (S->in_use + R->bound > S->o.hbm_budget) break;  // strict arrival order
    S->queue.pop_front();
    R->st.admit_us = now_us(S);
    S->in_use += R->bound;  // reserved until its set-up reports the actual allocation
    S->n_active += 1;
    S->peak_active = std::max(S->peak_active, S->n_active);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->to_setup.push_back(R);
    }
    S->cv.notify_one();
  }
  return SGP_OK;
}

bool setups_ready(sgp_server* S) {
  std::lock_guard<std::mutex> lk(S->mu);
  return !S->setup_done.empty();
}

// Requests of a lane whose round has finished: finish the stopped ones, keep the rest.
sgp_status harvest(sgp_server* S, Lane* ln, int* done) {
  std::vector<Request*> keep;
  const bool voided = ln->hflags[2 * kMaxSlots] != 0;  // a bulk-copy wait gave up
  if (voided) {
    set_error("sgp_server: a bulk-copy wait of the preconditioner gave up; the requests of "
              "that round completed with SGP_ERR_CUDA");
    ln->hflags[2 * kMaxSlots] = 0;
    SRV_CHECK(cudaMemsetAsync(ln->dflags + 2 * kMaxSlots, 0, sizeof(int), ln->st),
              "clear lane error");
  }
  for (int q = 0; q < (int)ln->active.size(); ++q) {
    Request* R = ln->active[q];
    if (voided && q < ln->ntab) {
      (void)cudaStreamSynchronize(ln->st);
      R->st.status = SGP_ERR_CUDA;
      R->st.iters = ln->hflags[2 * q + 1];
      R->st.bytes = R->held;
      R->st.done_us = now_us(S);
      R->st.done = 1;
      release(S, R, ln->st);
      S->n_active -= 1;
      ++*done;
    } else if (q < ln->ntab && ln->hflags[2 * q] == 0) {
      if (sgp_status s = finish(S, R, ln->st)) return s;
      S->n_active -= 1;
      ++*done;
    } else if (expired(S, R)) {  // still iterating past its deadline: cancel
      (void)cudaStreamSynchronize(ln->st);
      R->st.status = SGP_ERR_TIMEOUT;
      R->st.iters = q < ln->ntab ? ln->hflags[2 * q + 1] : 0;
      R->st.bytes = R->held;
      R->st.done_us = now_us(S);
      R->st.done = 1;
      release(S, R, ln->st);
      S->n_active -= 1;
      ++*done;
    } else {
      keep.push_back(R);
    }
  }
  if ((int)keep.size() != ln->ntab || keep.size() != ln->active.size()) ln->dirty = true;
  ln->active.swap(keep);
  ln->in_flight = false;
  return SGP_OK;
}

sgp_status launch(sgp_server* S, Lane* ln) {
  const int ns = (int)ln->active.size();
  Table& t = *ln->htab;
  bool any_pre = false;
  for (Request* R : ln->active) any_pre = any_pre || R->l > 0;
  const bool inject = any_pre && S->inject_ring_wait;
  if (inject) ln->dirty = true;
  if (ln->dirty) {
    std::memset(&t, 0, sizeof(Table));
    t.nslots = ns;
    t.kp = S->kp;
    t.flags = ln->dflags;
    t.err = ln->dflags + 2 * kMaxSlots;
    t.wait_limit = inject ? 0 : kSpinLimit;
    for (int q = 0; q < ns; ++q) {
      Request* R = ln->active[q];
      fill_slot(S, R, t.s[q]);
      for (int u = 0; u < U_KINDS; ++u) t.pre[u][q + 1] = t.pre[u][q] + R->vb[u];
      if (!R->waited) {
        SRV_CHECK(cudaStreamWaitEvent(ln->st, R->ready, 0), "wait for set-up");
        R->waited = true;
      }
    }
    SRV_CHECK(cudaMemcpyAsync(ln->dtab, &t, sizeof(Table), cudaMemcpyHostToDevice, ln->st),
              "copy table");
    ln->ntab = ns;
    ln->dirty = inject;  // after an injected round the table is uploaded again, limit restored
    S->inject_ring_wait = S->inject_ring_wait && !inject;
  }
  int dmax = 1;
  bool sparse = false, pre = false;
  for (Request* R : ln->active) {
    dmax = std::max(dmax, R->L->D);
    sparse = sparse || R->L->sparse;
    pre = pre || R->l > 0;
  }
  cudaGraphExec_t ex = nullptr;
  if (sgp_status s = graph_for(S, ln, dmax, sparse, pre, &ex)) return s;
  const int key = graph_key(dmax, sparse, pre);
  for (int i = 0; i < S->o.check_every; ++i) {
    SRV_CHECK(cudaGraphLaunch(ex, ln->st), "launching the batched CG iteration");
    note_launches(ln->graph_kernels[key]);
  }
  SRV_CHECK(cudaMemcpyAsync(ln->hflags, ln->dflags, 2 * ns * sizeof(int), cudaMemcpyDeviceToHost,
                            ln->st),
            "copy flags");
  SRV_CHECK(cudaMemcpyAsync(ln->hflags + 2 * kMaxSlots, ln->dflags + 2 * kMaxSlots, sizeof(int),
                            cudaMemcpyDeviceToHost, ln->st),
            "copy lane error");
  SRV_CHECK(cudaEventRecord(ln->ev, ln->st), "record flags");
  ln->in_flight = true;
  return SGP_OK;
}

sgp_status server_step(sgp_server* S, int* completed) {
  int done = 0;
  if (sgp_status s = collect_setups(S, &done)) return s;  // 0. requests ready to join
  for (auto& kv : S->lanes) {  // 1. lanes whose round has finished
    Lane* ln = kv.second.get();
    if (!ln->in_flight) continue;
    const cudaError_t q = cudaEventQuery(ln->ev);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return cuda_status(q, "waiting for a lane");
    if (sgp_status s = harvest(S, ln, &done)) return s;
  }
  if (sgp_status s = admit(S)) return s;  // 2. set-up (another thread) overlaps the lanes
  bool any = false;
  for (auto& kv : S->lanes) {  // 3. relaunch idle lanes
    Lane* ln = kv.second.get();
    if (!ln->in_flight && !ln->active.empty())
      if (sgp_status s = launch(S, ln)) return s;
    any = any || ln->in_flight;
  }
  // 4. without a finished request, wait a little for a lane or a set-up to finish
  const bool setting_up = S->n_active > 0;
  if (done == 0 && (any || setting_up)) {
    const double deadline = now_us(S) + kStepWaitUs;
    bool ready = false;
    while (!ready && now_us(S) < deadline) {
      for (auto& kv : S->lanes) {
        Lane* ln = kv.second.get();
        if (ln->in_flight && cudaEventQuery(ln->ev) != cudaErrorNotReady) ready = true;
      }
      ready = ready || setups_ready(S);
      if (!ready) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    clear_pending_error();  // cudaEventQuery's not-ready status
  }
  if (completed) *completed = done;
  return SGP_OK;
}

bool have_device() {
  int count = 0;
  return cudaGetDeviceCount(&count) == cudaSuccess && count > 0;
}

}  // namespace

extern "C" {

void sgp_server_opts_init(sgp_server_opts* o) {
  if (!o) return;
  size_t freeb = 0, total = 0;
  if (have_device() && cudaMemGetInfo(&freeb, &total) == cudaSuccess) o->hbm_budget = total / 2;
  else o->hbm_budget = 0;
  clear_pending_error();
  o->max_active = 16;
  o->probes = 8;
  o->order_r = 1;
  o->kernel = SGP_KERNEL_RBF_BINOMIAL;
  o->spacing_s = 0.0;
  o->value_dtype = SGP_VALUES_F32;
  o->tol = 1e-3;
  o->max_iter = 1000;
  o->check_every = 8;
  o->precond_rank = 100;
  o->precond_min_kappa = 1e3;
  o->lane_classes = 1;
}

unsigned long long sgp_request_bytes_bound(long long n_points, int d, int order_r, int k,
                                           int value_dtype, int precond_rank) {
  if (n_points < 1 || d < 1 || order_r < 1 || k < 1 || precond_rank < 0 ||
      precond_rank > kMaxRank)
    return 0;
  const unsigned long long n = (unsigned long long)n_points, D = (unsigned long long)d + 1;
  const unsigned long long nD = n * D, m = nD, r = (unsigned long long)order_r;
  const unsigned long long kp = ((unsigned long long)k + 3) / 4 * 4;
  const unsigned long long vbytes = value_dtype == SGP_VALUES_BF16 ? 2 : 4;
  unsigned long long cap = 1024;
  while (cap < 2 * nD) cap <<= 1;
  const unsigned long long nseg = nD / kSplatSeg + m;  // segments and fix-up rows
  // lattice arrays kept by the handle
  const unsigned long long lattice = 4 * n + 2 * m * D + 8 * nD + 8 * D * r * m + 8 * nD +
                                     4 * (m + 1) + 16 * (nseg + 2 * m) + 256;
  // build work space (all counted at once)
  const unsigned long long build = 7 * nD + 8 * cap + 4 * nD + 4 * nD +
                                   4 * scan_temp_elems((int64_t)nD) + 4 * cap + 16 * nD +
                                   4 * radix_temp_elems((int64_t)nD) + 16 * n +
                                   4 * radix_temp_elems((int64_t)n) + 4 * n * d;
  // values, splat partials, permuted input; CG vectors and partials; probe products
  const unsigned long long values = 2 * m * kp * vbytes + nseg * kp * 4 + n * kp * 4;
  const unsigned long long solve = 6 * n * kp * 4 + (n / 4 + 1) * kp * 8 + 2 * n * kp * 4 +
                                   n * 4 + sizeof(Table) + 4096;
  // preconditioner: B, Minv, apply partials, and the factorisation's scratch
  unsigned long long pre = 0;
  if (precond_rank > 0) {
    const unsigned long long l = (unsigned long long)precond_rank, ld = (l + 3) / 4 * 4;
    const unsigned long long nbt = n / kBtVbRows + 1;
    pre = n * ld * 4 + l * l * 8 + (nbt + nbt / kBtSeg + 1) * ld * kp * 4 + ld * kp * 12 +
          (n / 4 + 1) * kp * 8 + nystrom_masked_scratch_bytes((int)l, (int64_t)n) + 1024;
  }
  return lattice + build + values + solve + pre;
}

sgp_status sgp_server_create(const sgp_server_opts* opts, sgp_server** out) {
  if (!out) {
    set_error("sgp_server_create: out is null");
    return SGP_ERR_INVALID_ARG;
  }
  *out = nullptr;
  sgp_server_opts o;
  sgp_server_opts_init(&o);
  if (opts) o = *opts;
  if (o.max_active < 1 || o.max_active > kMaxSlots || o.probes < 0 ||
      o.probes + 2 > kMaxServeK || o.order_r < 1 || o.order_r > kMaxOrder || o.max_iter < 0 ||
      !(o.tol >= 0.0) || o.check_every < 1 ||
      (o.value_dtype != SGP_VALUES_F32 && o.value_dtype != SGP_VALUES_BF16) ||
      o.precond_rank < 0 || o.precond_rank > kMaxRank || !(o.precond_min_kappa >= 0.0) ||
      (o.lane_classes != 0 && o.lane_classes != 1)) {
    set_error("sgp_server_create: need 1 <= max_active <= 64, 0 <= probes <= 30, "
              "1 <= order_r <= 4, max_iter >= 0, tol >= 0, check_every >= 1, "
              "0 <= precond_rank <= 128, precond_min_kappa >= 0, lane_classes 0 or 1");
    return SGP_ERR_INVALID_ARG;
  }
  double sp, c[kMaxOrder + 1], g[kMaxOrder + 1];
  if (!make_stencil(o.kernel, o.order_r, o.spacing_s, &sp, c, g)) {
    set_error("sgp_server_create: unknown kernel");
    return SGP_ERR_INVALID_ARG;
  }
  if (!have_device()) {
    set_error("sgp_server_create: no CUDA device (this library has no CPU path)");
    return SGP_ERR_CUDA;
  }
  clear_pending_error();
  auto S = std::make_unique<sgp_server>();
  S->o = o;
  S->S = o.probes;
  S->kp = (o.probes + 2 + 3) / 4 * 4;  // y, S probes, the ones column, padding
  S->t0 = std::chrono::steady_clock::now();
  {
    const char* f = std::getenv("SGP_FAULT");
    S->inject_ring_wait = f && std::strcmp(f, "ring_wait") == 0;
  }
  SRV_CHECK(cudaGetDevice(&S->device), "cudaGetDevice");
  // the attribute is per kernel, shared by every server: allow the largest kp
  SRV_CHECK(bt_smem_attributes(kMaxServeK), "shared memory of the preconditioner kernels");
  SRV_CHECK(apply_z_smem_attributes(kMaxServeK), "shared memory of the preconditioner kernels");
  SRV_CHECK(cudaStreamCreateWithFlags(&S->bs, cudaStreamNonBlocking), "stream");
  sgp_server* raw = S.get();
  const int nthreads = std::min(kSetupThreads, o.max_active);
  for (int i = 0; i < nthreads; ++i) S->workers.emplace_back(setup_worker, raw);
  *out = S.release();
  return SGP_OK;
}

sgp_status sgp_server_submit(sgp_server* S, const sgp_request* req, long long* id) {
  if (!S || !req || !id) {
    set_error("sgp_server_submit: null argument");
    return SGP_ERR_INVALID_ARG;
  }
  const sgp_request& r = *req;
  if (!r.X || !r.y || !r.Xs || !r.lengthscales || !r.mean || (S->S > 0 && !r.var) || r.n < 1 ||
      r.ns < 1 || r.d < 1 || r.d + 1 > kMaxD || !(r.outputscale > 0.f) || !(r.noise > 0.f) ||
      (r.n + r.ns) * (long long)(r.d + 1) > 0x7fffffffLL) {
    set_error("sgp_server_submit: need X, y, Xs, lengthscales, mean (and var when probes > 0), "
              "n >= 1, ns >= 1, 1 <= d <= 127, outputscale > 0, noise > 0 and "
              "(n + ns)(d + 1) < 2^31");
    return SGP_ERR_INVALID_ARG;
  }
  // a BF16 server may switch a request to fp32 values after its condition estimate:
  // reserve the fp32 bound
  const unsigned long long bound =
      sgp_request_bytes_bound(r.n + r.ns, r.d, S->o.order_r, S->kp, SGP_VALUES_F32,
                              S->o.precond_rank);
  if (bound > S->o.hbm_budget) {
    set_error("sgp_server_submit: the request's memory bound exceeds the server's budget");
    return SGP_ERR_INVALID_ARG;
  }
  auto R = std::make_unique<Request>();
  R->id = S->next_id++;
  R->in = r;
  R->bound = bound;
  R->st.arrival_us = r.arrival_us >= 0.0 ? r.arrival_us : now_us(S);
  R->st.status = SGP_OK;
  *id = R->id;
  S->queue.push_back(R.get());
  S->reqs[R->id] = std::move(R);
  return SGP_OK;
}

sgp_status sgp_server_step(sgp_server* S, int* completed) {
  if (completed) *completed = 0;
  if (!S) {
    set_error("sgp_server_step: null server");
    return SGP_ERR_INVALID_ARG;
  }
  clear_pending_error();
  NvtxRange nvtx("sgp_serve_step");
  return server_step(S, completed);
}

sgp_status sgp_server_stats(const sgp_server* S, long long id, sgp_request_stats* out) {
  if (!S || !out) {
    set_error("sgp_server_stats: null argument");
    return SGP_ERR_INVALID_ARG;
  }
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) {
    set_error("sgp_server_stats: unknown request id");
    return SGP_ERR_INVALID_ARG;
  }
  *out = it->second->st;
  return SGP_OK;
}

sgp_status sgp_server_info(const sgp_server* S, int* queued, int* active,
                           unsigned long long* bytes_in_use, int* peak_active) {
  if (!S) {
    set_error("sgp_server_info: null server");
    return SGP_ERR_INVALID_ARG;
  }
  if (queued) *queued = (int)S->queue.size();
  if (active) *active = S->n_active;
  if (bytes_in_use) *bytes_in_use = S->in_use;
  if (peak_active) *peak_active = S->peak_active;
  return SGP_OK;
}

sgp_status sgp_server_cache_info(const sgp_server* S, int* lattices, unsigned long long* bytes) {
  if (!S) {
    set_error("sgp_server_cache_info: null server");
    return SGP_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(const_cast<sgp_server*>(S)->mu);
  if (lattices) *lattices = (int)S->cache.size();
  if (bytes) *bytes = S->cache_bytes;
  return SGP_OK;
}

double sgp_server_clock_us(const sgp_server* S) { return S ? now_us(S) : 0.0; }

void sgp_server_destroy(sgp_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (std::thread& w : S->workers)
    if (w.joinable()) w.join();
  cudaStreamSynchronize(S->bs);
  for (auto& rs : S->setup_done) {  // set up but never joined a lane
    S->in_use -= rs.first->bound;
    release(S, rs.first, S->bs);
  }
  S->setup_done.clear();
  S->to_setup.clear();
  for (auto& kv : S->lanes) {
    Lane* ln = kv.second.get();
    cudaStreamSynchronize(ln->st);
    for (Request* R : ln->active) release(S, R, ln->st);
    ln->active.clear();
  }
  S->queue.clear();
  for (auto& kv : S->lanes) destroy_lane(kv.second.get());
  for (auto& kv : S->cache) {
    sgp_set_stream(kv.second.L, S->bs);
    sgp_lattice_free(kv.second.L);
  }
  S->cache.clear();
  cudaStreamSynchronize(S->bs);
  cudaStreamDestroy(S->bs);
  delete S;
  clear_pending_error();
}

}  // extern "C"
