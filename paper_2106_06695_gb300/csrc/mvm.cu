// The lattice MVM  out = alpha * W B W^T V + beta * V  (Sec. 3.2, Eq. ski_to_bf).
//
//   k_splat  W^T: each lattice vertex gathers w * V[point] over its list of incident
//            (point, weight) pairs, cut into segments of at most kSplatSeg items; long
//            lists are finished by an ordered fix-up.  Gathers only: deterministic.
//   k_blur   one lattice direction u_j: out[v] = c_0 in[v] + sum_t c_t (in[v - t u_j] +
//            in[v + t u_j]) with absent neighbours contributing 0 (Sec. 3.2 "Blur"); the
//            neighbour ids come from the table built with the lattice.
//   k_slice  W: each point interpolates its d+1 vertices with its barycentric weights,
//            fused with the alpha/beta epilogue.
//
// All of them are bound by memory traffic.  The caller's vectors are fp32 [rows][k]
// row-major.  Lattice values are stored as S = float or __nv_bfloat16 (SGP_VALUES_BF16:
// half the bytes of the dominant blur traffic); every sum is accumulated in fp32.  A
// thread owns 4 consecutive columns of a row when k is a multiple of 4 and the buffers are
// aligned, else one column; the blur gives each thread 8 columns when k allows.
#include <atomic>

#include <cuda_bf16.h>

#include "sgp_internal.cuh"
#include "values.cuh"

namespace sgp {
namespace {

constexpr int kThreads = 256;

// ---- splat ---------------------------------------------------------------------------
// Incidences and vertex rows are gathered kChunk at a time: a thread first loads the
// (point, weight) pairs or (vertex id, weight) pairs of a chunk, then issues all of the
// chunk's row loads, then accumulates in order.  The row loads of a chunk are independent,
// so kChunk of them are in flight per thread instead of one dependent pair at a time; the
// sums keep the incidence order, so results do not change with the chunking.
constexpr int kChunk = 8;

// One thread-group of G threads per segment of at most kSplatSeg incidences.
template <int VEC, class S>
__global__ void __launch_bounds__(kThreads) k_splat(int64_t nseg, int G, int k,
                                                    const int4* __restrict__ seg,
                                                    const int2* __restrict__ items,
                                                    const float* __restrict__ V,
                                                    S* __restrict__ lat,
                                                    float* __restrict__ partial) {
  using Vt = Vec<VEC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = gid / G;
  if (s >= nseg) return;
  const int col = (int)(gid - s * G) * VEC;
  const int4 sg = __ldg(seg + s);
  typename Vt::T acc = Vt::zero();
  for (int p0 = sg.y; p0 < sg.z; p0 += kChunk) {
    int2 it[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j)
      it[j] = p0 + j < sg.z ? __ldg(items + p0 + j) : make_int2(-1, 0);
    typename Vt::T row[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j)
      row[j] = it[j].x >= 0 ? Vt::ldg(V + (int64_t)it[j].x * k + col) : Vt::zero();
#pragma unroll
    for (int j = 0; j < kChunk; ++j)
      if (it[j].x >= 0) acc = Vt::fma(__int_as_float(it[j].y), row[j], acc);
  }
  if (sg.w < 0) Vt::sts(lat + (int64_t)sg.x * k + col, acc);
  else Vt::st(partial + (int64_t)sg.w * k + col, acc);
}

// Fix-up for vertices with 2..kSplatMedSegs segments: one thread-group sums in order.
template <int VEC, class S>
__global__ void __launch_bounds__(kThreads) k_splat_med(int64_t nrows, int G, int k,
                                                        const int4* __restrict__ rows,
                                                        const float* __restrict__ partial,
                                                        S* __restrict__ lat) {
  using Vt = Vec<VEC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t q = gid / G;
  if (q >= nrows) return;
  const int col = (int)(gid - q * G) * VEC;
  const int4 rw = rows[q];
  typename Vt::T acc = Vt::zero();
  for (int j = 0; j < rw.z; ++j) acc = Vt::add(acc, Vt::ld(partial + (int64_t)(rw.y + j) * k + col));
  Vt::sts(lat + (int64_t)rw.x * k + col, acc);
}

// Fix-up for vertices with more segments: one block per vertex, groups of G threads take
// strided partials, then a fixed-shape shared-memory tree combines the groups.
template <int VEC, class S>
__global__ void __launch_bounds__(kThreads) k_splat_huge(int G, int k, const int4* __restrict__ rows,
                                                         const float* __restrict__ partial,
                                                         S* __restrict__ lat) {
  using Vt = Vec<VEC>;
  __shared__ typename Vt::T red[kThreads];
  const int groups = blockDim.x / G;
  const int g = threadIdx.x / G;
  const int col = (int)(threadIdx.x % G) * VEC;
  const int4 rw = rows[blockIdx.x];
  typename Vt::T acc = Vt::zero();
  if (g < groups)
    for (int j = g; j < rw.z; j += groups)
      acc = Vt::add(acc, Vt::ld(partial + (int64_t)(rw.y + j) * k + col));
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int half = groups / 2; half >= 1; half /= 2) {
    if (g < half) red[threadIdx.x] = Vt::add(red[threadIdx.x], red[threadIdx.x + half * G]);
    __syncthreads();
  }
  if (g == 0) Vt::sts(lat + (int64_t)rw.x * k + col, red[threadIdx.x]);
}

// ---- blur ----------------------------------------------------------------------------
// One value per thread (any k).
template <class S>
__global__ void __launch_bounds__(kThreads) k_blur(int64_t m, int k, int r, Taps tp,
                                                   const int32_t* __restrict__ nbr,
                                                   const S* __restrict__ in, S* __restrict__ out) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t v = gid / k;
  if (v >= m) return;
  const int col = (int)(gid - v * k);
  float acc = tp.t[0] * Store<S>::ld1(in + v * k + col);
  for (int t = 1; t <= r; ++t) {
    const int a = nbr[(int64_t)(2 * (t - 1)) * m + v];
    const int c = nbr[(int64_t)(2 * (t - 1) + 1) * m + v];
    float s = 0.f;
    if (a >= 0) s += Store<S>::ld1(in + (int64_t)a * k + col);
    if (c >= 0) s += Store<S>::ld1(in + (int64_t)c * k + col);
    acc = fmaf(tp.t[t], s, acc);
  }
  Store<S>::st1(out + v * k + col, acc);
}

// Rows of k = 4 CH G values.  Each thread owns 4 CH consecutive columns of U rows (R =
// stencil order): it issues all id loads, then all own and neighbour row loads, then the
// arithmetic, so 3 U row loads per order are in flight at once.  A block covers U
// consecutive runs of kThreads / G rows (coalesced per run, local per block).
template <int CH, int U, int R, class S>
__global__ void __launch_bounds__(kThreads) k_blur_rows(int64_t m, int G, int k, Taps tp,
                                                        const int32_t* __restrict__ nbr,
                                                        const S* __restrict__ in,
                                                        S* __restrict__ out) {
  static_assert(CH == 1 || CH == 2, "one or two groups of four columns per thread");
  const int rows_per_run = blockDim.x / G;
  const int col = (int)(threadIdx.x % G) * (4 * CH);
  int64_t v[U];
  int ia[U][R], ic[U][R];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    v[u] = ((int64_t)blockIdx.x * U + u) * rows_per_run + threadIdx.x / G;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      ia[u][t] = v[u] < m ? __ldg(nbr + (int64_t)(2 * t) * m + v[u]) : -1;
      ic[u][t] = v[u] < m ? __ldg(nbr + (int64_t)(2 * t + 1) * m + v[u]) : -1;
    }
  }
  auto load = [&](int64_t row, float4* x) {
    if (CH == 2) Store<S>::ldg8(in + row * k + col, x[0], x[CH - 1]);
    else x[0] = Store<S>::ldg4(in + row * k + col);
  };
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 own[U][CH], sa[U][R][CH], sc[U][R][CH];
#pragma unroll
  for (int u = 0; u < U; ++u) {
#pragma unroll
    for (int c = 0; c < CH; ++c) own[u][c] = zero;
    if (v[u] < m) load(v[u], own[u]);
#pragma unroll
    for (int t = 0; t < R; ++t) {
#pragma unroll
      for (int c = 0; c < CH; ++c) sa[u][t][c] = sc[u][t][c] = zero;
      if (ia[u][t] >= 0) load(ia[u][t], sa[u][t]);
      if (ic[u][t] >= 0) load(ic[u][t], sc[u][t]);
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (v[u] >= m) continue;
    float4 acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      acc[c] = make_float4(tp.t[0] * own[u][c].x, tp.t[0] * own[u][c].y, tp.t[0] * own[u][c].z,
                           tp.t[0] * own[u][c].w);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const float w = tp.t[t + 1];
        acc[c].x = fmaf(w, sa[u][t][c].x + sc[u][t][c].x, acc[c].x);
        acc[c].y = fmaf(w, sa[u][t][c].y + sc[u][t][c].y, acc[c].y);
        acc[c].z = fmaf(w, sa[u][t][c].z + sc[u][t][c].z, acc[c].z);
        acc[c].w = fmaf(w, sa[u][t][c].w + sc[u][t][c].w, acc[c].w);
      }
    }
    if (CH == 2) Store<S>::st8(out + v[u] * k + col, acc[0], acc[CH - 1]);
    else Store<S>::st4(out + v[u] * k + col, acc[0]);
  }
}

// Stencil order 1 with eight columns per thread, persistent and software-pipelined: each
// thread group walks rows v, v + stride, ...; while it combines row v, the rows of v +
// stride (own and both neighbours) and the neighbour ids of v + 2 stride are in flight, so
// the memory system sees a steady stream instead of one burst per block.  Same arithmetic
// as k_blur_rows (bitwise equal results).
template <class S>
__global__ void __launch_bounds__(kThreads) k_blur_pipe(int64_t m, int G, int k, Taps tp,
                                                        const int32_t* __restrict__ nbr,
                                                        const S* __restrict__ in,
                                                        S* __restrict__ out) {
  const int rows_per_block = blockDim.x / G;
  const int col = (int)(threadIdx.x % G) * 8;
  const int64_t stride = (int64_t)gridDim.x * rows_per_block;
  int64_t row = (int64_t)blockIdx.x * rows_per_block + threadIdx.x / G;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  auto ids = [&](int64_t v, int& a, int& c) {  // neighbour ids of v - u_j, v + u_j
    if (v < m) {
      a = __ldg(nbr + v);
      c = __ldg(nbr + m + v);
    } else {
      a = c = -1;
    }
  };
  auto load = [&](int64_t v, int a, int c, float4 (&x)[3][2]) {  // own, minus, plus rows
    x[0][0] = x[0][1] = x[1][0] = x[1][1] = x[2][0] = x[2][1] = zero;
    if (v < m) Store<S>::ldg8(in + v * k + col, x[0][0], x[0][1]);
    if (a >= 0) Store<S>::ldg8(in + (int64_t)a * k + col, x[1][0], x[1][1]);
    if (c >= 0) Store<S>::ldg8(in + (int64_t)c * k + col, x[2][0], x[2][1]);
  };
  int a0, c0, a1, c1;
  ids(row, a0, c0);
  ids(row + stride, a1, c1);
  float4 cur[3][2];
  load(row, a0, c0, cur);
  while (row < m) {
    const int64_t nrow = row + stride;
    int a2, c2;
    ids(nrow + stride, a2, c2);
    float4 nxt[3][2];
    load(nrow, a1, c1, nxt);
    float4 acc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      acc[h] = make_float4(tp.t[0] * cur[0][h].x, tp.t[0] * cur[0][h].y, tp.t[0] * cur[0][h].z,
                           tp.t[0] * cur[0][h].w);
      acc[h].x = fmaf(tp.t[1], cur[1][h].x + cur[2][h].x, acc[h].x);
      acc[h].y = fmaf(tp.t[1], cur[1][h].y + cur[2][h].y, acc[h].y);
      acc[h].z = fmaf(tp.t[1], cur[1][h].z + cur[2][h].z, acc[h].z);
      acc[h].w = fmaf(tp.t[1], cur[1][h].w + cur[2][h].w, acc[h].w);
    }
    Store<S>::st8(out + row * k + col, acc[0], acc[1]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      cur[q][0] = nxt[q][0];
      cur[q][1] = nxt[q][1];
    }
    a1 = a2;
    c1 = c2;
    row = nrow;
  }
}

// Blocks of k_blur_pipe<S> the device keeps resident (one wave), cached per device.
template <class S>
int blur_pipe_blocks() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int b = cache[dev].load();
  if (b > 0) return b;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_blur_pipe<S>, kThreads, 0) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    clear_pending_error();
    return 152;
  }
  b = std::max(1, per_sm) * std::max(1, sms);
  cache[dev].store(b);
  return b;
}

// ---- sparse blur (lattices whose direction lists are short) ------------------------------
// Stored rows carry a lazy factor: the value of vertex x before pass t is
// g0^(t - epoch[x]) stored[x] (g0 = the pass's centre tap), since a vertex without a
// neighbour along a pass's direction is only scaled by the centre tap.  Pass t (direction
// j) computes the new rows of the vertices on list j into tmp; a second kernel stores them
// and sets their epoch to t + 1.  After the last pass, k_sparse_finish applies the
// remaining factors.
template <int VEC, class S>
__global__ void __launch_bounds__(kThreads) k_sparse_blur(int64_t count, int G, int k, int r,
                                                          Taps tp, int t,
                                                          const int32_t* __restrict__ act,
                                                          const int32_t* __restrict__ nbr_j,
                                                          int64_t m,
                                                          const int32_t* __restrict__ epoch,
                                                          const float* __restrict__ pw,
                                                          const S* __restrict__ stored,
                                                          S* __restrict__ tmp) {
  using Vt = Vec<VEC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t a = gid / G;
  if (a >= count) return;
  const int col = (int)(gid - a * G) * VEC;
  const int64_t v = act[a];
  auto value = [&](int64_t x) {
    const float f = pw ? pw[t - epoch[x]] : 1.f;
    return Vt::scale(f, Vt::lds(stored + x * k + col));
  };
  typename Vt::T acc = Vt::scale(tp.t[0], value(v));
  for (int q = 1; q <= r; ++q) {
    const int ua = nbr_j[(int64_t)(2 * (q - 1)) * m + v];
    const int uc = nbr_j[(int64_t)(2 * (q - 1) + 1) * m + v];
    typename Vt::T sum = Vt::zero();
    if (ua >= 0) sum = value(ua);
    if (uc >= 0) sum = Vt::add(sum, value(uc));
    acc = Vt::fma(tp.t[q], sum, acc);
  }
  Vt::sts(tmp + a * k + col, acc);
}

template <int VEC, class S>
__global__ void __launch_bounds__(kThreads) k_sparse_store(int64_t count, int G, int k, int t,
                                                           const int32_t* __restrict__ act,
                                                           const S* __restrict__ tmp,
                                                           S* __restrict__ stored,
                                                           int32_t* __restrict__ epoch) {
  using Vt = Vec<VEC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t a = gid / G;
  if (a >= count) return;
  const int col = (int)(gid - a * G) * VEC;
  const int64_t v = act[a];
  Vt::sts(stored + v * k + col, Vt::lds(tmp + a * k + col));
  if (col == 0) epoch[v] = t + 1;
}

template <int VEC, class S>
__global__ void __launch_bounds__(kThreads) k_sparse_finish(int64_t m, int G, int k, int P,
                                                            const int32_t* __restrict__ epoch,
                                                            const float* __restrict__ pw,
                                                            S* __restrict__ stored) {
  using Vt = Vec<VEC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t v = gid / G;
  if (v >= m) return;
  const int e = epoch[v];
  if (e == P) return;
  const int col = (int)(gid - v * G) * VEC;
  Vt::sts(stored + v * k + col, Vt::scale(pw[P - e], Vt::lds(stored + v * k + col)));
}

// ---- slice ---------------------------------------------------------------------------
// sum_c w[p][c] lat[idx[p][c]] for the VEC columns at col, in vertex order c = 0..D-1,
// loading the ids and weights of kChunk vertices before their rows.
template <int VEC, class S>
__device__ __forceinline__ typename Vec<VEC>::T slice_row(int64_t p, int D, int k, int col,
                                                          const int32_t* __restrict__ idx,
                                                          const float* __restrict__ w,
                                                          const S* __restrict__ lat) {
  using Vt = Vec<VEC>;
  typename Vt::T acc = Vt::zero();
  const int64_t e0 = p * D;
  for (int c0 = 0; c0 < D; c0 += kChunk) {
    int id[kChunk];
    float wt[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      const bool in = c0 + j < D;
      id[j] = in ? __ldg(idx + e0 + c0 + j) : -1;
      wt[j] = in ? __ldg(w + e0 + c0 + j) : 0.f;
    }
    typename Vt::T row[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j)
      row[j] = id[j] >= 0 ? Vt::ldgs(lat + (int64_t)id[j] * k + col) : Vt::zero();
#pragma unroll
    for (int j = 0; j < kChunk; ++j)
      if (id[j] >= 0) acc = Vt::fma(wt[j], row[j], acc);
  }
  return acc;
}

// PERM: V and out rows are in the caller's order (row perm[p]); else in locality order.
template <int VEC, bool BETA, bool PERM, class S>
__global__ void __launch_bounds__(kThreads) k_slice(int64_t n, int G, int k, int D,
                                                    const int32_t* __restrict__ perm,
                                                    const int32_t* __restrict__ idx,
                                                    const float* __restrict__ w,
                                                    const S* __restrict__ lat,
                                                    const float* __restrict__ V, float alpha,
                                                    float beta, float* __restrict__ out) {
  using Vt = Vec<VEC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p = gid / G;
  if (p >= n) return;
  const int col = (int)(gid - p * G) * VEC;
  const typename Vt::T acc = slice_row<VEC, S>(p, D, k, col, idx, w, lat);
  const int64_t i = PERM ? (int64_t)perm[p] : p;
  typename Vt::T res = Vt::scale(alpha, acc);
  if (BETA) res = Vt::fma(beta, Vt::ld(V + i * k + col), res);
  Vt::st(out + i * k + col, res);
}

// The CG's slice: V and out in locality order, out = alpha W lat + beta V, and the
// per-block column sums of V * out for <p, A p> (exact products and double-float
// accumulation per thread, fp64 across threads).  Grid-stride over points.
template <int VEC, class S>
__global__ void __launch_bounds__(kThreads) k_slice_dot(int64_t n, int G, int k, int D,
                                                        const int32_t* __restrict__ idx,
                                                        const float* __restrict__ w,
                                                        const S* __restrict__ lat,
                                                        const float* __restrict__ V, float alpha,
                                                        float beta, float* __restrict__ out,
                                                        double* __restrict__ dot_partial) {
  using Vt = Vec<VEC>;
  const int rows = blockDim.x / G;
  const int col = (int)(threadIdx.x % G) * VEC;
  dfloat d[VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) d[j] = {0.f, 0.f};
  for (int64_t p = (int64_t)blockIdx.x * rows + threadIdx.x / G; p < n;
       p += (int64_t)gridDim.x * rows) {
    const typename Vt::T acc = slice_row<VEC, S>(p, D, k, col, idx, w, lat);
    const typename Vt::T v = Vt::ld(V + p * k + col);
    const typename Vt::T res = Vt::fma(beta, v, Vt::scale(alpha, acc));
    Vt::st(out + p * k + col, res);
    const float* vv = reinterpret_cast<const float*>(&v);
    const float* rr = reinterpret_cast<const float*>(&res);
#pragma unroll
    for (int j = 0; j < VEC; ++j) d[j] = df_add(d[j], df_two_prod(vv[j], rr[j]));
  }
  double dd[VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) dd[j] = df_to_double(d[j]);
  block_column_sums<VEC>(dd, k, dot_partial + (int64_t)blockIdx.x * k);
}

// Vp[p] = V[perm[p]]: the caller's rows in locality order.
template <int VEC>
__global__ void __launch_bounds__(kThreads) k_permute_rows(int64_t n, int G, int k,
                                                           const int32_t* __restrict__ perm,
                                                           const float* __restrict__ V,
                                                           float* __restrict__ Vp) {
  using Vt = Vec<VEC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p = gid / G;
  if (p >= n) return;
  const int col = (int)(gid - p * G) * VEC;
  Vt::st(Vp + p * k + col, Vt::ld(V + (int64_t)perm[p] * k + col));
}

inline bool vec4_ok(int k, const void* a, const void* b) {
  return (k % 4 == 0) && ((uintptr_t)a % 16 == 0) && ((uintptr_t)b % 16 == 0);
}

// ---- launchers -----------------------------------------------------------------------
template <class S>
void launch_splat_t(const Lattice* L, const float* V, int k, S* lat, float* partial,
                    cudaStream_t st) {
  const bool v4 = vec4_ok(k, V, lat);
  const int G = v4 ? k / 4 : k;
  if (v4)
    k_splat<4, S><<<(unsigned)ceil_div(L->nseg * G, kThreads), kThreads, 0, st>>>(
        L->nseg, G, k, L->seg, L->items, V, lat, partial);
  else
    k_splat<1, S><<<(unsigned)ceil_div(L->nseg * G, kThreads), kThreads, 0, st>>>(
        L->nseg, G, k, L->seg, L->items, V, lat, partial);
  note_launches(1);
  if (L->nmed > 0) {
    if (v4)
      k_splat_med<4, S><<<(unsigned)ceil_div(L->nmed * G, kThreads), kThreads, 0, st>>>(
          L->nmed, G, k, L->med_rows, partial, lat);
    else
      k_splat_med<1, S><<<(unsigned)ceil_div(L->nmed * G, kThreads), kThreads, 0, st>>>(
          L->nmed, G, k, L->med_rows, partial, lat);
    note_launches(1);
  }
  if (L->nhuge > 0) {
    int groups = 1;  // a power-of-two number of G-thread groups per block for the tree
    while (groups * 2 * G <= kThreads) groups *= 2;
    if (v4)
      k_splat_huge<4, S><<<(unsigned)L->nhuge, groups * G, 0, st>>>(G, k, L->huge_rows, partial, lat);
    else
      k_splat_huge<1, S><<<(unsigned)L->nhuge, groups * G, 0, st>>>(G, k, L->huge_rows, partial, lat);
    note_launches(1);
  }
}

template <int CH, int U, class S>
void launch_blur_rows(const Lattice* L, const int32_t* nbr, const Taps& taps, const S* in,
                      S* out, int k, cudaStream_t st) {
  const int G = k / (4 * CH);
  const int threads = G * (kThreads / G);  // a whole number of rows per run
  const int64_t runs = ceil_div(L->m, threads / G);
  const unsigned grid = (unsigned)ceil_div(runs, U);
  switch (L->r) {
    case 1: k_blur_rows<CH, U, 1, S><<<grid, threads, 0, st>>>(L->m, G, k, taps, nbr, in, out); break;
    case 2: k_blur_rows<CH, U, 2, S><<<grid, threads, 0, st>>>(L->m, G, k, taps, nbr, in, out); break;
    case 3: k_blur_rows<CH, U, 3, S><<<grid, threads, 0, st>>>(L->m, G, k, taps, nbr, in, out); break;
    default: k_blur_rows<CH, U, 4, S><<<grid, threads, 0, st>>>(L->m, G, k, taps, nbr, in, out); break;
  }
}

template <class S>
void launch_blur_t(const Lattice* L, int j, const Taps& taps, const S* in, S* out, int k,
                   cudaStream_t st) {
  const int32_t* nbr = L->nbr + (size_t)j * L->r * 2 * L->m;
  if (k % 8 == 0 && k / 8 <= kThreads && L->r == 1) {  // eight columns, pipelined rows
    const int G = k / 8, threads = G * (kThreads / G);
    const int64_t blocks = std::min<int64_t>(blur_pipe_blocks<S>(), ceil_div(L->m, threads / G));
    k_blur_pipe<S><<<(unsigned)blocks, threads, 0, st>>>(L->m, G, k, taps, nbr, in, out);
  } else if (k % 8 == 0 && k / 8 <= kThreads) {  // eight columns of two rows per thread
    launch_blur_rows<2, 2, S>(L, nbr, taps, in, out, k, st);
  } else if (k % 4 == 0 && k / 4 <= kThreads) {
    launch_blur_rows<1, 2, S>(L, nbr, taps, in, out, k, st);
  } else {
    k_blur<S><<<(unsigned)ceil_div(L->m * k, kThreads), kThreads, 0, st>>>(L->m, k, L->r, taps, nbr,
                                                                          in, out);
  }
  note_launches(1);
}

template <bool PERM, class S>
void launch_slice_t(const Lattice* L, const S* lat, const float* V, int k, float alpha,
                    float beta, float* out, cudaStream_t st) {
  const bool v4 = vec4_ok(k, out, V ? (const void*)V : (const void*)out);
  const int G = v4 ? k / 4 : k;
  const unsigned grid = (unsigned)ceil_div(L->n * G, kThreads);
  const bool use_beta = beta != 0.f && V != nullptr;
  if (v4) {
    if (use_beta)
      k_slice<4, true, PERM, S><<<grid, kThreads, 0, st>>>(L->n, G, k, L->D, L->perm, L->idx, L->w,
                                                           lat, V, alpha, beta, out);
    else
      k_slice<4, false, PERM, S><<<grid, kThreads, 0, st>>>(L->n, G, k, L->D, L->perm, L->idx,
                                                            L->w, lat, V, alpha, beta, out);
  } else {
    if (use_beta)
      k_slice<1, true, PERM, S><<<grid, kThreads, 0, st>>>(L->n, G, k, L->D, L->perm, L->idx, L->w,
                                                           lat, V, alpha, beta, out);
    else
      k_slice<1, false, PERM, S><<<grid, kThreads, 0, st>>>(L->n, G, k, L->D, L->perm, L->idx,
                                                            L->w, lat, V, alpha, beta, out);
  }
  note_launches(1);
}

template <class S>
void launch_slice_dot(const Lattice* L, const S* lat, const float* V, int k, float alpha,
                      float beta, float* out, double* dot_partial, cudaStream_t st) {
  const int vec = k % 4 == 0 ? 4 : 1;
  const int T = column_block_threads(k, vec);
  const unsigned grid = (unsigned)slice_dot_blocks(L, k);
  if (vec == 4)
    k_slice_dot<4, S><<<grid, T, 0, st>>>(L->n, k / 4, k, L->D, L->idx, L->w, lat, V, alpha, beta,
                                          out, dot_partial);
  else
    k_slice_dot<1, S><<<grid, T, 0, st>>>(L->n, k, k, L->D, L->idx, L->w, lat, V, alpha, beta, out,
                                          dot_partial);
  note_launches(1);
}

void launch_permute(const Lattice* L, const float* V, int k, float* Vp, cudaStream_t st) {
  if (vec4_ok(k, V, Vp)) {
    const int G = k / 4;
    k_permute_rows<4><<<(unsigned)ceil_div(L->n * G, kThreads), kThreads, 0, st>>>(
        L->n, G, k, L->perm, V, Vp);
  } else {
    k_permute_rows<1><<<(unsigned)ceil_div(L->n * k, kThreads), kThreads, 0, st>>>(
        L->n, k, k, L->perm, V, Vp);
  }
  note_launches(1);
}

// The blur passes of `blur` on the splatted values in lat0 (lat1: ping-pong buffer);
// returns the buffer that holds the result.  Sparse lattices use the direction lists
// (lat1 unused) unless `dense` is set.
template <class S>
S* blur_passes_t(const Lattice* L, int blur, S* lat0, S* lat1, int k, cudaStream_t st,
                 int* passes_out, bool dense) {
  Taps c{}, g{};
  for (int t = 0; t <= L->r; ++t) {
    c.t[t] = (float)L->coef[t];
    g.t[t] = (float)L->half[t];
  }
  const int D = L->D;
  const int P = blur == SGP_BLUR_SYMMETRIC ? 2 * D : D;
  auto dir = [&](int t) {
    if (blur == SGP_BLUR_SEQUENTIAL) return t;
    if (blur == SGP_BLUR_TRANSPOSE) return D - 1 - t;
    return t < D ? t : 2 * D - 1 - t;
  };
  const Taps& tp = blur == SGP_BLUR_SYMMETRIC ? g : c;
  if (passes_out) *passes_out = P;
  if (!L->sparse || dense) {
    S* a = lat0;
    S* b = lat1;
    for (int t = 0; t < P; ++t) {
      launch_blur_t<S>(L, dir(t), tp, a, b, k, st);
      S* x = a;
      a = b;
      b = x;
    }
    return a;
  }
  // sparse: lazy centre-tap factors (none when the centre tap is 1)
  const float* pw = tp.t[0] == 1.f ? nullptr : L->g0pow;
  const bool v4 = k % 4 == 0;
  const int G = v4 ? k / 4 : k;
  if (pw) cudaMemsetAsync(L->epoch, 0, (size_t)L->m * sizeof(int32_t), st);
  S* tmp = static_cast<S*>(L->act_tmp);
  for (int t = 0; t < P; ++t) {
    const int j = dir(t);
    const int64_t count = L->act_off[j + 1] - L->act_off[j];
    if (count == 0) continue;
    const int32_t* act = L->act + L->act_off[j];
    const int32_t* nbr_j = L->nbr + (size_t)j * L->r * 2 * L->m;
    const unsigned grid = (unsigned)ceil_div(count * G, kThreads);
    if (v4) {
      k_sparse_blur<4, S><<<grid, kThreads, 0, st>>>(count, G, k, L->r, tp, t, act, nbr_j, L->m,
                                                     L->epoch, pw, lat0, tmp);
      k_sparse_store<4, S><<<grid, kThreads, 0, st>>>(count, G, k, t, act, tmp, lat0, L->epoch);
    } else {
      k_sparse_blur<1, S><<<grid, kThreads, 0, st>>>(count, G, k, L->r, tp, t, act, nbr_j, L->m,
                                                     L->epoch, pw, lat0, tmp);
      k_sparse_store<1, S><<<grid, kThreads, 0, st>>>(count, G, k, t, act, tmp, lat0, L->epoch);
    }
    note_launches(2);
  }
  if (pw) {
    const unsigned grid = (unsigned)ceil_div(L->m * G, kThreads);
    if (v4) k_sparse_finish<4, S><<<grid, kThreads, 0, st>>>(L->m, G, k, P, L->epoch, pw, lat0);
    else k_sparse_finish<1, S><<<grid, kThreads, 0, st>>>(L->m, G, k, P, L->epoch, pw, lat0);
    note_launches(1);
  }
  return lat0;
}

// The whole operator with explicit buffers.  internal: V and out in locality order;
// else V and out are in the caller's order and V is first gathered into `vperm`.
template <class S>
int enqueue_t(const Lattice* L, const float* V, int k, int blur, float alpha, float beta,
              float* out, S* lat0, S* lat1, float* partial, float* vperm, cudaStream_t st,
              cudaEvent_t* ev, bool internal, double* dot_partial = nullptr,
              bool dense = false) {
  const float* src = V;
  if (!internal) {
    launch_permute(L, V, k, vperm, st);
    src = vperm;
  }
  if (ev) cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal);
  launch_splat_t<S>(L, src, k, lat0, partial, st);
  // External: inside a stream capture this becomes an event-record node of the graph
  if (ev) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
  int passes = 0;
  S* a = blur_passes_t<S>(L, blur, lat0, lat1, k, st, &passes, dense);
  if (ev) cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
  if (internal && dot_partial) launch_slice_dot<S>(L, a, V, k, alpha, beta, out, dot_partial, st);
  else if (internal) launch_slice_t<false, S>(L, a, V, k, alpha, beta, out, st);
  else launch_slice_t<true, S>(L, a, V, k, alpha, beta, out, st);
  if (ev) cudaEventRecordWithFlags(ev[3], st, cudaEventRecordExternal);
  return passes;
}

// Splat (locality-ordered input) and blur only; returns the buffer holding the result.
template <class S>
S* splat_blur_t(const Lattice* L, const float* Vp, int k, int blur, S* lat0, S* lat1,
                float* partial, cudaStream_t st) {
  launch_splat_t<S>(L, Vp, k, lat0, partial, st);
  return blur_passes_t<S>(L, blur, lat0, lat1, k, st, nullptr, false);
}

size_t value_size(const Lattice* L) {
  return L->value_dtype == SGP_VALUES_BF16 ? sizeof(bf16) : sizeof(float);
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

size_t mvm_work_bytes(const Lattice* L, int k) {
  return 2 * round256((size_t)L->m * k * value_size(L)) +
         round256((size_t)L->nslots * k * sizeof(float)) + round256((size_t)L->n * k * sizeof(float));
}

sgp_status ensure_lattice_values(Lattice* L, int k, cudaStream_t st) {
  if (L->sparse && L->act_tmp_elems < (size_t)L->act_max * k) {
    if (L->act_tmp) cudaFreeAsync(L->act_tmp, st);
    L->act_tmp = nullptr;
    const size_t bytes = std::max<size_t>((size_t)L->act_max * k * value_size(L), 16);
    cudaError_t e = dev_malloc(&L->act_tmp, bytes, st);
    if (e != cudaSuccess) return cuda_status(e, "allocating the sparse blur buffer");
    L->act_tmp_elems = (size_t)L->act_max * k;
  }
  if (L->lat_elems >= (size_t)L->m * k && L->lat[0] && L->vperm_elems >= (size_t)L->n * k)
    return SGP_OK;
  void** bufs[4] = {(void**)&L->lat[0], (void**)&L->lat[1], (void**)&L->partial,
                    (void**)&L->vperm};
  for (void** b : bufs) {
    if (*b) cudaFreeAsync(*b, st);
    *b = nullptr;
  }
  L->bytes -= L->lat_bytes;
  L->lat_bytes = 0;
  L->lat_elems = 0;
  L->vperm_elems = 0;
  const size_t vbytes = (size_t)L->m * k * value_size(L);
  const size_t sizes[4] = {vbytes, vbytes, (size_t)L->nslots * k * sizeof(float),
                           (size_t)L->n * k * sizeof(float)};
  for (int b = 0; b < 4; ++b) {
    cudaError_t e = dev_malloc(bufs[b], std::max<size_t>(sizes[b], 16), st);
    if (e != cudaSuccess) return cuda_status(e, "allocating lattice values");
  }
  L->lat_elems = (size_t)L->m * k;
  L->vperm_elems = (size_t)L->n * k;
  L->lat_bytes = sizes[0] + sizes[1] + sizes[2] + sizes[3];
  L->bytes += L->lat_bytes;
  return SGP_OK;
}

int enqueue_mvm(const Lattice* L, const float* V, int k, int blur, float alpha, float beta,
                float* out, cudaStream_t st, cudaEvent_t* ev, bool internal, double* dot_partial) {
  if (L->value_dtype == SGP_VALUES_BF16)
    return enqueue_t<bf16>(L, V, k, blur, alpha, beta, out, (bf16*)L->lat[0], (bf16*)L->lat[1],
                           L->partial, L->vperm, st, ev, internal, dot_partial);
  return enqueue_t<float>(L, V, k, blur, alpha, beta, out, (float*)L->lat[0], (float*)L->lat[1],
                          L->partial, L->vperm, st, ev, internal, dot_partial);
}

void enqueue_mvm_bf16_values(const Lattice* L, const float* V, int k, int blur, float alpha,
                             float* out, cudaStream_t st) {
  enqueue_t<bf16>(L, V, k, blur, alpha, 0.f, out, (bf16*)L->lat[0], (bf16*)L->lat[1], L->partial,
                  L->vperm, st, nullptr, /*internal=*/true);
}

int64_t slice_dot_blocks(const Lattice* L, int k) {
  const int vec = k % 4 == 0 ? 4 : 1;
  const int G = k / vec;
  const int T = column_block_threads(k, vec);
  // one wave: as many blocks as the device keeps resident (a grid-stride kernel whose
  // grid exceeds that runs a second, mostly idle wave)
  int per_sm = 0, sms = 0, dev = 0;
  const void* fn = vec == 4 ? (L->value_dtype == SGP_VALUES_BF16
                                   ? (const void*)k_slice_dot<4, bf16>
                                   : (const void*)k_slice_dot<4, float>)
                            : (L->value_dtype == SGP_VALUES_BF16
                                   ? (const void*)k_slice_dot<1, bf16>
                                   : (const void*)k_slice_dot<1, float>);
  int64_t resident = kVecBlocks;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, T, 0) == cudaSuccess &&
      per_sm > 0)
    resident = (int64_t)per_sm * sms;
  else
    (void)cudaGetLastError();
  return std::min<int64_t>(resident, std::max<int64_t>(1, ceil_div(L->n, T / G)));
}

void enqueue_mvm_into(const Lattice* L, const float* V_user, int k, int blur, float alpha,
                      float beta, float* out, void* work, cudaStream_t st) {
  char* w = static_cast<char*>(work);
  const size_t vb = round256((size_t)L->m * k * value_size(L));
  void* lat0 = w;
  void* lat1 = w + vb;
  float* partial = reinterpret_cast<float*>(w + 2 * vb);
  float* vperm = reinterpret_cast<float*>(w + 2 * vb + round256((size_t)L->nslots * k * sizeof(float)));
  // the fixed work area holds no direction-list buffers: dense passes
  if (L->value_dtype == SGP_VALUES_BF16)
    enqueue_t<bf16>(L, V_user, k, blur, alpha, beta, out, (bf16*)lat0, (bf16*)lat1, partial, vperm,
                    st, nullptr, false, nullptr, /*dense=*/true);
  else
    enqueue_t<float>(L, V_user, k, blur, alpha, beta, out, (float*)lat0, (float*)lat1, partial,
                     vperm, st, nullptr, false, nullptr, /*dense=*/true);
}

void* enqueue_splat_blur(const Lattice* L, const float* Vp, int k, int blur, void* lat0,
                         void* lat1, float* partial, cudaStream_t st) {
  if (L->value_dtype == SGP_VALUES_BF16)
    return splat_blur_t<bf16>(L, Vp, k, blur, (bf16*)lat0, (bf16*)lat1, partial, st);
  return splat_blur_t<float>(L, Vp, k, blur, (float*)lat0, (float*)lat1, partial, st);
}

void enqueue_permute(const Lattice* L, const float* V, int k, float* Vp, cudaStream_t st) {
  launch_permute(L, V, k, Vp, st);
}

void enqueue_slice_caller(const Lattice* L, const void* lat, int k, float alpha, float* out,
                          cudaStream_t st) {
  if (L->value_dtype == SGP_VALUES_BF16)
    launch_slice_t<true, bf16>(L, (const bf16*)lat, nullptr, k, alpha, 0.f, out, st);
  else
    launch_slice_t<true, float>(L, (const float*)lat, nullptr, k, alpha, 0.f, out, st);
}

size_t lattice_value_bytes(const Lattice* L, int k) { return (size_t)L->m * k * value_size(L); }

sgp_status run_mvm(Lattice* L, const float* V, int k, int blur, float alpha, float beta,
                   float* out) {
  sgp_status s = ensure_lattice_values(L, k, L->stream);
  if (s != SGP_OK) return s;
  enqueue_mvm(L, V, k, blur, alpha, beta, out, L->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "launching the lattice MVM");
  return SGP_OK;
}

}  // namespace sgp
