// The lattice MVM  out = alpha * W B W^T V + beta * V  (Sec. 3.2, Eq. ski_to_bf).
//
//   k_splat  W^T: each lattice vertex gathers w * V[point] over its list of incident
//            (point, weight) pairs.  A gather, so the result is deterministic.
//   k_blur   one lattice direction u_j: out[v] = c_0 in[v] + sum_t c_t (in[v - t u_j] +
//            in[v + t u_j]) with absent neighbours contributing 0 (Sec. 3.2 "Blur"); the
//            neighbour ids come from the table built with the lattice.
//   k_slice  W: each point interpolates its d+1 vertices with its barycentric weights,
//            fused with the alpha/beta epilogue.
//
// All three are bound by memory traffic.  Values are fp32 [rows][k] row-major; a thread
// owns 4 consecutive columns of one row (16-byte vector loads) when k is a multiple of 4
// and the caller's buffers are 16-byte aligned, else one column.
#include "sgp_internal.cuh"

namespace sgp {
namespace {

constexpr int kThreads = 256;

template <int VEC>
struct Vec;
template <>
struct Vec<4> {
  using T = float4;
  static __device__ __forceinline__ T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ T ld(const float* p) { return *reinterpret_cast<const float4*>(p); }
  static __device__ __forceinline__ void st(float* p, T v) { *reinterpret_cast<float4*>(p) = v; }
  static __device__ __forceinline__ T fma(float a, T x, T y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
  }
  static __device__ __forceinline__ T add(T x, T y) {
    return make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
  }
  static __device__ __forceinline__ T scale(float a, T x) {
    return make_float4(a * x.x, a * x.y, a * x.z, a * x.w);
  }
};
template <>
struct Vec<1> {
  using T = float;
  static __device__ __forceinline__ T zero() { return 0.f; }
  static __device__ __forceinline__ T ld(const float* p) { return *p; }
  static __device__ __forceinline__ void st(float* p, T v) { *p = v; }
  static __device__ __forceinline__ T fma(float a, T x, T y) { return fmaf(a, x, y); }
  static __device__ __forceinline__ T add(T x, T y) { return x + y; }
  static __device__ __forceinline__ T scale(float a, T x) { return a * x; }
};

// One thread-group of G threads per segment of at most kSplatSeg incidences.
template <int VEC>
__global__ void __launch_bounds__(kThreads) k_splat(int64_t nseg, int G, int k,
                                                    const int4* __restrict__ seg,
                                                    const int2* __restrict__ items,
                                                    const float* __restrict__ V,
                                                    float* __restrict__ lat,
                                                    float* __restrict__ partial) {
  using Vt = Vec<VEC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = gid / G;
  if (s >= nseg) return;
  const int col = (int)(gid - s * G) * VEC;
  const int4 sg = seg[s];
  typename Vt::T acc = Vt::zero();
  for (int p = sg.y; p < sg.z; ++p) {
    const int2 it = items[p];
    acc = Vt::fma(__int_as_float(it.y), Vt::ld(V + (int64_t)it.x * k + col), acc);
  }
  if (sg.w < 0) Vt::st(lat + (int64_t)sg.x * k + col, acc);
  else Vt::st(partial + (int64_t)sg.w * k + col, acc);
}

// Fix-up for vertices with 2..kSplatMedSegs segments: one thread-group sums in order.
template <int VEC>
__global__ void __launch_bounds__(kThreads) k_splat_med(int64_t nrows, int G, int k,
                                                        const int4* __restrict__ rows,
                                                        const float* __restrict__ partial,
                                                        float* __restrict__ lat) {
  using Vt = Vec<VEC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t q = gid / G;
  if (q >= nrows) return;
  const int col = (int)(gid - q * G) * VEC;
  const int4 rw = rows[q];
  typename Vt::T acc = Vt::zero();
  for (int j = 0; j < rw.z; ++j) acc = Vt::add(acc, Vt::ld(partial + (int64_t)(rw.y + j) * k + col));
  Vt::st(lat + (int64_t)rw.x * k + col, acc);
}

// Fix-up for vertices with more segments: one block per vertex, groups of G threads take
// strided partials, then a fixed-shape shared-memory tree combines the groups.
template <int VEC>
__global__ void __launch_bounds__(kThreads) k_splat_huge(int G, int k, const int4* __restrict__ rows,
                                                         const float* __restrict__ partial,
                                                         float* __restrict__ lat) {
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
  if (g == 0) Vt::st(lat + (int64_t)rw.x * k + col, red[threadIdx.x]);
}

template <int VEC>
__global__ void __launch_bounds__(kThreads) k_blur(int64_t m, int G, int k, int r, Taps tp,
                                                   const int32_t* __restrict__ nbr,
                                                   const float* __restrict__ in,
                                                   float* __restrict__ out) {
  using Vt = Vec<VEC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t v = gid / G;
  if (v >= m) return;
  const int col = (int)(gid - v * G) * VEC;
  typename Vt::T acc = Vt::scale(tp.t[0], Vt::ld(in + v * k + col));
  for (int t = 1; t <= r; ++t) {
    const int a = nbr[(int64_t)(2 * (t - 1)) * m + v];
    const int c = nbr[(int64_t)(2 * (t - 1) + 1) * m + v];
    typename Vt::T s = Vt::zero();
    if (a >= 0) s = Vt::add(s, Vt::ld(in + (int64_t)a * k + col));
    if (c >= 0) s = Vt::add(s, Vt::ld(in + (int64_t)c * k + col));
    acc = Vt::fma(tp.t[t], s, acc);
  }
  Vt::st(out + v * k + col, acc);
}

// Rows of k = 4 CH G floats: each thread owns CH consecutive float4 chunks of one row, so
// it has 3 CH independent row loads in flight per stencil order after its two id loads.
template <int CH>
__global__ void __launch_bounds__(kThreads) k_blur_rows(int64_t m, int G, int k, int r,
                                                        Taps tp,
                                                        const int32_t* __restrict__ nbr,
                                                        const float* __restrict__ in,
                                                        float* __restrict__ out) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t v = gid / G;
  if (v >= m) return;
  const int col = (int)(gid - v * G) * (4 * CH);
  int ia[kMaxOrder], ic[kMaxOrder];
#pragma unroll
  for (int t = 0; t < kMaxOrder; ++t) {
    if (t < r) {
      ia[t] = __ldg(nbr + (int64_t)(2 * t) * m + v);
      ic[t] = __ldg(nbr + (int64_t)(2 * t + 1) * m + v);
    }
  }
  float4 acc[CH];
  const float4* own = reinterpret_cast<const float4*>(in + v * k + col);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const float4 x = __ldg(own + c);
    acc[c] = make_float4(tp.t[0] * x.x, tp.t[0] * x.y, tp.t[0] * x.z, tp.t[0] * x.w);
  }
#pragma unroll
  for (int t = 0; t < kMaxOrder; ++t) {
    if (t >= r) break;
    float4 sa[CH], sc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) sa[c] = sc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ia[t] >= 0) {
      const float4* pa = reinterpret_cast<const float4*>(in + (int64_t)ia[t] * k + col);
#pragma unroll
      for (int c = 0; c < CH; ++c) sa[c] = __ldg(pa + c);
    }
    if (ic[t] >= 0) {
      const float4* pc = reinterpret_cast<const float4*>(in + (int64_t)ic[t] * k + col);
#pragma unroll
      for (int c = 0; c < CH; ++c) sc[c] = __ldg(pc + c);
    }
    const float w = tp.t[t + 1];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      acc[c].x = fmaf(w, sa[c].x + sc[c].x, acc[c].x);
      acc[c].y = fmaf(w, sa[c].y + sc[c].y, acc[c].y);
      acc[c].z = fmaf(w, sa[c].z + sc[c].z, acc[c].z);
      acc[c].w = fmaf(w, sa[c].w + sc[c].w, acc[c].w);
    }
  }
  float4* dst = reinterpret_cast<float4*>(out + v * k + col);
#pragma unroll
  for (int c = 0; c < CH; ++c) dst[c] = acc[c];
}

// PERM: V and out rows are in the caller's order (row perm[p]); else in locality order.
template <int VEC, bool BETA, bool PERM>
__global__ void __launch_bounds__(kThreads) k_slice(int64_t n, int G, int k, int D,
                                                    const int32_t* __restrict__ perm,
                                                    const int32_t* __restrict__ idx,
                                                    const float* __restrict__ w,
                                                    const float* __restrict__ lat,
                                                    const float* __restrict__ V, float alpha,
                                                    float beta, float* __restrict__ out) {
  using Vt = Vec<VEC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p = gid / G;
  if (p >= n) return;
  const int col = (int)(gid - p * G) * VEC;
  typename Vt::T acc = Vt::zero();
  for (int c = 0; c < D; ++c) {
    const int64_t e = p * D + c;
    acc = Vt::fma(w[e], Vt::ld(lat + (int64_t)idx[e] * k + col), acc);
  }
  const int64_t i = PERM ? (int64_t)perm[p] : p;
  typename Vt::T res = Vt::scale(alpha, acc);
  if (BETA) res = Vt::fma(beta, Vt::ld(V + i * k + col), res);
  Vt::st(out + i * k + col, res);
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

}  // namespace

sgp_status ensure_lattice_values(Lattice* L, int k, cudaStream_t st) {
  const size_t need = (size_t)L->m * k;
  if (L->lat_elems >= need && L->lat[0] && L->vperm_elems >= (size_t)L->n * k) return SGP_OK;
  float** bufs[4] = {&L->lat[0], &L->lat[1], &L->partial, &L->vperm};
  for (float** b : bufs) {
    if (*b) cudaFreeAsync(*b, st);
    *b = nullptr;
  }
  L->bytes -= L->lat_bytes;
  L->lat_bytes = 0;
  L->lat_elems = 0;
  L->vperm_elems = 0;
  const size_t sizes[4] = {need, need, (size_t)L->nslots * k, (size_t)L->n * k};
  for (int b = 0; b < 4; ++b) {
    cudaError_t e = cudaMallocAsync((void**)bufs[b], std::max<size_t>(sizes[b], 1) * sizeof(float), st);
    if (e != cudaSuccess) return cuda_status(e, "allocating lattice values");
  }
  L->lat_elems = need;
  L->vperm_elems = sizes[3];
  L->lat_bytes = (sizes[0] + sizes[1] + sizes[2] + sizes[3]) * sizeof(float);
  L->bytes += L->lat_bytes;
  return SGP_OK;
}

void launch_splat(const Lattice* L, const float* V, int k, float* lat, cudaStream_t st) {
  const bool v4 = vec4_ok(k, V, lat);
  const int G = v4 ? k / 4 : k;
  if (v4)
    k_splat<4><<<(unsigned)ceil_div(L->nseg * G, kThreads), kThreads, 0, st>>>(
        L->nseg, G, k, L->seg, L->items, V, lat, L->partial);
  else
    k_splat<1><<<(unsigned)ceil_div(L->nseg * G, kThreads), kThreads, 0, st>>>(
        L->nseg, G, k, L->seg, L->items, V, lat, L->partial);
  note_launches(1);
  if (L->nmed > 0) {
    if (v4)
      k_splat_med<4><<<(unsigned)ceil_div(L->nmed * G, kThreads), kThreads, 0, st>>>(
          L->nmed, G, k, L->med_rows, L->partial, lat);
    else
      k_splat_med<1><<<(unsigned)ceil_div(L->nmed * G, kThreads), kThreads, 0, st>>>(
          L->nmed, G, k, L->med_rows, L->partial, lat);
    note_launches(1);
  }
  if (L->nhuge > 0) {
    // a power-of-two number of G-thread groups per block for the tree
    int groups = 1;
    while (groups * 2 * G <= kThreads) groups *= 2;
    if (v4)
      k_splat_huge<4><<<(unsigned)L->nhuge, groups * G, 0, st>>>(G, k, L->huge_rows, L->partial, lat);
    else
      k_splat_huge<1><<<(unsigned)L->nhuge, groups * G, 0, st>>>(G, k, L->huge_rows, L->partial, lat);
    note_launches(1);
  }
}

void launch_blur_pass(const Lattice* L, int j, const Taps& taps, const float* in, float* out,
                      int k, cudaStream_t st) {
  const int32_t* nbr = L->nbr + (size_t)j * L->r * 2 * L->m;
  if (k % 8 == 0) {  // two float4 chunks (one 32-byte sector) per thread
    const int G = k / 8;
    k_blur_rows<2><<<(unsigned)ceil_div(L->m * G, kThreads), kThreads, 0, st>>>(
        L->m, G, k, L->r, taps, nbr, in, out);
  } else if (k % 4 == 0) {
    const int G = k / 4;
    k_blur_rows<1><<<(unsigned)ceil_div(L->m * G, kThreads), kThreads, 0, st>>>(
        L->m, G, k, L->r, taps, nbr, in, out);
  } else {
    k_blur<1><<<(unsigned)ceil_div(L->m * k, kThreads), kThreads, 0, st>>>(L->m, k, k, L->r, taps,
                                                                          nbr, in, out);
  }
  note_launches(1);
}

template <bool PERM>
void launch_slice_t(const Lattice* L, const float* lat, const float* V, int k, float alpha,
                    float beta, float* out, cudaStream_t st) {
  const bool v4 = vec4_ok(k, out, V ? (const void*)V : (const void*)out);
  const int G = v4 ? k / 4 : k;
  const unsigned grid = (unsigned)ceil_div(L->n * G, kThreads);
  const bool use_beta = beta != 0.f && V != nullptr;
  if (v4) {
    if (use_beta)
      k_slice<4, true, PERM><<<grid, kThreads, 0, st>>>(L->n, G, k, L->D, L->perm, L->idx, L->w,
                                                        lat, V, alpha, beta, out);
    else
      k_slice<4, false, PERM><<<grid, kThreads, 0, st>>>(L->n, G, k, L->D, L->perm, L->idx, L->w,
                                                         lat, V, alpha, beta, out);
  } else {
    if (use_beta)
      k_slice<1, true, PERM><<<grid, kThreads, 0, st>>>(L->n, G, k, L->D, L->perm, L->idx, L->w,
                                                        lat, V, alpha, beta, out);
    else
      k_slice<1, false, PERM><<<grid, kThreads, 0, st>>>(L->n, G, k, L->D, L->perm, L->idx, L->w,
                                                         lat, V, alpha, beta, out);
  }
  note_launches(1);
}

void launch_slice(const Lattice* L, const float* lat, const float* V, int k, float alpha,
                  float beta, float* out, cudaStream_t st) {
  launch_slice_t<true>(L, lat, V, k, alpha, beta, out, st);
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

// Enqueue the whole operator on `st`.  Lattice value buffers must already hold m*k.
int enqueue_mvm(const Lattice* L, const float* V, int k, int blur, float alpha, float beta,
                float* out, cudaStream_t st, cudaEvent_t* ev, bool internal) {
  Taps c{}, g{};
  for (int t = 0; t <= L->r; ++t) {
    c.t[t] = (float)L->coef[t];
    g.t[t] = (float)L->half[t];
  }
  float* a = L->lat[0];
  float* b = L->lat[1];
  const float* src = V;
  if (!internal) {
    launch_permute(L, V, k, L->vperm, st);
    src = L->vperm;
  }
  launch_splat(L, src, k, a, st);
  // External: inside a stream capture this becomes an event-record node of the graph
  if (ev) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
  const int D = L->D;
  int passes = 0;
  auto pass = [&](int j, const Taps& tp) {
    launch_blur_pass(L, j, tp, a, b, k, st);
    float* t = a;
    a = b;
    b = t;
    ++passes;
  };
  if (blur == SGP_BLUR_SEQUENTIAL) {
    for (int j = 0; j < D; ++j) pass(j, c);
  } else if (blur == SGP_BLUR_TRANSPOSE) {
    for (int j = D - 1; j >= 0; --j) pass(j, c);
  } else {
    for (int j = 0; j < D; ++j) pass(j, g);
    for (int j = D - 1; j >= 0; --j) pass(j, g);
  }
  if (ev) cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
  if (internal) launch_slice_t<false>(L, a, V, k, alpha, beta, out, st);
  else launch_slice_t<true>(L, a, V, k, alpha, beta, out, st);
  return passes;
}

// Same operator as enqueue_mvm, with the two value buffers and the splat partials given
// by the caller (used by the allocation-free entry point).
void enqueue_mvm_into(const Lattice* L, const float* V_user, int k, int blur, float alpha,
                      float beta, float* out, float* lat0, float* lat1, float* partial,
                      float* vperm, cudaStream_t st) {
  launch_permute(L, V_user, k, vperm, st);
  const float* V = vperm;
  const bool v4 = vec4_ok(k, V, lat0);
  const int G = v4 ? k / 4 : k;
  if (v4)
    k_splat<4><<<(unsigned)ceil_div(L->nseg * G, kThreads), kThreads, 0, st>>>(
        L->nseg, G, k, L->seg, L->items, V, lat0, partial);
  else
    k_splat<1><<<(unsigned)ceil_div(L->nseg * G, kThreads), kThreads, 0, st>>>(
        L->nseg, G, k, L->seg, L->items, V, lat0, partial);
  note_launches(1);
  if (L->nmed > 0) {
    if (v4)
      k_splat_med<4><<<(unsigned)ceil_div(L->nmed * G, kThreads), kThreads, 0, st>>>(
          L->nmed, G, k, L->med_rows, partial, lat0);
    else
      k_splat_med<1><<<(unsigned)ceil_div(L->nmed * G, kThreads), kThreads, 0, st>>>(
          L->nmed, G, k, L->med_rows, partial, lat0);
    note_launches(1);
  }
  if (L->nhuge > 0) {
    int groups = 1;
    while (groups * 2 * G <= kThreads) groups *= 2;
    if (v4)
      k_splat_huge<4><<<(unsigned)L->nhuge, groups * G, 0, st>>>(G, k, L->huge_rows, partial, lat0);
    else
      k_splat_huge<1><<<(unsigned)L->nhuge, groups * G, 0, st>>>(G, k, L->huge_rows, partial, lat0);
    note_launches(1);
  }
  Taps c{}, g{};
  for (int t = 0; t <= L->r; ++t) {
    c.t[t] = (float)L->coef[t];
    g.t[t] = (float)L->half[t];
  }
  float* a = lat0;
  float* b = lat1;
  auto pass = [&](int j, const Taps& tp) {
    launch_blur_pass(L, j, tp, a, b, k, st);
    float* t = a;
    a = b;
    b = t;
  };
  const int D = L->D;
  if (blur == SGP_BLUR_SEQUENTIAL) {
    for (int j = 0; j < D; ++j) pass(j, c);
  } else if (blur == SGP_BLUR_TRANSPOSE) {
    for (int j = D - 1; j >= 0; --j) pass(j, c);
  } else {
    for (int j = 0; j < D; ++j) pass(j, g);
    for (int j = D - 1; j >= 0; --j) pass(j, g);
  }
  launch_slice(L, a, V_user, k, alpha, beta, out, st);
}

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
