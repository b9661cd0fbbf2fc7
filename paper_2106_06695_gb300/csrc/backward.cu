// Backward of the lattice MVM  out = alpha W B W^T V  (Sec. 3.2; Sec. 4.2).
//
// For a scalar loss L with G = dL/dout:
//   dV = alpha W B^T W^T G: the transpose product on the same lattice (the sequential
//        blur's transpose runs the directions in reverse; the symmetric blur is its own).
//   dX, dl, two ways (sgp_mvm_backward's `grad`):
//   SGP_GRAD_LATTICE  the exact derivative of the product the forward computes.  It is
//        multilinear in V and in the barycentric weights w_ik, and the weights are
//        piecewise linear in the elevated point y (ranks, remainder-0 points and vertex
//        ids are piecewise constant):
//          dw_ik = alpha (<G_i, (B W^T V)[v_ik]> + <V_i, (B^T W^T G)[v_ik]>)
//          dy_ic = (dw_i[d - rank_ic] - dw_i[(D - rank_ic) mod D]) / D
//        then the transpose of the elevation y = E (x / l) (triangular basis E, scaled).
//   SGP_GRAD_FILTER   Sec. 4.2: the kernel's own input gradient
//          dL/dz_n = 2 sum_j k'_nj [(g_n . v_j) + (g_j . v_n)] (z_n - z_j),  z = x / l,
//        from one filtering of the columns [z (.) g, g, z (.) v, v] with k' = dk/d(d^2);
//        for the RBF k' = -k / 2, so the filter is the lattice operator itself.
//   Both: dX = dz / l, and dl_j = -sum_i dX_ij x_ij / l_j (fixed-order reduction).
#include <algorithm>
#include <cmath>
#include <vector>

#include "sgp_internal.cuh"
#include "values.cuh"

namespace sgp {
namespace {

constexpr int kBT = 128;
constexpr int kDlsBlocks = 2 * 152;
constexpr int kFilterChunk = 256;  // columns per filtering product

template <class S, int VEC>
__device__ __forceinline__ float row_dot2(const float* g, const S* bu, const float* v,
                                          const S* bs, int k) {
  float acc = 0.f;
  if (VEC == 4) {
    for (int c = 0; c < k; c += 4) {
      const float4 gv = *reinterpret_cast<const float4*>(g + c);
      const float4 vv = *reinterpret_cast<const float4*>(v + c);
      const float4 a = Store<S>::ld4(bu + c);
      const float4 b = Store<S>::ld4(bs + c);
      acc = fmaf(gv.x, a.x, acc);
      acc = fmaf(gv.y, a.y, acc);
      acc = fmaf(gv.z, a.z, acc);
      acc = fmaf(gv.w, a.w, acc);
      acc = fmaf(vv.x, b.x, acc);
      acc = fmaf(vv.y, b.y, acc);
      acc = fmaf(vv.z, b.z, acc);
      acc = fmaf(vv.w, b.w, acc);
    }
  } else {
    for (int c = 0; c < k; ++c) {
      acc = fmaf(g[c], Store<S>::ld1(bu + c), acc);
      acc = fmaf(v[c], Store<S>::ld1(bs + c), acc);
    }
  }
  return acc;
}

// Exact derivative through the weights: one thread per point (locality order p); dX in
// the caller's order.  f[j] = scale / sqrt((j+1)(j+2)) are the elevation factors.
template <int MAXD, int VEC, class S>
__global__ void __launch_bounds__(kBT) k_weight_grad(int64_t n, int d, int k,
                                                     const int32_t* __restrict__ perm,
                                                     const int32_t* __restrict__ idx,
                                                     const uint8_t* __restrict__ rank,
                                                     const S* __restrict__ BU,
                                                     const S* __restrict__ BS,
                                                     const float* __restrict__ Vp,
                                                     const float* __restrict__ Gp, float alpha,
                                                     const double* __restrict__ f,
                                                     const float* __restrict__ ls,
                                                     float* __restrict__ dX) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int D = d + 1;
  float dw[MAXD];
  for (int kk = 0; kk < D; ++kk) {
    const int64_t v = idx[p * D + kk];
    dw[kk] = alpha * row_dot2<S, VEC>(Gp + p * k, BU + v * k, Vp + p * k, BS + v * k, k);
  }
  double dy[MAXD];
  for (int c = 0; c < D; ++c) {
    const int rk = rank[p * D + c];
    dy[c] = ((double)dw[d - rk] - (double)dw[(D - rk) % D]) / (double)D;
  }
  // y_0 = sum_l a_l, y_i = sum_{l > i} a_l - i a_i, a_l = z_{l-1} f_{l-1}
  const int64_t i = perm[p];
  double below = dy[0];
  for (int l = 1; l <= d; ++l) {
    const double da = below - (double)l * dy[l];
    below += dy[l];
    dX[i * d + (l - 1)] = (float)(da * f[l - 1] / (double)ls[l - 1]);
  }
}

// Filter inputs, columns [col0, col0 + kc) of [z (.) g | g | z (.) v | v] ([n][kk],
// kk = 2 k (d + 1); column c d + t of a z-block holds g_c z_t), caller's order.
__global__ void k_filter_in(int64_t n, int d, int k, int col0, int kc,
                            const float* __restrict__ X, const float* __restrict__ ls,
                            const float* __restrict__ V, const float* __restrict__ G,
                            float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * kc) return;
  const int64_t i = e / kc;
  const int q = col0 + (int)(e - i * kc);
  const int kd = k * d;
  float val;
  if (q < kd) {
    val = G[i * k + q / d] * (X[i * d + q % d] / ls[q % d]);
  } else if (q < kd + k) {
    val = G[i * k + (q - kd)];
  } else if (q < 2 * kd + k) {
    const int r = q - kd - k;
    val = V[i * k + r / d] * (X[i * d + r % d] / ls[r % d]);
  } else {
    val = V[i * k + (q - 2 * kd - k)];
  }
  out[e] = val;
}

// Accumulate the filtered columns [col0, col0 + kc) into dZ ([n][d], fp32, caller's order)
// without the factor 2 alpha k'/k: one thread per point, columns in order.
__global__ void k_filter_acc(int64_t n, int d, int k, int col0, int kc,
                             const float* __restrict__ X, const float* __restrict__ ls,
                             const float* __restrict__ V, const float* __restrict__ G,
                             const float* __restrict__ F, float* __restrict__ dZ) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int kd = k * d;
  float* dz = dZ + i * d;
  for (int j = 0; j < kc; ++j) {
    const int q = col0 + j;
    const float fv = F[i * kc + j];
    if (q < kd) {  // K (z (.) g): - v_c (K z_t g_c)
      dz[q % d] -= V[i * k + q / d] * fv;
    } else if (q < kd + k) {  // K g: + z_t v_c (K g_c)
      const float vc = V[i * k + (q - kd)] * fv;
      for (int t = 0; t < d; ++t) dz[t] += (X[i * d + t] / ls[t]) * vc;
    } else if (q < 2 * kd + k) {  // K (z (.) v): - g_c (K z_t v_c)
      const int r = q - kd - k;
      dz[r % d] -= G[i * k + r / d] * fv;
    } else {  // K v: + z_t g_c (K v_c)
      const float gc = G[i * k + (q - 2 * kd - k)] * fv;
      for (int t = 0; t < d; ++t) dz[t] += (X[i * d + t] / ls[t]) * gc;
    }
  }
}

__global__ void k_filter_finish(int64_t n, int d, float scale, const float* __restrict__ ls,
                                float* __restrict__ dX) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * d) return;
  dX[e] = scale * dX[e] / ls[e % d];
}

// dl_j = -sum_i dX_ij x_ij / l_j: per-block partials (thread t owns column t % d and
// rows t / d, t / d + P, ... of the block's range, P = floor(256 / d)), combined in a
// fixed order; then the blocks in order.
__global__ void __launch_bounds__(256) k_dls_partial(int64_t n, int d, const float* __restrict__ X,
                                                     const float* __restrict__ dX,
                                                     double* __restrict__ partial) {
  __shared__ double sh[256];
  const int P = 256 / d;
  const int t = threadIdx.x;
  const int j = t % d, phase = t / d;
  const int64_t rows = ceil_div(n, (int64_t)gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int64_t r1 = std::min<int64_t>(n, r0 + rows);
  double acc = 0.0;
  if (phase < P)
    for (int64_t i = r0 + phase; i < r1; i += P) acc += (double)dX[i * d + j] * (double)X[i * d + j];
  sh[t] = acc;
  __syncthreads();
  if (t < d) {
    double s = 0.0;
    for (int ph = 0; ph < P; ++ph) s += sh[ph * d + t];
    partial[(int64_t)blockIdx.x * d + t] = s;
  }
}

__global__ void k_dls_final(int nblk, int d, const double* __restrict__ partial,
                            const float* __restrict__ ls, float* __restrict__ dls) {
  const int j = threadIdx.x;
  if (j >= d) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * d + j];
  dls[j] = (float)(-s / (double)ls[j]);
}

#define BW_CHECK(expr, what)                                  \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return cuda_status(e_, what);      \
  } while (0)

struct Work {
  cudaStream_t st;
  std::vector<void*> ptrs;
  ~Work() {
    for (void* p : ptrs) (void)cudaFreeAsync(p, st);
  }
  template <class T>
  cudaError_t get(T** p, size_t bytes) {
    cudaError_t e = dev_malloc((void**)p, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) ptrs.push_back((void*)*p);
    return e;
  }
};

template <class S, int VEC>
void launch_weight_grad(const Lattice* L, int k, const void* BU, const void* BS, const float* Vp,
                        const float* Gp, float alpha, const double* f, const float* ls, float* dX,
                        cudaStream_t st) {
  const unsigned grid = (unsigned)ceil_div(L->n, kBT);
  const int D = L->D;
#define SGP_WG(MAXD)                                                                        \
  k_weight_grad<MAXD, VEC, S><<<grid, kBT, 0, st>>>(L->n, L->d, k, L->perm, L->idx, L->rank, \
                                                    (const S*)BU, (const S*)BS, Vp, Gp,      \
                                                    alpha, f, ls, dX)
  if (D <= 8) SGP_WG(8);
  else if (D <= 16) SGP_WG(16);
  else if (D <= 32) SGP_WG(32);
  else if (D <= 64) SGP_WG(64);
  else SGP_WG(128);
#undef SGP_WG
  note_launches(1);
}

int transpose_blur(int blur) {
  return blur == SGP_BLUR_SEQUENTIAL ? SGP_BLUR_TRANSPOSE
         : blur == SGP_BLUR_TRANSPOSE ? SGP_BLUR_SEQUENTIAL
                                      : SGP_BLUR_SYMMETRIC;
}

}  // namespace

sgp_status run_mvm_backward(Lattice* L, const float* X, const float* ls, const float* V,
                            const float* G, int k, int blur, float alpha, int grad, float* dV,
                            float* dX, float* dls) {
  cudaStream_t st = L->stream;
  const int64_t n = L->n;
  const int d = L->d;
  Work w{st, {}};
  const bool want_x = dX || dls;
  float* dXw = dX;
  if (want_x && !dXw) BW_CHECK(w.get(&dXw, (size_t)n * d * sizeof(float)), "alloc dX");

  if (grad == SGP_GRAD_LATTICE) {
    sgp_status s = ensure_lattice_values(L, k, st);
    if (s != SGP_OK) return s;
    const size_t vb = lattice_value_bytes(L, k);
    void *b0 = nullptr, *b1 = nullptr;
    float *Vp = nullptr, *Gp = nullptr;
    BW_CHECK(w.get(&b0, vb), "alloc lattice values");
    BW_CHECK(w.get(&b1, vb), "alloc lattice values");
    BW_CHECK(w.get(&Vp, (size_t)n * k * sizeof(float)), "alloc V");
    BW_CHECK(w.get(&Gp, (size_t)n * k * sizeof(float)), "alloc G");
    enqueue_permute(L, G, k, Gp, st);
    // B^T W^T G into (b0, b1), B W^T V into the handle's buffers
    const void* BS = enqueue_splat_blur(L, Gp, k, transpose_blur(blur), b0, b1, L->partial, st);
    if (dV) enqueue_slice_caller(L, BS, k, alpha, dV, st);
    if (want_x) {
      enqueue_permute(L, V, k, Vp, st);
      const void* BU = enqueue_splat_blur(L, Vp, k, blur, L->lat[0], L->lat[1], L->partial, st);
      const double scale = std::sqrt((double)(d * (d + 1))) / L->s;
      std::vector<double> hf(d);
      for (int j = 0; j < d; ++j) hf[j] = scale / std::sqrt((double)((j + 1) * (j + 2)));
      double* f = nullptr;
      BW_CHECK(w.get(&f, d * sizeof(double)), "alloc f");
      // pageable source: the call returns once hf has been staged
      BW_CHECK(cudaMemcpyAsync(f, hf.data(), d * sizeof(double), cudaMemcpyHostToDevice, st),
               "copy f");
      const bool v4 = k % 4 == 0;
      if (L->value_dtype == SGP_VALUES_BF16) {
        if (v4) launch_weight_grad<bf16, 4>(L, k, BU, BS, Vp, Gp, alpha, f, ls, dXw, st);
        else launch_weight_grad<bf16, 1>(L, k, BU, BS, Vp, Gp, alpha, f, ls, dXw, st);
      } else {
        if (v4) launch_weight_grad<float, 4>(L, k, BU, BS, Vp, Gp, alpha, f, ls, dXw, st);
        else launch_weight_grad<float, 1>(L, k, BU, BS, Vp, Gp, alpha, f, ls, dXw, st);
      }
    }
  } else {  // SGP_GRAD_FILTER
    if (dV) {
      sgp_status s = ensure_lattice_values(L, k, st);
      if (s != SGP_OK) return s;
      enqueue_mvm(L, G, k, transpose_blur(blur), alpha, 0.f, dV, st);
    }
    if (want_x) {
      const int kk = 2 * k * (d + 1);
      const int chunk = std::min(kk, kFilterChunk);
      sgp_status s = ensure_lattice_values(L, chunk, st);
      if (s != SGP_OK) return s;
      float *in = nullptr, *F = nullptr;
      BW_CHECK(w.get(&in, (size_t)n * chunk * sizeof(float)), "alloc filter input");
      BW_CHECK(w.get(&F, (size_t)n * chunk * sizeof(float)), "alloc filter output");
      BW_CHECK(cudaMemsetAsync(dXw, 0, (size_t)n * d * sizeof(float), st), "clear dX");
      for (int col0 = 0; col0 < kk; col0 += chunk) {
        const int kc = std::min(chunk, kk - col0);
        k_filter_in<<<(unsigned)ceil_div(n * kc, 256), 256, 0, st>>>(n, d, k, col0, kc, X, ls, V,
                                                                      G, in);
        enqueue_mvm(L, in, kc, blur, 1.f, 0.f, F, st);
        k_filter_acc<<<(unsigned)ceil_div(n, kBT), kBT, 0, st>>>(n, d, k, col0, kc, X, ls, V, G,
                                                                 F, dXw);
        note_launches(2);
      }
      // dz = 2 alpha (k'/k) dZ with k' = -k/2 for the RBF; dX = dz / l
      k_filter_finish<<<(unsigned)ceil_div(n * d, 256), 256, 0, st>>>(n, d, -alpha, ls, dXw);
      note_launches(1);
    }
  }
  if (dls) {
    double* part = nullptr;
    BW_CHECK(w.get(&part, (size_t)kDlsBlocks * d * sizeof(double)), "alloc partials");
    k_dls_partial<<<kDlsBlocks, 256, 0, st>>>(n, d, X, dXw, part);
    k_dls_final<<<1, 128, 0, st>>>(kDlsBlocks, d, part, ls, dls);
    note_launches(2);
  }
  BW_CHECK(cudaGetLastError(), "launching the MVM backward");
  return SGP_OK;
}

}  // namespace sgp
