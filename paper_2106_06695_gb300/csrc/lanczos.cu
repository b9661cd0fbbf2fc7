// Log-determinant of A = outputscale K~ + noise I by stochastic Lanczos quadrature (the
// log-det term of Eq. gp_mll; App. A: at most 100 Lanczos iterations).
//
// For a probe z, m steps of Lanczos on (A, z / ||z||) give a symmetric tridiagonal T_m
// with z^T log(A) z ~ ||z||^2 e1^T log(T_m) e1 (Gauss quadrature of the spectral measure
// of z); averaging over probes with E[z z^T] = I estimates tr log(A) = log det A.  The
// Lanczos coefficients are read off the plain CG run on A x = z (the CG-Lanczos
// correspondence): with CG's step sizes alpha_j and ratios beta_j,
//   T[j][j]   = 1 / alpha_j + beta_{j-1} / alpha_{j-1}     (the second term absent at j = 0)
//   T[j+1][j] = sqrt(beta_j) / alpha_j.
// e1^T log(T) e1 = sum_i q_i^2 log(lambda_i) over T's eigenpairs, with q_i the first
// component of eigenvector i: computed per probe by the implicit QL iteration with
// Wilkinson shifts (Bowdler, Martin, Reinsch & Wilkinson 1968), carrying only the first
// row of the accumulated rotations.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sgp_internal.cuh"

namespace sgp {
namespace {

constexpr int kMaxLanczos = 256;
constexpr int kQlSweeps = 64;  // QL iterations allowed per eigenvalue

// One thread per probe column c: quad[c] = ||z_c||^2 e1^T log(T_c) e1; NaN when T is not
// positive definite or QL did not converge (flagged in *bad).
__global__ void k_slq(const double* __restrict__ ha, const double* __restrict__ hb, int k, int cap,
                      const int* __restrict__ iters, const double* __restrict__ bnorm,
                      double* __restrict__ quad, int* __restrict__ bad) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const int m = min(iters[c], cap);
  const double nz2 = bnorm[c] * bnorm[c];
  if (m == 0) {
    quad[c] = 0.0;
    return;
  }
  double d[kMaxLanczos], e[kMaxLanczos], q[kMaxLanczos];
  for (int j = 0; j < m; ++j) {
    const double a = ha[(int64_t)j * k + c];
    d[j] = 1.0 / a + (j > 0 ? hb[(int64_t)(j - 1) * k + c] / ha[(int64_t)(j - 1) * k + c] : 0.0);
    e[j] = j + 1 < m ? sqrt(hb[(int64_t)j * k + c]) / a : 0.0;
    q[j] = j == 0 ? 1.0 : 0.0;
  }
  // implicit QL: e[i] couples i and i + 1
  bool ok = true;
  for (int l = 0; l < m && ok; ++l) {
    for (int sweep = 0;; ++sweep) {
      int mm = l;
      for (; mm < m - 1; ++mm) {
        const double dd = fabs(d[mm]) + fabs(d[mm + 1]);
        if (fabs(e[mm]) <= 1e-15 * dd) break;
      }
      if (mm == l) break;
      if (sweep == kQlSweeps) {
        ok = false;
        break;
      }
      // Wilkinson shift from the leading 2 x 2 block
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
      double s = 1.0, cc = 1.0, p = 0.0;
      int i = mm - 1;
      for (; i >= l; --i) {
        const double f = s * e[i];
        const double b = cc * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {  // split: deflate and restart this eigenvalue
          d[i + 1] -= p;
          e[mm] = 0.0;
          break;
        }
        s = f / r;
        cc = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * cc * b;
        p = s * r;
        d[i + 1] = g + p;
        g = cc * r - b;
        const double qi1 = q[i + 1];  // first row of the accumulated rotations
        q[i + 1] = s * q[i] + cc * qi1;
        q[i] = cc * q[i] - s * qi1;
      }
      if (r == 0.0 && i >= l) continue;
      d[l] -= p;
      e[l] = g;
      e[mm] = 0.0;
    }
  }
  double acc = 0.0;
  for (int j = 0; j < m && ok; ++j) {
    if (!(d[j] > 0.0)) ok = false;
    else acc += q[j] * q[j] * log(d[j]);
  }
  if (!ok) {
    quad[c] = nan("");
    atomicOr(bad, 1);
    return;
  }
  quad[c] = nz2 * acc;
}

}  // namespace

sgp_status run_logdet(Lattice* L, const float* Z, int s, float noise, int max_lanczos, float tol,
                      double* logdet, double* quad) {
  cudaStream_t st = L->stream;
  const int cap = std::min(max_lanczos, kMaxLanczos);
  struct Bufs {
    cudaStream_t st;
    std::vector<void*> p;
    ~Bufs() {
      for (void* x : p) (void)cudaFreeAsync(x, st);
    }
  } b{st, {}};
  auto get = [&](void** x, size_t bytes) {
    cudaError_t e = dev_malloc(x, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) b.p.push_back(*x);
    return e;
  };
#define LZ_CHECK(expr, what)                                 \
  do {                                                       \
    cudaError_t e_ = (expr);                                 \
    if (e_ != cudaSuccess) return cuda_status(e_, what);     \
  } while (0)
  LanczosRecord rec{};
  rec.cap = cap;
  float* X = nullptr;
  double* dq = nullptr;
  int* bad = nullptr;
  LZ_CHECK(get((void**)&rec.alpha, (size_t)cap * s * sizeof(double)), "alloc Lanczos record");
  LZ_CHECK(get((void**)&rec.beta, (size_t)cap * s * sizeof(double)), "alloc Lanczos record");
  LZ_CHECK(get((void**)&rec.bnorm, (size_t)s * sizeof(double)), "alloc Lanczos record");
  LZ_CHECK(get((void**)&rec.iters, (size_t)s * sizeof(int)), "alloc Lanczos record");
  LZ_CHECK(get((void**)&X, (size_t)L->n * s * sizeof(float)), "alloc CG solution");
  LZ_CHECK(get((void**)&dq, (size_t)s * sizeof(double)), "alloc quadratures");
  LZ_CHECK(get((void**)&bad, sizeof(int)), "alloc flag");
  LZ_CHECK(cudaMemsetAsync(bad, 0, sizeof(int), st), "clear flag");
  sgp_status status = run_cg(L, Z, s, SGP_BLUR_SYMMETRIC, noise, tol, cap, X, nullptr, nullptr,
                             0, 0, &rec);
  if (status != SGP_OK) return status;
  k_slq<<<(unsigned)ceil_div(s, 64), 64, 0, st>>>(rec.alpha, rec.beta, s, cap, rec.iters,
                                                   rec.bnorm, dq, bad);
  note_launches(1);
  LZ_CHECK(cudaGetLastError(), "Lanczos quadrature");
  std::vector<double> hq(s);
  int hbad = 0;
  LZ_CHECK(cudaMemcpyAsync(hq.data(), dq, s * sizeof(double), cudaMemcpyDeviceToHost, st),
           "read quadratures");
  LZ_CHECK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
  LZ_CHECK(cudaStreamSynchronize(st), "sync Lanczos");
#undef LZ_CHECK
  if (quad) std::copy(hq.begin(), hq.end(), quad);
  double sum = 0.0;
  for (double v : hq) sum += v;
  if (logdet) *logdet = sum / s;
  if (hbad) {
    set_error("sgp_logdet: a Lanczos tridiagonal was not positive definite or its eigenvalues "
              "did not converge");
    return SGP_ERR_NONFINITE;
  }
  return SGP_OK;
}

}  // namespace sgp
