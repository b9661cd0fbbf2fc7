// Simplex-GP oracle: a plain, slow, FP64 CPU statement of the permutohedral-lattice
// kernel MVM  K~ V = W B W^T V  (splat, blur, slice) and of the conjugate-gradient solve
// that drives it.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline / reference legs load this library.  The product path (the CUDA library
// under paper_2106_06695_gb300/) never calls it, links it or shares code with it.
//
// Every step follows the paper's text in its order and notation:
//   * RBF kernel == Gaussian filter after dividing inputs by the lengthscale (Sec. 3.1).
//   * Elevation into H_d with a triangular basis E, enclosing simplex by rounding to the
//     nearest remainder-0 point and ranking the residuals, barycentric weights, the
//     canonical simplex s_k (Sec. 3.2 "Splat", Eq. canon_simplex).
//   * Sparse set of lattice vertices touched by the data, kept fixed during the blur
//     (Sec. 3.2 "Splat" and "Blur").
//   * Blur: a 1-D stencil along each of the d+1 lattice directions in sequence
//     (Sec. 3.2 "Blur"); stencil taps are kernel values k(i*s) (Sec. 4.1).
//   * Slice: the transpose of splat with the cached weights (Sec. 3.2 "Slice").
//   * Spacing s by the spatial/Fourier coverage balance (Sec. 4.1, Eq. balance_coverage).
//   * CG that touches the matrix only through MVMs (Sec. 2; Sec. 5.4; App. A table).
//
// Readings taken where the paper is silent (each is pinned by a test or listed as a
// reading): E is the orthonormal triangular (Helmert) basis of H_d; the scale that maps
// one lattice step (norm sqrt(d(d+1)) in H_d) to s kernel units is sqrt(d(d+1))/s;
// rounding ties go down; rank ties go to the lower coordinate index; every one of the
// d+1 vertices of a simplex is inserted even when its weight is 0; vertex ids follow
// first occurrence in (point, vertex) order; the forward blur runs directions 0..d and
// the transpose runs d..0.  On a truncated lattice the per-direction blurs do not commute,
// so W B W^T is not symmetric; CG (which needs a symmetric positive-definite matrix, as
// K_UU of Eq. k_ski is) uses the symmetric blur M^T M, where M is the same sequence of
// per-direction blurs with the taps g of the half kernel (self-convolution ~ k).
//
// Pins (tests/test_oracle_*.py): the canonical simplex for a point at the origin;
// brute-force enclosing-simplex search for d <= 3; barycentric reconstruction y =
// sum_k w_k key_k; key invariants; the closed form K~(0,0) = 1 + 2^-(d+1) of the
// binomial stencil; the explicit d = 1 matrix; an explicit product of per-direction blur
// matrices built independently from the exported keys; the adjoint identity; the
// Gaussian coverage closed form s = sqrt(2 pi / (2r+1)); CG against a dense solve;
// the exact RBF MVM against scipy's pairwise distances.
//
// Built with -O2 -ffp-contract=off (no fused multiply-add, no fast-math) so that every
// floating-point operation of the lattice construction is one IEEE-rounded operation.
//
// Threads (orc_set_threads, OpenMP when the compiler has it): with more than one thread
// the per-point elevation, the per-vertex blur, the per-point slice, the CG's per-column
// updates and the neighbour lookups run in parallel, each output computed by exactly the
// same operations in the same order as with one thread; the splat becomes a per-vertex
// gather over the vertex's incidences in increasing point order, which is the order in
// which the sequential scatter adds them.  Results are therefore bit-identical for every
// thread count (pinned by a test).  Vertex insertion stays sequential (first-occurrence
// ids).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { ORC_OK = 0, ORC_ERR_INVALID_ARG = 1 };

int g_threads = 1;  // threads of the parallel loops (orc_set_threads)

enum { ORC_RBF_BINOMIAL = 0, ORC_RBF_COVERAGE = 1, ORC_MATERN32_COVERAGE = 2 };

struct Lattice {
  int64_t n = 0;
  int d = 0;
  int D = 0;  // d + 1
  int r = 0;  // stencil order: taps t = -r..r
  std::vector<double> coef;  // c_0..c_r
  std::vector<double> half;  // g_0..g_r: taps of the half kernel, for the symmetric blur
  double s = 0.0;            // lattice spacing in lengthscale-normalised units
  std::vector<double> y;     // [n][D] elevated points
  std::vector<int> rem0;     // [n][D] enclosing remainder-0 point (after the sum fix)
  std::vector<int> rank;     // [n][D] rank of each coordinate (after the sum fix)
  std::vector<double> w;     // [n][D] barycentric weight of vertex k
  std::vector<int> idx;      // [n][D] id of vertex k of point i
  std::vector<int> keys;     // [m][D] integer coordinates of each vertex
  std::vector<double> z;     // [n][d] lengthscale-normalised points x / l
  std::vector<double> f;     // [d] elevation factors scale / sqrt((j+1)(j+2))
  std::vector<double> ls;    // [d] lengthscales
  std::unordered_map<std::string, int> table;  // key -> vertex id
  int64_t m = 0;
  // memo of neighbour lookups: nbr[((j * r + (t-1)) * 2 + (sgn > 0)) * m + v] = id of
  // key_v + sgn t u_j or -1, filled on first use
  std::vector<int> nbr;
  // memo of the splat incidences grouped by vertex (used with more than one thread):
  // the incidences (point i, vertex slot kk) of vertex v are inc[inc_ptr[v] .. inc_ptr[v+1])
  // as i * D + kk, in increasing i
  std::vector<int64_t> inc_ptr;
  std::vector<int64_t> inc;
};

std::string key_bytes(const int* key, int D) {
  return std::string(reinterpret_cast<const char*>(key), sizeof(int) * (size_t)D);
}

int find_vertex(const Lattice& L, const int* key) {
  auto it = L.table.find(key_bytes(key, L.D));
  return it == L.table.end() ? -1 : it->second;
}

// ---------------------------------------------------------------------------------
// Kernels and stencils (Sec. 4.1).
// ---------------------------------------------------------------------------------

double kernel_value(int kind, double tau) {
  tau = std::fabs(tau);
  if (kind == ORC_MATERN32_COVERAGE) {
    const double b = std::sqrt(3.0);
    return (1.0 + b * tau) * std::exp(-b * tau);
  }
  return std::exp(-0.5 * tau * tau);
}

// The "half kernel" k_h, whose self-convolution is proportional to k: its spectral
// density is the square root of k's.  RBF: exp(-tau^2).  Matern-3/2 (spectral density
// (3 + w^2)^-2): exp(-sqrt(3) tau).
double half_kernel_value(int kind, double tau) {
  tau = std::fabs(tau);
  if (kind == ORC_MATERN32_COVERAGE) return std::exp(-std::sqrt(3.0) * tau);
  return std::exp(-tau * tau);
}

// Fraction of the kernel's mass inside [-a, a] (spatial coverage).
double spatial_coverage(int kind, double a) {
  if (kind == ORC_MATERN32_COVERAGE) {
    // integral of (1 + b t) e^{-b t} on [0, a], divided by its value on [0, inf) = 2/b
    const double b = std::sqrt(3.0);
    return 1.0 - std::exp(-b * a) * (1.0 + 0.5 * b * a);
  }
  // Gaussian: erf(a / sqrt 2)
  return std::erf(a / std::sqrt(2.0));
}

// Fraction of the kernel's spectral mass inside [-W, W] (Fourier coverage).
double fourier_coverage(int kind, double W) {
  if (kind == ORC_MATERN32_COVERAGE) {
    // spectral density proportional to (b^2 + w^2)^-2
    const double b = std::sqrt(3.0);
    return (2.0 / M_PI) * (b * W / (b * b + W * W) + std::atan(W / b));
  }
  // Gaussian spectrum is again a unit Gaussian: erf(W / sqrt 2)
  return std::erf(W / std::sqrt(2.0));
}

// Solve Eq. balance_coverage for s by bisection: the spatial side grows with s and the
// Fourier side (Nyquist pi/s) shrinks with s.
double coverage_spacing(int kind, int r) {
  const double taps = 2.0 * r + 1.0;
  double lo = 1e-6, hi = 1e3;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double g = spatial_coverage(kind, 0.5 * mid * taps) - fourier_coverage(kind, M_PI / mid);
    if (g > 0.0) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// ---------------------------------------------------------------------------------
// Splat geometry (Sec. 3.2 "Splat", Eq. canon_simplex).
// ---------------------------------------------------------------------------------

// Elevate one lengthscale-normalised point z (length d) into H_d (length D).
// E has columns e_j = (1, ..., 1, -(j+1), 0, ..., 0) / sqrt((j+1)(j+2)) with j+1 ones:
// orthonormal, each summing to 0.  The extra factor `scale` makes one lattice step equal
// to s kernel units.
void elevate(const double* z, int d, const std::vector<double>& f, double* y) {
  double sm = 0.0;
  for (int i = d; i >= 1; --i) {
    const double cf = z[i - 1] * f[i - 1];
    y[i] = sm - (double)i * cf;
    sm = sm + cf;
  }
  y[0] = sm;
}

// Enclosing simplex of y: nearest remainder-0 point, rank of residuals, sum fix, then
// barycentric weights b[0..d].
void enclosing_simplex(const double* y, int d, int* rem0, int* rank, double* wout) {
  const int D = d + 1;
  std::vector<double> delta(D);
  long long sum = 0;
  for (int i = 0; i < D; ++i) {
    const double q = y[i] / (double)D;
    const double lo = std::floor(q);
    const double down = lo * (double)D;
    const double up = down + (double)D;
    const double r0 = (up - y[i] < y[i] - down) ? up : down;  // ties go down
    rem0[i] = (int)r0;
    sum += rem0[i];
  }
  for (int i = 0; i < D; ++i) delta[i] = y[i] - (double)rem0[i];
  // rank_i = number of residuals strictly larger, plus equal residuals at lower index
  for (int i = 0; i < D; ++i) {
    int rk = 0;
    for (int j = 0; j < D; ++j) {
      if (delta[j] > delta[i] || (delta[j] == delta[i] && j < i)) ++rk;
    }
    rank[i] = rk;
  }
  // rem0 may lie off H_d (coordinate sum h*D != 0): shift the h extreme coordinates
  const long long h = sum / D;
  for (int i = 0; i < D; ++i) {
    rank[i] += (int)h;
    if (rank[i] < 0) {
      rank[i] += D;
      rem0[i] += D;
    } else if (rank[i] > d) {
      rank[i] -= D;
      rem0[i] -= D;
    }
  }
  std::vector<double> b(D + 1, 0.0);
  for (int i = 0; i < D; ++i) {
    const double v = (y[i] - (double)rem0[i]) / (double)D;
    b[d - rank[i]] += v;
    b[D - rank[i]] -= v;
  }
  b[0] = b[0] + (1.0 + b[D]);
  for (int k = 0; k < D; ++k) wout[k] = b[k];
}

// Vertex k of the simplex: rem0 plus the canonical vertex s_k with its coordinates
// permuted by rank.
void vertex_key(const int* rem0, const int* rank, int d, int k, int* key) {
  const int D = d + 1;
  for (int i = 0; i < D; ++i) key[i] = rem0[i] + k - (rank[i] > d - k ? D : 0);
}

// ---------------------------------------------------------------------------------
// Blur (Sec. 3.2 "Blur"): one direction u_j = D e_j - 1 at a time, vertex set fixed,
// absent neighbours contribute nothing.
// ---------------------------------------------------------------------------------

const std::vector<int>& neighbours(const Lattice& L) {
  Lattice& M = const_cast<Lattice&>(L);
  if (M.nbr.empty() && L.m > 0) {
    const int D = L.D;
    M.nbr.assign((size_t)D * L.r * 2 * L.m, -1);
    for (int j = 0; j < D; ++j)
      for (int t = 1; t <= L.r; ++t)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
          for (int64_t v = 0; v < L.m; ++v) {
            std::vector<int> nk(D);
            const int* key = &L.keys[v * D];
            for (int i = 0; i < D; ++i) nk[i] = key[i] + sgn * t * ((i == j ? D : 0) - 1);
            M.nbr[(((size_t)j * L.r + (t - 1)) * 2 + (sgn > 0)) * L.m + v] =
                find_vertex(L, nk.data());
          }
        }
  }
  return M.nbr;
}

void blur_direction(const Lattice& L, int j, int k, const std::vector<double>& in,
                    std::vector<double>& out) {
  const std::vector<int>& nbr = neighbours(L);
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t v = 0; v < L.m; ++v) {
    for (int c = 0; c < k; ++c) out[v * k + c] = L.coef[0] * in[v * k + c];
    for (int t = 1; t <= L.r; ++t) {
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        const int u = nbr[(((size_t)j * L.r + (t - 1)) * 2 + (sgn > 0)) * L.m + v];
        if (u < 0) continue;
        for (int c = 0; c < k; ++c) out[v * k + c] += L.coef[t] * in[(int64_t)u * k + c];
      }
    }
  }
}

// Symmetric blur M^T M with M = B_d ... B_0 built from the half-kernel taps g: passes
// j = 0..d, then j = d..0, each the same per-direction stencil as the paper's blur.
// Every such pass is a symmetric matrix, so M^T M is symmetric positive semi-definite;
// on an untruncated lattice it applies g * g (~ c) along every direction.
void blur_symmetric(const Lattice& L, int k, std::vector<double>& lat) {
  Lattice& G = const_cast<Lattice&>(L);
  std::vector<double> saved = G.coef;
  G.coef = G.half;
  std::vector<double> tmp((size_t)L.m * k);
  for (int step = 0; step < 2 * L.D; ++step) {
    const int j = step < L.D ? step : (2 * L.D - 1 - step);
    blur_direction(L, j, k, lat, tmp);
    lat.swap(tmp);
  }
  G.coef = saved;
}

// Incidences grouped by vertex, in increasing point order (built once, sequentially).
const Lattice& incidences(const Lattice& L) {
  Lattice& M = const_cast<Lattice&>(L);
  if (M.inc_ptr.empty()) {
    M.inc_ptr.assign((size_t)L.m + 1, 0);
    for (int64_t e = 0; e < L.n * L.D; ++e) ++M.inc_ptr[(size_t)L.idx[e] + 1];
    for (int64_t v = 0; v < L.m; ++v) M.inc_ptr[v + 1] += M.inc_ptr[v];
    M.inc.assign((size_t)L.n * L.D, 0);
    std::vector<int64_t> fill(M.inc_ptr.begin(), M.inc_ptr.end() - 1);
    for (int64_t e = 0; e < L.n * L.D; ++e) M.inc[fill[L.idx[e]]++] = e;
  }
  return M;
}

void splat(const Lattice& L, const double* V, int k, std::vector<double>& lat) {
  lat.assign((size_t)L.m * k, 0.0);
  if (g_threads > 1) {
    // the same sums as the scatter below, each vertex's terms added in increasing i
    const Lattice& I = incidences(L);
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1024)
    for (int64_t v = 0; v < L.m; ++v)
      for (int64_t q = I.inc_ptr[v]; q < I.inc_ptr[v + 1]; ++q) {
        const int64_t e = I.inc[q];
        const int64_t i = e / L.D;
        const double wt = L.w[e];
        for (int c = 0; c < k; ++c) lat[v * k + c] += wt * V[i * k + c];
      }
    return;
  }
  for (int64_t i = 0; i < L.n; ++i)
    for (int kk = 0; kk < L.D; ++kk) {
      const int64_t v = L.idx[i * L.D + kk];
      const double wt = L.w[i * L.D + kk];
      for (int c = 0; c < k; ++c) lat[v * k + c] += wt * V[i * k + c];
    }
}

void blur(const Lattice& L, int k, int transpose, std::vector<double>& lat) {
  std::vector<double> tmp((size_t)L.m * k);
  for (int step = 0; step < L.D; ++step) {
    const int j = transpose ? (L.d - step) : step;
    blur_direction(L, j, k, lat, tmp);
    lat.swap(tmp);
  }
}

void slice(const Lattice& L, const std::vector<double>& lat, int k, double* out) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t i = 0; i < L.n; ++i)
    for (int c = 0; c < k; ++c) {
      double acc = 0.0;
      for (int kk = 0; kk < L.D; ++kk)
        acc += L.w[i * L.D + kk] * lat[(int64_t)L.idx[i * L.D + kk] * k + c];
      out[i * k + c] = acc;
    }
}

// out = alpha * K~ V + beta * V ; mode 0 sequential blur (directions 0..d), 1 its
// transpose (directions d..0), 2 symmetric blur M^T M.
void apply(const Lattice& L, const double* V, int k, int mode, double alpha, double beta,
           double* out) {
  std::vector<double> lat;
  std::vector<double> a((size_t)L.n * k);
  splat(L, V, k, lat);
  if (mode == 2) blur_symmetric(L, k, lat);
  else blur(L, k, mode == 1 ? 1 : 0, lat);
  slice(L, lat, k, a.data());
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t e = 0; e < L.n * k; ++e) out[e] = alpha * a[e] + beta * V[e];
}

}  // namespace

extern "C" {

// Threads used by the parallel loops (clamped to 1 without OpenMP); returns the count set.
int orc_set_threads(int t) {
#ifdef _OPENMP
  g_threads = t < 1 ? 1 : t;
#else
  (void)t;
  g_threads = 1;
#endif
  return g_threads;
}

// Processors available to the parallel loops (1 without OpenMP).
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_num_procs();
#else
  return 1;
#endif
}

// Stencil taps c_0..c_r = k(t s), the symmetric-blur taps g_0..g_r and the spacing s
// (Sec. 4.1).  kind: 0 RBF with
// s = sqrt(2 ln 2) (taps 2^-(t^2): the binomial [.5, 1, .5] at r = 1), 1 RBF with s from
// Eq. balance_coverage, 2 Matern-3/2 with s from Eq. balance_coverage.  s_override > 0
// replaces the rule's spacing.
int orc_stencil(int kind, int r, double s_override, double* s_out, double* coef_out,
                double* half_out) {
  if (r < 1 || r > 8 || kind < 0 || kind > 2) return ORC_ERR_INVALID_ARG;
  double s;
  if (s_override > 0.0) s = s_override;
  else if (kind == ORC_RBF_BINOMIAL) s = std::sqrt(2.0 * std::log(2.0));
  else s = coverage_spacing(kind, r);
  *s_out = s;
  for (int t = 0; t <= r; ++t) coef_out[t] = kernel_value(kind, t * s);
  // half taps g_t = k_h(t s), scaled so that sum_{t=-r..r} g_t^2 = c_0 = 1
  double sq = 0.0;
  for (int t = -r; t <= r; ++t) sq += half_kernel_value(kind, t * s) * half_kernel_value(kind, t * s);
  for (int t = 0; t <= r; ++t) half_out[t] = half_kernel_value(kind, t * s) / std::sqrt(sq);
  return ORC_OK;
}

double orc_spatial_coverage(int kind, double a) { return spatial_coverage(kind, a); }
double orc_fourier_coverage(int kind, double w) { return fourier_coverage(kind, w); }

// Build the lattice for n points X[n][d] (fp32, promoted exactly) with lengthscales
// ls[d] (fp32).  coef[0..r] are the stencil taps and s the spacing.
int orc_build(const float* X, const float* ls, int64_t n, int d, int r, const double* coef,
              const double* half, double s, void** out) {
  // coef: taps c_0..c_r of the paper's stencil; half: taps g_0..g_r of the symmetric blur
  if (n < 1 || d < 1 || r < 1 || !(s > 0.0)) return ORC_ERR_INVALID_ARG;
  for (int j = 0; j < d; ++j)
    if (!(ls[j] > 0.0f) || !std::isfinite(ls[j])) return ORC_ERR_INVALID_ARG;
  Lattice* L = new Lattice();
  L->n = n;
  L->d = d;
  L->D = d + 1;
  L->r = r;
  L->s = s;
  L->coef.assign(coef, coef + r + 1);
  L->half.assign(half, half + r + 1);
  const int D = L->D;
  const double scale = std::sqrt((double)(d * (d + 1))) / s;
  std::vector<double> f(d);
  for (int j = 0; j < d; ++j) f[j] = scale / std::sqrt((double)((j + 1) * (j + 2)));
  L->y.resize((size_t)n * D);
  L->rem0.resize((size_t)n * D);
  L->rank.resize((size_t)n * D);
  L->w.resize((size_t)n * D);
  L->idx.resize((size_t)n * D);
  L->f = f;
  L->ls.assign(ls, ls + d);
  L->z.resize((size_t)n * d);
  // per point: scale, elevate, enclosing simplex and weights (independent points)
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double* z = &L->z[i * d];
    for (int j = 0; j < d; ++j) z[j] = (double)X[i * d + j] / (double)ls[j];
    double* y = &L->y[i * D];
    elevate(z, d, f, y);
    enclosing_simplex(y, d, &L->rem0[i * D], &L->rank[i * D], &L->w[i * D]);
  }
  // vertex insertion in (point, vertex) order: ids by first occurrence
  std::vector<int> key(D);
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < D; ++k) {
      vertex_key(&L->rem0[i * D], &L->rank[i * D], d, k, key.data());
      auto ins = L->table.emplace(key_bytes(key.data(), D), (int)L->m);
      if (ins.second) {
        L->keys.insert(L->keys.end(), key.begin(), key.end());
        ++L->m;
      }
      L->idx[i * D + k] = ins.first->second;
    }
  }
  *out = L;
  return ORC_OK;
}

int64_t orc_m(void* h) { return static_cast<Lattice*>(h)->m; }

// Enclosing simplex of one elevated point y (length d+1, coordinates summing to 0):
// rem0, rank and the weights w; keys[k][d+1] of its d+1 vertices.
void orc_simplex(const double* y, int d, int* rem0, int* rank, double* w, int* keys) {
  enclosing_simplex(y, d, rem0, rank, w);
  for (int k = 0; k <= d; ++k) vertex_key(rem0, rank, d, k, keys + (size_t)k * (d + 1));
}

// Elevation of one lengthscale-normalised point z (length d) for spacing s.
void orc_elevate(const double* z, int d, double s, double* y) {
  const double scale = std::sqrt((double)(d * (d + 1))) / s;
  std::vector<double> f(d);
  for (int j = 0; j < d; ++j) f[j] = scale / std::sqrt((double)((j + 1) * (j + 2)));
  elevate(z, d, f, y);
}

// Copy out the build products; any pointer may be null.
void orc_export(void* h, double* y, int* rem0, int* rank, double* w, int* idx, int* keys) {
  const Lattice* L = static_cast<Lattice*>(h);
  const size_t nd = (size_t)L->n * L->D;
  if (y) std::memcpy(y, L->y.data(), nd * sizeof(double));
  if (rem0) std::memcpy(rem0, L->rem0.data(), nd * sizeof(int));
  if (rank) std::memcpy(rank, L->rank.data(), nd * sizeof(int));
  if (w) std::memcpy(w, L->w.data(), nd * sizeof(double));
  if (idx) std::memcpy(idx, L->idx.data(), nd * sizeof(int));
  if (keys) std::memcpy(keys, L->keys.data(), (size_t)L->m * L->D * sizeof(int));
}

// Vertex id of an integer key of length d+1, or -1 when the lattice does not hold it.
int orc_find(void* h, const int* key) { return find_vertex(*static_cast<Lattice*>(h), key); }

// The three stages separately: L = W^T V ; L <- B L (or B^T L) ; out = W L.
void orc_splat(void* h, const double* V, int k, double* lat_out) {
  const Lattice* L = static_cast<Lattice*>(h);
  std::vector<double> lat;
  splat(*L, V, k, lat);
  std::memcpy(lat_out, lat.data(), lat.size() * sizeof(double));
}

void orc_blur(void* h, double* lat_io, int k, int transpose) {
  const Lattice* L = static_cast<Lattice*>(h);
  std::vector<double> lat(lat_io, lat_io + (size_t)L->m * k);
  blur(*L, k, transpose, lat);
  std::memcpy(lat_io, lat.data(), lat.size() * sizeof(double));
}

void orc_slice(void* h, const double* lat_in, int k, double* out) {
  const Lattice* L = static_cast<Lattice*>(h);
  std::vector<double> lat(lat_in, lat_in + (size_t)L->m * k);
  slice(*L, lat, k, out);
}

// out[n][k] = alpha * K~ V + beta * V.  mode 0: K~ = W B W^T with blur directions 0..d;
// 1: its transpose (directions d..0); 2: the symmetric blur M^T M.
int orc_mvm(void* h, const double* V, int k, int mode, double alpha, double beta, double* out) {
  if (k < 1 || mode < 0 || mode > 2) return ORC_ERR_INVALID_ARG;
  apply(*static_cast<Lattice*>(h), V, k, mode, alpha, beta, out);
  return ORC_OK;
}

// Conjugate gradients on (outputscale K~ + noise I) X = B, every column independent
// (Sec. 2: the solver touches the matrix only through MVMs).  A column stops when
// ||r|| / ||b|| <= tol, after max_iter iterations, or when <p, A p> <= 0.
// history (may be null): [max_iter][k]; entry (j, c) receives ||r|| / ||b|| of column c
// after its iteration j + 1 (entries of iterations a column did not run are untouched).
int orc_cg_history(void* h, const double* B, int k, double outputscale, double noise,
                   double tol, int max_iter, int mode, double* X, int* iters, double* relres,
                   double* history) {
  const Lattice* L = static_cast<Lattice*>(h);
  if (k < 1 || max_iter < 0) return ORC_ERR_INVALID_ARG;
  const int64_t n = L->n;
  std::vector<double> r(B, B + n * k), p(B, B + n * k), q((size_t)n * k);
  std::vector<double> rho(k, 0.0), bnorm(k), rel(k, 1.0);
  std::vector<int> active(k, 1), it(k, 0);
  for (int64_t e = 0; e < n * k; ++e) X[e] = 0.0;
  for (int c = 0; c < k; ++c) {
    for (int64_t i = 0; i < n; ++i) rho[c] += r[i * k + c] * r[i * k + c];
    bnorm[c] = std::sqrt(rho[c]);
    if (bnorm[c] == 0.0) {
      active[c] = 0;
      rel[c] = 0.0;
    } else if (1.0 <= tol) {
      active[c] = 0;
    }
  }
  for (int iter = 0; iter < max_iter; ++iter) {
    bool any = false;
    for (int c = 0; c < k; ++c) any = any || active[c];
    if (!any) break;
    apply(*L, p.data(), k, mode, outputscale, noise, q.data());
    // columns are independent; each column's sums run over i in order on one thread
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1)
    for (int c = 0; c < k; ++c) {
      if (!active[c]) continue;
      double pq = 0.0;
      for (int64_t i = 0; i < n; ++i) pq += p[i * k + c] * q[i * k + c];
      if (!(pq > 0.0)) {
        active[c] = 0;
        continue;
      }
      const double alpha = rho[c] / pq;
      double rr = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        X[i * k + c] += alpha * p[i * k + c];
        r[i * k + c] -= alpha * q[i * k + c];
        rr += r[i * k + c] * r[i * k + c];
      }
      it[c] += 1;
      rel[c] = std::sqrt(rr) / bnorm[c];
      if (history) history[(int64_t)iter * k + c] = rel[c];
      if (rel[c] <= tol) {
        active[c] = 0;
        continue;
      }
      const double beta = rr / rho[c];
      rho[c] = rr;
      for (int64_t i = 0; i < n; ++i) p[i * k + c] = r[i * k + c] + beta * p[i * k + c];
    }
  }
  for (int c = 0; c < k; ++c) {
    if (iters) iters[c] = it[c];
    if (relres) relres[c] = rel[c];
  }
  return ORC_OK;
}

int orc_cg(void* h, const double* B, int k, double outputscale, double noise, double tol,
           int max_iter, int mode, double* X, int* iters, double* relres) {
  return orc_cg_history(h, B, k, outputscale, noise, tol, max_iter, mode, X, iters, relres,
                        nullptr);
}

// Exact RBF MVM: out_i = sum_j exp(-||(x_i - x_j) / l||^2 / 2) V_j (Sec. 3.1).
void orc_dense_rbf(const float* X, const float* ls, int64_t n, int d, const double* V, int k,
                   double* out) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    for (int c = 0; c < k; ++c) out[i * k + c] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      double d2 = 0.0;
      for (int a = 0; a < d; ++a) {
        const double t = ((double)X[i * d + a] - (double)X[j * d + a]) / (double)ls[a];
        d2 += t * t;
      }
      const double kv = std::exp(-0.5 * d2);
      for (int c = 0; c < k; ++c) out[i * k + c] += kv * V[j * k + c];
    }
  }
}

// Gradients of the scalar L = <G, alpha K~ V> (G, V: [n][k]) with respect to V, the
// points X and the lengthscales.  K~ V = W B W^T V is linear in V and in every weight
// w_ik; the weights are piecewise linear in the elevated point y (the ranks, remainder-0
// points and vertex ids are piecewise constant), so:
//   dV     = alpha W B^T W^T G                                     (mode 0 <-> 1, 2 = 2)
//   dw_ik  = alpha (<G_i, (B W^T V)[v_ik]> + <V_i, (B^T W^T G)[v_ik]>)
//   dy_ic  = (dw_i[d - rank_ic] - dw_i[(D - rank_ic) mod D]) / D  (from the weight formula:
//            (y_c - rem0_c)/D is added to b[d - rank_c] and subtracted from b[D - rank_c],
//            and b[D] is added to b[0])
//   dz     from y_0 = sum_l a_l, y_i = sum_{l > i} a_l - i a_i with a_l = z_{l-1} f_{l-1}
//   dX_ij  = dz_ij / l_j ;  dl_j = -sum_i dz_ij z_ij / l_j.
// Any output pointer may be null.
int orc_mvm_backward(void* h, const double* V, const double* G, int k, int mode, double alpha,
                     double* dV, double* dX, double* dls) {
  if (k < 1 || mode < 0 || mode > 2) return ORC_ERR_INVALID_ARG;
  const Lattice& L = *static_cast<Lattice*>(h);
  const int d = L.d, D = L.D;
  const int tmode = mode == 2 ? 2 : 1 - mode;
  // B W^T V and B^T W^T G
  std::vector<double> BU, BS;
  splat(L, V, k, BU);
  if (mode == 2) blur_symmetric(L, k, BU);
  else blur(L, k, mode, BU);
  splat(L, G, k, BS);
  if (tmode == 2) blur_symmetric(L, k, BS);
  else blur(L, k, tmode, BS);
  if (dV) {
    slice(L, BS, k, dV);
    for (int64_t e = 0; e < L.n * k; ++e) dV[e] *= alpha;
  }
  if (!dX && !dls) return ORC_OK;
  std::vector<double> dw(D), dy(D), dz(d);
  if (dls) std::fill(dls, dls + d, 0.0);
  for (int64_t i = 0; i < L.n; ++i) {
    for (int kk = 0; kk < D; ++kk) {
      const int64_t v = L.idx[i * D + kk];
      double t = 0.0;
      for (int c = 0; c < k; ++c)
        t += G[i * k + c] * BU[v * k + c] + V[i * k + c] * BS[v * k + c];
      dw[kk] = alpha * t;
    }
    for (int c = 0; c < D; ++c) {
      const int rk = L.rank[i * D + c];
      dy[c] = (dw[d - rk] - dw[(D - rk) % D]) / (double)D;
    }
    // a_l (l = 1..d) enters y_0 and y_i (i < l) with +1 and y_l with -l
    double below = dy[0];  // sum of dy_i for i < l
    for (int l = 1; l <= d; ++l) {
      const double da = below - (double)l * dy[l];
      below += dy[l];
      dz[l - 1] = da * L.f[l - 1];
    }
    for (int j = 0; j < d; ++j) {
      if (dX) dX[i * d + j] = dz[j] / L.ls[j];
      if (dls) dls[j] -= dz[j] * L.z[i * d + j] / L.ls[j];
    }
  }
  return ORC_OK;
}

void orc_free(void* h) { delete static_cast<Lattice*>(h); }

}  // extern "C"
