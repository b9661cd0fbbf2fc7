// Blur stencils for stationary kernels (Sec. 4.1).
//
// The taps are kernel values at the lattice points, c_t = k(t s), t = 0..r (symmetric in
// t).  The spacing s is either fixed (the binomial rule: k(s) = 1/2, which for the RBF
// and r = 1 is the [.5, 1, .5] stencil of Sec. 3.2) or chosen by balancing coverage
// (Eq. balance_coverage): the share of the kernel's mass inside [-s m/2, s m/2] (m = 2r+1
// taps) must equal the share of its spectral mass below the Nyquist frequency pi/s.
// Both shares are computed by numerical integration, as the paper does, so any
// stationary kernel only needs its profile k(tau):
//   spatial   int_0^a k / int_0^T k                                   (Simpson)
//   spectral  int_0^W F[k] / int_0^inf F[k] = (2 / (pi k(0))) int_0^T k(t) sin(W t)/t dt
//             (the spectral integral taken in closed form over w inside the tau integral;
//             int_{-inf}^{inf} F[k] = 2 pi k(0))
// and s follows by bisection (the spatial share grows with s, the spectral one shrinks).
//
// The symmetric blur uses the taps g_t of the half kernel k_h (spectral density the
// square root of k's, so k_h * k_h is proportional to k), normalised to sum_t g_t^2 = 1.
#include <cmath>

#include "sgp_internal.cuh"

namespace sgp {
namespace {

double profile(int kernel, double t) {
  t = std::fabs(t);
  if (kernel == SGP_KERNEL_MATERN32_COVERAGE) {
    const double a = std::sqrt(3.0) * t;
    return (1.0 + a) * std::exp(-a);
  }
  return std::exp(-0.5 * t * t);
}

double half_profile(int kernel, double t) {
  t = std::fabs(t);
  if (kernel == SGP_KERNEL_MATERN32_COVERAGE) return std::exp(-std::sqrt(3.0) * t);
  return std::exp(-t * t);
}

constexpr double kTail = 40.0;  // both profiles are below 1e-30 beyond this

template <class F>
double simpson(F f, double a, double b, int intervals) {
  if (intervals % 2) ++intervals;
  const double h = (b - a) / intervals;
  double s = f(a) + f(b);
  for (int i = 1; i < intervals; ++i) s += f(a + i * h) * (i % 2 ? 4.0 : 2.0);
  return s * h / 3.0;
}

double spatial_share(int kernel, double a, double total) {
  return simpson([&](double t) { return profile(kernel, t); }, 0.0, a, 20000) / total;
}

double spectral_share(int kernel, double W) {
  auto f = [&](double t) {
    return t == 0.0 ? W * profile(kernel, 0.0) : profile(kernel, t) * std::sin(W * t) / t;
  };
  return 2.0 / (M_PI * profile(kernel, 0.0)) * simpson(f, 0.0, kTail, 80000);
}

double coverage_spacing(int kernel, int r) {
  const double total = simpson([&](double t) { return profile(kernel, t); }, 0.0, kTail, 80000);
  const double taps = 2.0 * r + 1.0;
  double lo = 0.05, hi = 20.0;
  for (int it = 0; it < 60; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double g = spatial_share(kernel, 0.5 * mid * taps, total) - spectral_share(kernel, M_PI / mid);
    if (g > 0.0) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace

bool make_stencil(int kernel, int r, double spacing_override, double* s, double* coef,
                  double* half) {
  if (r < 1 || r > kMaxOrder) return false;
  if (kernel != SGP_KERNEL_RBF_BINOMIAL && kernel != SGP_KERNEL_RBF_COVERAGE &&
      kernel != SGP_KERNEL_MATERN32_COVERAGE)
    return false;
  double sp;
  if (spacing_override > 0.0) sp = spacing_override;
  else if (kernel == SGP_KERNEL_RBF_BINOMIAL) sp = std::sqrt(2.0 * std::log(2.0));
  else sp = coverage_spacing(kernel, r);
  *s = sp;
  double sq = 0.0;
  for (int t = -r; t <= r; ++t) sq += half_profile(kernel, t * sp) * half_profile(kernel, t * sp);
  for (int t = 0; t <= r; ++t) {
    coef[t] = profile(kernel, t * sp);
    half[t] = half_profile(kernel, t * sp) / std::sqrt(sq);
  }
  return true;
}

}  // namespace sgp
