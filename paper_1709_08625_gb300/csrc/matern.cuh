// matern.cuh -- device evaluation of the Matern covariance of eq. (3),
//
//   C(h) = sigma2 / (2^(nu-1) Gamma(nu)) (h/ell)^nu K_nu(h/ell),  C(0) = sigma2,
//
// with the modified Bessel function of the second kind written from its
// integral representation (DLMF 10.32.9)
//
//   K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt,
//
// evaluated by the trapezoidal rule.  The integrand is even and analytic in
// the strip |Im t| < pi/2, so the rule with step h converges like
// exp(-pi^2 / h) (Trefethen & Weideman, SIAM Review 56, 2014); h = 1/6 puts
// the discretisation error below 1e-20 relative.  The scaled form
// e^x K_nu(x) = int exp(-x (cosh t - 1)) cosh(nu t) dt keeps the sum in range
// for large x; the sum stops once a term is below 1e-18 of the sum and the
// terms are decaying.  The nodes (cosh t_j - 1, cosh(nu t_j)) depend only on
// nu and are tabulated on the host once per parameter set.
//
// nu = 1/2, 3/2, 5/2 use the half-integer closed forms
//   sigma2 e^-x, sigma2 (1 + x) e^-x, sigma2 (1 + x + x^2/3) e^-x.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace hlc {

constexpr int KNU_NODES = 512;     // t_j = j * KNU_STEP, up to t = 85
constexpr double KNU_STEP = 1.0 / 6.0;

struct MaternDev {
  double sigma2, ell, nu, nugget;
  double coef;      // sigma2 / (2^(nu-1) Gamma(nu))
  int kind;         // 0: nu=1/2, 1: nu=3/2, 2: nu=5/2, 3: general nu
  int nnodes;
  const double* cm1;  // cosh(t_j) - 1
  const double* wnu;  // cosh(nu t_j)
};

// Matern value at distance h (FP64).  x = h / ell exactly as in eq. (3).
__device__ __forceinline__ double matern_f64(double h, const MaternDev& p) {
  if (h == 0.0) return p.sigma2;
  const double x = h / p.ell;
  if (p.kind == 0) return p.sigma2 * exp(-x);
  if (p.kind == 1) return p.sigma2 * (1.0 + x) * exp(-x);
  if (p.kind == 2) return p.sigma2 * (1.0 + x + x * x / 3.0) * exp(-x);
  // Below 1e-30 the first correction of x^nu K_nu(x) to its limit
  // 2^(nu-1) Gamma(nu) is (x/2)^(2 nu) Gamma(1-nu)/Gamma(1+nu) < 1e-17 for nu >= 0.3.
  if (x < 1e-30) return p.sigma2;
  // scaled trapezoidal sum S = e^x K_nu(x) / h_step
  double s = 0.5 * p.wnu[0];
  for (int j = 1; j < p.nnodes; ++j) {
    const double e = x * p.cm1[j];
    const double term = exp(-e) * p.wnu[j];
    s += term;
    if (term < 1e-18 * s && e > p.nu * (j * KNU_STEP)) break;
  }
  const double lg = p.nu * log(x) - x;  // log(x^nu e^-x)
  return p.coef * exp(lg) * (s * KNU_STEP);
}

// Euclidean distance without contraction, so that it is rounded like the
// reference host computation.
__device__ __forceinline__ double dist_f64(double x0, double y0, double x1, double y1) {
  const double dx = __dsub_rn(x0, x1), dy = __dsub_rn(y0, y1);
  return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

}  // namespace hlc
