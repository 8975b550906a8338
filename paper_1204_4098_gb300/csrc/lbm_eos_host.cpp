// Host-side Carnahan-Starling helpers (Li, Luo & Li, Eq. 23): exact critical
// point and Maxwell coexistence densities (Eq. 7).  Used to pick initial
// densities for runs; not part of the per-step path.
//
// With eta = b rho / 4 and g(eta) = eta Z(eta), Z the CS compressibility
// factor, p = (4 R T / b) g(eta) - (16 a / b^2) eta^2 and
//   g'(eta)  = (1 + 4 eta + 4 eta^2 - 4 eta^3 + eta^4) / (1 - eta)^4,
//   g''(eta) = (8 + 20 eta - 4 eta^2) / (1 - eta)^5.
// The critical point has dp/deta = d^2p/deta^2 = 0, i.e. g' = eta g'', whose
// numerator is eta^5 - 5 eta^4 + 4 eta^3 + 20 eta^2 + 5 eta - 1 = 0, and
// R T_c = 8 a / (b g''(eta_c)).
// Maxwell's equal-area rule is solved as equal pressure and equal chemical
// potential, mu = R T [ln rho + (8 eta - 9 eta^2 + 3 eta^3)/(1 - eta)^3] - 2 a rho
// (the CS excess free energy plus the mean-field attraction).
#include <cmath>

#include "lbm.h"

namespace {

struct CS {
  double a, b, R, T;
  double p(double rho) const {
    const double e = b * rho / 4.0;
    return rho * R * T * (1 + e + e * e - e * e * e) / ((1 - e) * (1 - e) * (1 - e)) -
           a * rho * rho;
  }
  double dp(double rho) const {
    const double e = b * rho / 4.0;
    const double om = 1 - e;
    const double g1 = (1 + 4 * e + 4 * e * e - 4 * e * e * e + e * e * e * e) / (om * om * om * om);
    return R * T * g1 - 2 * a * rho;
  }
  double mu(double rho) const {
    const double e = b * rho / 4.0;
    const double om = 1 - e;
    return R * T * (std::log(rho) + (8 * e - 9 * e * e + 3 * e * e * e) / (om * om * om)) -
           2 * a * rho;
  }
};

template <class F>
double bisect(F f, double lo, double hi, int iters = 200) {
  double flo = f(lo);
  for (int i = 0; i < iters; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    const double fm = f(mid);
    if ((fm < 0) == (flo < 0)) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
  }
  return 0.5 * (lo + hi);
}

}  // namespace

extern "C" lbm_status lbm_cs_critical_point(double a, double b, double R, double* rho_c,
                                            double* T_c, double* p_c) {
  if (!(a > 0) || !(b > 0) || !(R > 0) || !rho_c || !T_c || !p_c) return LBM_E_INVAL;
  auto poly = [](double e) {
    return ((((e - 5) * e + 4) * e + 20) * e + 5) * e - 1;
  };
  // single sign change on (0, 1/2): poly(0) = -1, poly(1/2) > 0
  const double eta = bisect(poly, 0.0, 0.5);
  const double om = 1 - eta;
  const double g2 = (8 + 20 * eta - 4 * eta * eta) / (om * om * om * om * om);
  *rho_c = 4.0 * eta / b;
  *T_c = 8.0 * a / (b * g2 * R);
  CS eos{a, b, R, *T_c};
  *p_c = eos.p(*rho_c);
  return LBM_OK;
}

extern "C" lbm_status lbm_cs_maxwell(double T, double a, double b, double R, double* rho_g,
                                     double* rho_l, double* p0_out) {
  if (!rho_g || !rho_l || !p0_out) return LBM_E_INVAL;
  double rc, Tc, pc;
  if (lbm_cs_critical_point(a, b, R, &rc, &Tc, &pc) != LBM_OK) return LBM_E_INVAL;
  if (!(T > 0) || !(T < Tc)) return LBM_E_INVAL;
  CS eos{a, b, R, T};
  const double rmax = 4.0 / b;
  // spinodal: dp = 0 at s1 < rho_c < s2 (dp decreases then increases)
  const int n = 4000;
  double s1 = -1, s2 = -1, prev = eos.dp(rmax * 1e-9);
  for (int i = 1; i <= n; ++i) {
    const double r = rmax * (1e-9 + (1 - 2e-9) * i / n);
    const double d = eos.dp(r);
    if (s1 < 0 && prev > 0 && d <= 0) {
      const double lo = rmax * (1e-9 + (1 - 2e-9) * (i - 1) / n);
      s1 = bisect([&](double x) { return eos.dp(x); }, lo, r);
    } else if (s1 > 0 && s2 < 0 && prev <= 0 && d > 0) {
      const double lo = rmax * (1e-9 + (1 - 2e-9) * (i - 1) / n);
      s2 = bisect([&](double x) { return eos.dp(x); }, lo, r);
      break;
    }
    prev = d;
  }
  if (s1 < 0 || s2 < 0) return LBM_E_INVAL;
  const double p_hi = eos.p(s1);
  double p_lo = eos.p(s2);
  if (p_lo < 0) p_lo = 0;
  auto roots = [&](double p0, double& rg, double& rl) {
    rg = bisect([&](double r) { return eos.p(r) - p0; }, 1e-300, s1);
    rl = bisect([&](double r) { return eos.p(r) - p0; }, s2, rmax * (1 - 1e-15));
  };
  // mu_l - mu_g decreases monotonically in p0 (d mu = dp / rho on each branch)
  auto D = [&](double p0) {
    double rg, rl;
    roots(p0, rg, rl);
    return eos.mu(rl) - eos.mu(rg);
  };
  const double span = p_hi - p_lo;
  const double p0 = bisect(D, p_lo + 1e-12 * span, p_hi - 1e-12 * span);
  roots(p0, *rho_g, *rho_l);
  *p0_out = p0;
  return LBM_OK;
}
