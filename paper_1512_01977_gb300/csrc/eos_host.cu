// Host-side EOS helpers of the library: critical temperature and the
// coexistence densities of the Maxwell construction.  Used to turn T/T_c into
// the absolute temperature of a solve and to build two-phase initial states.
#include <math.h>

#include "lbm_axi.h"
#include "lbm_eos_host.h"

namespace lbm {

// P_k and dP_k/drho at absolute temperature T (same formulas as the device EOS).
static void eos_eval(const lbm_eos& e, double T, double rho, double* p, double* dp) {
    if (e.kind == LBM_EOS_VDW) {
        const double d = 3.0 - rho;
        *p = e.lambda * (8.0 * rho * T / d - 3.0 * rho * rho);
        *dp = e.lambda * (24.0 * T / (d * d) - 6.0 * rho);
        return;
    }
    const double x = e.b * rho * 0.25, om = 1.0 - x, om2 = om * om;
    const double num = 1.0 + x * (1.0 + x * (1.0 - x));
    *p = rho * e.R * T * num / (om2 * om) - e.a * rho * rho;
    const double nd = 1.0 + x * (4.0 + x * (4.0 + x * (-4.0 + x)));
    *dp = e.R * T * nd / (om2 * om2) - 2.0 * e.a * rho;
}

static double eos_p_at(const lbm_eos& e, double T, double rho) {
    double p, dp;
    eos_eval(e, T, rho, &p, &dp);
    return p;
}
static double eos_dp_at(const lbm_eos& e, double T, double rho) {
    double p, dp;
    eos_eval(e, T, rho, &p, &dp);
    return dp;
}

static double rho_max(const lbm_eos& e) { return e.kind == LBM_EOS_VDW ? 3.0 : 4.0 / e.b; }

// Critical point.  vdW in reduced units: T_c = rho_c = 1.  CS: with x = b rho/4
// the pressure is (4RT/b) g(x) - (16a/b^2) x^2, g(x) = x(1+x+x^2-x^3)/(1-x)^3,
// g'(x) = N(x)/(1-x)^4, N = 1 + 4x + 4x^2 - 4x^3 + x^4.  dp/dx = d2p/dx2 = 0
// gives g'(x) = x g''(x), i.e. N(1 - 5x) - x(1 - x) N' = 0, solved by
// bisection on (0, 0.2); then T_c = 8a / (b R g''(x_c)).
bool critical_point(const lbm_eos& e, double* Tc, double* rho_c) {
    if (e.kind == LBM_EOS_VDW) {
        *Tc = 1.0;
        *rho_c = 1.0;
        return true;
    }
    if (!(e.a > 0) || !(e.b > 0) || !(e.R > 0)) return false;
    auto N = [](double x) { return 1.0 + x * (4.0 + x * (4.0 + x * (-4.0 + x))); };
    auto Np = [](double x) { return 4.0 + x * (8.0 + x * (-12.0 + 4.0 * x)); };
    auto cond = [&](double x) { return N(x) * (1.0 - 5.0 * x) - x * (1.0 - x) * Np(x); };
    double lo = 1e-6, hi = 0.2;
    for (int it = 0; it < 200; it++) {
        const double mid = 0.5 * (lo + hi);
        if (cond(mid) > 0) lo = mid; else hi = mid;
    }
    const double x = 0.5 * (lo + hi), om = 1.0 - x;
    const double g2 = (Np(x) * om + 4.0 * N(x)) / (om * om * om * om * om);
    *Tc = 8.0 * e.a / (e.b * e.R * g2);
    *rho_c = 4.0 * x / e.b;
    return true;
}

static double bisect_root(const lbm_eos& e, double T, double lo, double hi, double target, bool use_dp) {
    // f(lo) and f(hi) bracket the root of f(rho) = value(rho) - target.
    auto f = [&](double r) { return (use_dp ? eos_dp_at(e, T, r) : eos_p_at(e, T, r)) - target; };
    double flo = f(lo);
    for (int it = 0; it < 300; it++) {
        const double mid = 0.5 * (lo + hi);
        const double fm = f(mid);
        if ((fm > 0) == (flo > 0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
        if (hi - lo <= 1e-17 * hi) break;
    }
    return 0.5 * (lo + hi);
}

// integral_{rv}^{rl} (P_k - ps) / rho^2 drho, in s = ln(rho): integrand (P_k - ps)/rho,
// 256 panels of 8-point Gauss-Legendre.
static double equal_area_residual(const lbm_eos& e, double T, double rv, double rl, double ps) {
    static const double gx[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    static const double gw[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    const double s0 = log(rv), s1 = log(rl);
    const int panels = 256;
    const double hpan = (s1 - s0) / panels;
    double acc = 0.0;
    for (int q = 0; q < panels; q++) {
        const double c = s0 + (q + 0.5) * hpan, hh = 0.5 * hpan;
        for (int g = 0; g < 4; g++) {
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                const double s = c + sgn * gx[g] * hh;
                const double r = exp(s);
                acc += gw[g] * hh * (eos_p_at(e, T, r) - ps) / r;
            }
        }
    }
    return acc;
}

bool coexistence(const lbm_eos& e, double T, double* rv_out, double* rl_out) {
    double Tc, rc;
    if (!critical_point(e, &Tc, &rc) || !(T > 0) || !(T < Tc)) return false;
    const double rmax = rho_max(e) * (1.0 - 1e-12);
    // spinodals: dP/drho changes sign at ra < rc < rb
    const double ra = bisect_root(e, T, 1e-300, rc, 0.0, true);
    const double rb = bisect_root(e, T, rc, rmax, 0.0, true);
    const double pa = eos_p_at(e, T, ra), pb = eos_p_at(e, T, rb);
    double lo = pb > 1e-12 * pa ? pb : 1e-12 * pa, hi = pa;
    double rv = 0, rl = 0;
    for (int it = 0; it < 200; it++) {
        const double ps = 0.5 * (lo + hi);
        rv = bisect_root(e, T, 0.0, ra, ps, false);
        rl = bisect_root(e, T, rb, rmax, ps, false);
        // the residual decreases with ps
        if (equal_area_residual(e, T, rv, rl, ps) > 0) lo = ps; else hi = ps;
        if (hi - lo <= 1e-16 * hi) break;
    }
    const double ps = 0.5 * (lo + hi);
    *rv_out = bisect_root(e, T, 0.0, ra, ps, false);
    *rl_out = bisect_root(e, T, rb, rmax, ps, false);
    return true;
}

double absolute_temperature(const lbm_eos& e) {
    double Tc, rc;
    if (!critical_point(e, &Tc, &rc)) return -1.0;
    return e.T_over_Tc * Tc;
}

void eos_pressure(const lbm_eos& e, double T, double rho, double* p, double* dp) { eos_eval(e, T, rho, p, dp); }

}  // namespace lbm
