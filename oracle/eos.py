"""Equation-of-state helpers of the oracle: critical point and Maxwell
coexistence densities.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The pressure and its derivative are evaluated by the oracle's C functions
(orc_eos_p, orc_eos_dpdrho), so these helpers and the oracle's update use one
definition of the EOS.

* van der Waals, Eq. (kupershtokvdwpressure): reduced variables, so the critical
  point is T = 1, rho = 1 exactly; lambda only scales the pressure.
* Carnahan-Starling (a, b, R): not in the paper; the critical temperature is
  the largest T at which dP/drho still has a zero, found here by bracketing
  min_rho dP/drho(rho, T) = 0 in T.
* Maxwell construction (equal areas in the p-v plane, v = 1/rho): the
  coexistence pair satisfies p(rho_v) = p(rho_l) = p_s and
  integral_{v_l}^{v_v} (p(v) - p_s) dv = 0.
"""
import numpy as np
from scipy import integrate, optimize


def _p(params, rho):
    from . import core

    return core.eos_p(params, rho)


def _dp(params, rho):
    from . import core

    return core.eos_dpdrho(params, rho)


def _rho_max(params):
    """Upper density bound of the EOS (packing limit)."""
    return 3.0 if params.eos == 0 else 4.0 / params.b


def critical_point(params):
    """(T_c, rho_c) of the EOS in `params` (its T is ignored)."""
    if params.eos == 0:
        return 1.0, 1.0
    hi_rho = 0.999 * _rho_max(params)

    def min_slope(T):
        p2 = params.replace(T=T)
        res = optimize.minimize_scalar(
            lambda r: _dp(p2, r), bounds=(1e-6, hi_rho), method="bounded", options={"xatol": 1e-13}
        )
        return res.fun, res.x

    # dP/drho is linear in T (p = T g(rho) - a rho^2): bracket the T where its minimum is 0.
    lo, hi = 1e-4, 1.0
    while min_slope(hi)[0] < 0:
        hi *= 2.0
    Tc = optimize.brentq(lambda T: min_slope(T)[0], lo, hi, xtol=1e-15, rtol=1e-15)
    return Tc, min_slope(Tc)[1]


def spinodals(params):
    """Densities (rho_a < rho_b) where dP/drho = 0 at T < T_c."""
    Tc, rc = critical_point(params)
    if params.T >= Tc:
        raise ValueError("no spinodal above the critical temperature")
    hi_rho = 0.999 * _rho_max(params)
    res = optimize.minimize_scalar(lambda r: _dp(params, r), bounds=(1e-8, hi_rho), method="bounded",
                                   options={"xatol": 1e-13})
    rmin = res.x
    ra = optimize.brentq(lambda r: _dp(params, r), 1e-12, rmin, xtol=1e-15)
    rb = optimize.brentq(lambda r: _dp(params, r), rmin, hi_rho, xtol=1e-15)
    return ra, rb


def maxwell_densities(params):
    """Coexistence densities (rho_v, rho_l) from the equal-area construction."""
    ra, rb = spinodals(params)
    p_a, p_b = _p(params, ra), _p(params, rb)  # local max (vapour side), local min (liquid side)
    hi_rho = 0.999 * _rho_max(params)

    def branch_densities(ps):
        rv = optimize.brentq(lambda r: _p(params, r) - ps, 0.0, ra, xtol=1e-16, rtol=1e-15)
        rl = optimize.brentq(lambda r: _p(params, r) - ps, rb, hi_rho, xtol=1e-16, rtol=1e-15)
        return rv, rl

    def area(ps):
        rv, rl = branch_densities(ps)
        # integral over v of (p - ps) from v_l to v_v; dv = -drho / rho^2.  Taken in
        # s = ln(rho) (drho = rho ds) so the integrand (p - ps)/rho stays bounded.
        val, _ = integrate.quad(lambda s: (_p(params, np.exp(s)) - ps) / np.exp(s), np.log(rv),
                                np.log(rl), epsabs=1e-14, epsrel=1e-13, limit=400)
        return val

    lo = max(p_b, 1e-12 * p_a) + 1e-15 * abs(p_a)
    hi = p_a - 1e-15 * abs(p_a)
    ps = optimize.brentq(area, lo, hi, xtol=1e-18, rtol=1e-15)
    rv, rl = branch_densities(ps)
    return rv, rl


def temperature_from_ratio(params, T_over_Tc):
    """Absolute EOS temperature for a reduced temperature T/T_c."""
    Tc, _ = critical_point(params)
    return T_over_Tc * Tc


def sound_speed_sq(params, rho):
    """c_k^2 = dP/drho at rho."""
    return _dp(params, rho)
