"""Closed-form results the paper compares its method with, restated for use
as pins of the oracle.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import numpy as np
from scipy import integrate, special


def bessel_wave(rho1_0, R, ck, t, r, n_terms=400, nu=0.0):
    """Cylindrical wave solution, Eq. (analyticdensityprop):
    rho1(r, t) = 2/R^2 sum_n J0(k_n r/R) cos(c_k k_n t / R) / J1(k_n)^2
                 * integral_0^R rho1(r', 0) J0(k_n r'/R) r' dr',
    with k_n the zeros of J0.  rho1_0 is a callable of r'.  nu > 0 damps
    every term by exp(-nu (k_n/R)^2 t): each term is a standing radial
    acoustic mode, and such a mode of the scheme decays at nu k^2 (shown by
    the radial-acoustic-mode test); nu = 0 is the paper's inviscid series."""
    kn = special.jn_zeros(0, n_terms)
    r = np.asarray(r, dtype=np.float64)
    out = np.zeros_like(r)
    rr = np.linspace(0.0, R, 8001)
    f0 = rho1_0(rr)
    for k in kn:
        coef = integrate.simpson(f0 * special.j0(k * rr / R) * rr, x=rr)
        out += coef * special.j0(k * r / R) * np.cos(ck * k * t / R) * np.exp(-nu * (k / R) ** 2 * t) / special.j1(k) ** 2
    return 2.0 / R**2 * out


def miller_scriven_omega2(sigma, R0, rho_l, rho_v, nu_l, nu_v, lam=1.0):
    """Mode-2 angular frequency of a viscous droplet, Eq. (oscillatingfreq):
    omega2 = omega* - alpha sqrt(omega*)/2 + alpha^2/4 with
    omega* = sqrt(24 lam sigma / (R0^3 (2 rho_v + 3 rho_l))) and
    alpha = 25 sqrt(nu_l nu_v) rho_l rho_v /
            (sqrt(2) R0 (2 rho_v + 3 rho_l)(sqrt(nu_l) rho_l + sqrt(nu_v) rho_v))."""
    w_star = np.sqrt(24.0 * lam * sigma / (R0**3 * (2.0 * rho_v + 3.0 * rho_l)))
    alpha = (25.0 * np.sqrt(nu_l * nu_v) * rho_l * rho_v) / (
        np.sqrt(2.0) * R0 * (2.0 * rho_v + 3.0 * rho_l) * (np.sqrt(nu_l) * rho_l + np.sqrt(nu_v) * rho_v)
    )
    return w_star - alpha * np.sqrt(w_star) / 2.0 + alpha**2 / 4.0


def hagen_poiseuille(g, R, nu, r):
    """Steady axial pipe flow driven by a body acceleration g: u_z = g (R^2 - r^2) / (4 nu)."""
    return g * (R**2 - np.asarray(r) ** 2) / (4.0 * nu)


def plane_poiseuille(g, R, nu, r):
    """Same drive in plane (2D) geometry with a symmetry line at r = 0: u = g (R^2 - r^2) / (2 nu)."""
    return g * (R**2 - np.asarray(r) ** 2) / (2.0 * nu)


def fit_damped_cosine(t, y, w_guess=None):
    """Least-squares fit y = a + b exp(-c t) cos(w t + d) + e t; returns (w, c).

    Starts from a scan of frequencies (around w_guess when given, else around
    the zero-crossing estimate) and phases and keeps the best fit; the linear
    term absorbs a slow drift of the mean (e.g. a droplet still relaxing)."""
    from scipy import optimize

    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    yc = y - y.mean()
    if w_guess is None:
        s = np.sign(yc)
        idx = np.nonzero(s[1:] * s[:-1] < 0)[0]
        w_guess = np.pi / np.mean(np.diff(t[idx])) if len(idx) >= 2 else 2 * np.pi / (t[-1] - t[0])
    a0, b0 = y.mean(), (y.max() - y.min()) / 2
    span = t[-1] - t[0]

    def model(p, tt):
        a, b, c, w, d, e = p
        return a + b * np.exp(-np.clip(c * (tt - t[0]), -50, 50)) * np.cos(w * tt + d) + e * (tt - t[0])

    best = None
    for wf in (0.5, 0.7, 0.85, 1.0, 1.2, 1.5, 2.0):
        for d0 in np.linspace(0, 2 * np.pi, 6, endpoint=False):
            try:
                res = optimize.least_squares(lambda p: model(p, t) - y, [a0, b0, 1.0 / span, w_guess * wf, d0, 0.0])
            except ValueError:
                continue
            if best is None or res.cost < best.cost:
                best = res
    a, b, c, w, d, e = best.x
    return abs(w), c
