"""Pins of the oracle's building blocks against exact identities and closed forms.

Each test fixes a piece of the paper's arithmetic by a property that a dropped
term, a wrong sign, a wrong index or a transposed operand would violate.
"""
import numpy as np
import pytest

import oracle as O
from oracle import core

CZ = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CR = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _lattice_from_feq():
    """Recover (c_i, w_i) of the oracle from f^eq(rho=1) and its u-derivative,
    so that the moment tests below do not lean on a table retyped here."""
    f0 = core.feq(1.0, 0.0, 0.0)
    e = 1e-6
    cz = np.rint((core.feq(1.0, e, 0.0) - core.feq(1.0, -e, 0.0)) / (2 * e) / (3 * f0)).astype(int)
    cr = np.rint((core.feq(1.0, 0.0, e) - core.feq(1.0, 0.0, -e)) / (2 * e) / (3 * f0)).astype(int)
    return f0, cz, cr


def test_lattice_is_d2q9():
    """Sec. II.A: nine velocities (0,0), (+-1,0), (0,+-1), (+-1,+-1); weights 4/9, 1/9, 1/36."""
    w, cz, cr = _lattice_from_feq()
    pairs = sorted(zip(cz.tolist(), cr.tolist()))
    assert pairs == sorted((a, b) for a in (-1, 0, 1) for b in (-1, 0, 1))
    for wi, a, b in zip(w, cz, cr):
        expect = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}[abs(a) + abs(b)]
        assert wi == pytest.approx(expect, rel=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_feq_moments(seed):
    """sum f^eq = rho, sum c f^eq = rho u, sum c c f^eq = rho (c_s^2 I + u u)."""
    rng = np.random.default_rng(seed)
    _, cz, cr = _lattice_from_feq()
    rho, uz, ur = rng.uniform(0.01, 2.0), rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1)
    f = core.feq(rho, uz, ur)
    assert f.sum() == pytest.approx(rho, rel=1e-14)
    assert (f * cz).sum() == pytest.approx(rho * uz, abs=1e-15 * rho)
    assert (f * cr).sum() == pytest.approx(rho * ur, abs=1e-15 * rho)
    assert (f * cz * cz).sum() == pytest.approx(rho * (1 / 3 + uz * uz), rel=1e-14)
    assert (f * cr * cr).sum() == pytest.approx(rho * (1 / 3 + ur * ur), rel=1e-14)
    assert (f * cz * cr).sum() == pytest.approx(rho * uz * ur, abs=1e-15 * rho)


@pytest.mark.parametrize("seed", [3, 4])
def test_source_h_moments(seed):
    """Sec. II.B: h_i's zeroth moment is the mass sink -rho u_r / r, its first
    moment is (H_z, H_r), its second moment is c_s^2 (-rho u_r / r) I."""
    rng = np.random.default_rng(seed)
    r, rho, ur, Hz, Hr = rng.uniform(0.5, 20), rng.uniform(0.1, 1), rng.uniform(-0.05, 0.05), \
        rng.uniform(-1e-3, 1e-3), rng.uniform(-1e-3, 1e-3)
    h = core.source_h(r, rho, ur, Hz, Hr)
    m0 = -rho * ur / r
    assert h.sum() == pytest.approx(m0, rel=1e-13)
    assert (h * CZ).sum() == pytest.approx(Hz, rel=1e-12, abs=1e-18)
    assert (h * CR).sum() == pytest.approx(Hr, rel=1e-12, abs=1e-18)
    assert (h * CZ * CZ).sum() == pytest.approx(m0 / 3, rel=1e-12)
    assert (h * CZ * CR).sum() == pytest.approx(0.0, abs=1e-18)


def test_source_H_reduces_to_hoop_terms():
    """H is the difference between the cylindrical and the planar momentum
    equations (Eq. momentumcylinderical): for a rigid axial translation H = 0;
    for pure radial flow u_r = a r (d_r u_r = a) the viscous hoop term
    2 mu (d_r u_r - u_r/r)/r vanishes and only the convective -rho u_r^2/r stays."""
    Hz, Hr = core.source_H(2.5, 1.3, 0.2, 0.07, 0.0, 0.0, 0.0, 0.0, -1)
    assert Hz == 0.0 and Hr == 0.0
    a, r, rho, mu = 1e-3, 3.5, 0.8, 0.1
    Hz, Hr = core.source_H(r, rho, mu, 0.0, a * r, 0.0, 0.0, a, -1)
    assert Hz == 0.0
    assert Hr == pytest.approx(-rho * (a * r) ** 2 / r, rel=1e-13)


# --------------------------------------------------------------------- EOS --

def _fd(fn, x, h):
    return (fn(x + h) - fn(x - h)) / (2 * h)


@pytest.mark.parametrize("kind,T", [(O.EOS_VDW, 0.8), (O.EOS_CS, 0.07)])
def test_eos_derivative_matches_pressure(kind, T):
    """c_k^2 = dP_k/drho (Eq. kupershtokhspeedofsound) agrees with a central
    difference of P_k at several densities."""
    p = O.Params(eos=kind, T=T, lam=0.01)
    for rho in (0.01, 0.1, 0.3, 0.6, 1.5, 2.2):
        if kind == O.EOS_CS and rho > 0.8:
            continue
        num = _fd(lambda x: core.eos_p(p, x), rho, 1e-6 * rho)
        assert core.eos_dpdrho(p, rho) == pytest.approx(num, rel=1e-7, abs=1e-12)


def test_vdw_eos_closed_form_points():
    """Reduced vdW: P(rho=1, T=1) = lambda, the critical pressure in these units,
    and the critical point is T = 1, rho = 1."""
    p = O.Params(eos=O.EOS_VDW, T=1.0, lam=0.01)
    assert core.eos_p(p, 1.0) == pytest.approx(0.01, rel=1e-15)
    assert core.eos_dpdrho(p, 1.0) == pytest.approx(0.0, abs=1e-15)
    assert O.eos.critical_point(p) == (1.0, 1.0)


def test_cs_critical_point():
    """CS critical point: dP/drho = d2P/drho2 = 0 at (T_c, rho_c); with a = 1,
    b = 4, R = 1 the literature values are T_c ~ 0.3773 a/(b R), rho_c ~ 0.5218/b."""
    p = O.Params(eos=O.EOS_CS)
    Tc, rc = O.eos.critical_point(p)
    q = p.replace(T=Tc)
    h = 1e-4
    assert core.eos_dpdrho(q, rc) == pytest.approx(0.0, abs=1e-12)
    d2 = (core.eos_dpdrho(q, rc + h) - core.eos_dpdrho(q, rc - h)) / (2 * h)
    d2_far = (core.eos_dpdrho(q, 2 * rc + h) - core.eos_dpdrho(q, 2 * rc - h)) / (2 * h)
    assert abs(d2) < 1e-5 * abs(d2_far)
    assert Tc == pytest.approx(0.3773 / 4, rel=2e-4)
    assert rc == pytest.approx(0.5218 / 4, rel=5e-4)


@pytest.mark.parametrize("kind,TT", [(O.EOS_VDW, 0.7), (O.EOS_VDW, 0.9), (O.EOS_CS, 0.5), (O.EOS_CS, 0.8)])
def test_maxwell_equal_pressure_and_chemical_potential(kind, TT):
    """Coexistence: equal pressure and equal chemical potential,
    mu_l - mu_v = integral_{rho_v}^{rho_l} (dP/drho) / rho drho = 0, checked
    with a different quadrature (of dP/drho, not of P) than the construction uses."""
    from scipy import integrate

    p = O.make_params(8, 8, 1.0, kind, TT, lam=0.01)
    rv, rl = O.eos.maxwell_densities(p)
    assert rv < rl
    assert core.eos_p(p, rv) == pytest.approx(core.eos_p(p, rl), rel=1e-9)
    dmu, _ = integrate.quad(lambda x: core.eos_dpdrho(p, x) / x, rv, rl, points=[(rv + rl) / 2], limit=500,
                            epsabs=1e-14, epsrel=1e-12)
    scale, _ = integrate.quad(lambda x: abs(core.eos_dpdrho(p, x)) / x, rv, rl, limit=500)
    assert abs(dmu) < 1e-9 * scale


def test_vdw_coexistence_near_critical_scaling():
    """Mean-field vdW: rho_l - rho_v -> 4 sqrt(1 - T) as T -> 1."""
    p = O.Params(eos=O.EOS_VDW, T=0.9999, lam=0.01)
    rv, rl = O.eos.maxwell_densities(p)
    assert (rl - rv) / (4 * np.sqrt(1e-4)) == pytest.approx(1.0, rel=2e-3)


# ------------------------------------------------------------------ stencils --

def _poly(deg, seed):
    rng = np.random.default_rng(seed)
    coef = {(a, b): rng.uniform(-1, 1) for a in range(deg + 1) for b in range(deg + 1 - a)}

    def f(Z, R):
        return sum(c * Z**a * R**b for (a, b), c in coef.items())

    def fz(Z, R):
        return sum(c * a * Z ** (a - 1) * R**b for (a, b), c in coef.items() if a > 0)

    def fr(Z, R):
        return sum(c * b * Z**a * R ** (b - 1) for (a, b), c in coef.items() if b > 0)

    return f, fz, fr


@pytest.mark.parametrize("deg", [1, 2, 3, 4])
def test_fd_stencil_exact_on_polynomials(deg):
    """Eq. (fifthorderaccuratefinitedifference): the (8, -1)/36 stencil is exact
    for polynomials up to degree 4 (odd Taylor terms of order 3 cancel)."""
    p = O.Params(nz=9, nr=7)
    f, fz, fr = _poly(deg, deg)
    ext = core.ext_from_function(p, lambda Z, R: f(Z / 10, R / 10))
    dz, dr = core.grad(p, ext)
    Z, R = np.meshgrid(np.arange(p.nz) + 0.5, np.arange(p.nr) + 0.5)
    np.testing.assert_allclose(dz, fz(Z / 10, R / 10) / 10, rtol=0, atol=1e-13)
    np.testing.assert_allclose(dr, fr(Z / 10, R / 10) / 10, rtol=0, atol=1e-13)


def test_fd_stencil_error_on_quintic():
    """Degree 5 is the first the stencil misses: for phi = z^5 the stencil sum is
    (1/36)[24((z+1)^5 - (z-1)^5) - 3((z+2)^5 - (z-2)^5)] = 5 z^4 - 4 exactly,
    i.e. a constant error of -4 (the 5th-order Taylor term, 8 - 2^5 = -24)."""
    p = O.Params(nz=5, nr=5)
    ext = core.ext_from_function(p, lambda Z, R: Z**5)
    dz, dr = core.grad(p, ext)
    z = np.arange(p.nz) + 0.5
    for row in dz:
        np.testing.assert_allclose(row, 5 * z**4 - 4, rtol=1e-13)
    np.testing.assert_allclose(dr, 0.0, atol=1e-11)


def test_ghost_fill_parities_and_small_grids():
    """Axis mirror -1-m <-> m, top mirror nr+m <-> nr-1-m, z wrap, with the
    given signs; grids thinner than the ghost width reflect repeatedly."""
    for nr in (1, 2, 3, 7):
        p = O.Params(nz=3, nr=nr, top=O.TOP_FREESLIP)
        g = core.ghost_width()
        ext = np.zeros(core.ext_shape(p))
        inner = np.arange(1, nr * 3 + 1, dtype=float).reshape(nr, 3)
        core.interior(p, ext)[:] = inner
        core.fill_ghosts(p, ext, -1, +1)
        for j in range(-g, nr + g):
            jj, s = j, 1
            while not 0 <= jj < nr:
                if jj < 0:
                    jj, s = -1 - jj, -s
                else:
                    jj = 2 * nr - 1 - jj
            for k in range(-g, 3 + g):
                assert ext[j + g, k + g] == s * inner[jj, k % 3]


# ------------------------------------------------------------------- forces --

@pytest.mark.parametrize("A", [0.0, -0.152, 0.3])
def test_kupershtokh_linear_psi(A):
    """Eq. (kupershtokhforcing) with dt = 1: for linear psi the discrete force is
    exactly 2 psi grad psi = grad psi^2 = -grad U, for any A."""
    p = O.Params(nz=6, nr=5, A=A)
    g = np.array([0.013, -0.021])
    ext = core.ext_from_function(p, lambda Z, R: 0.4 + g[0] * Z + g[1] * R)
    fz, fr = core.force_kupershtokh(p, ext)
    psi = core.interior(p, ext)
    np.testing.assert_allclose(fz, 2 * psi * g[0], rtol=1e-13)
    np.testing.assert_allclose(fr, 2 * psi * g[1], rtol=1e-13)


@pytest.mark.parametrize("A", [0.0, -0.152, 0.25])
def test_kupershtokh_quadratic_psi(A):
    """For quadratic psi the Taylor series of the discrete force ends at third
    order; with the D2Q9 fourth-moment isotropy it is exactly
    F = 2 psi grad psi + (2A/3) (grad psi lap psi + 2 (grad grad psi) . grad psi)."""
    p = O.Params(nz=6, nr=5, A=A)
    a0, gz, gr, hzz, hzr, hrr = 0.5, 0.02, -0.015, 0.003, -0.002, 0.004

    def psi(Z, R):
        return a0 + gz * Z + gr * R + 0.5 * hzz * Z * Z + hzr * Z * R + 0.5 * hrr * R * R

    ext = core.ext_from_function(p, psi)
    fz, fr = core.force_kupershtokh(p, ext)
    Z, R = np.meshgrid(np.arange(p.nz) + 0.5, np.arange(p.nr) + 0.5)
    ps = psi(Z, R)
    dz = gz + hzz * Z + hzr * R
    dr = gr + hzr * Z + hrr * R
    lap = hzz + hrr
    ez = 2 * ps * dz + 2 * A / 3 * (dz * lap + 2 * (hzz * dz + hzr * dr))
    er = 2 * ps * dr + 2 * A / 3 * (dr * lap + 2 * (hzr * dz + hrr * dr))
    np.testing.assert_allclose(fz, ez, rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(fr, er, rtol=1e-12, atol=1e-16)


def test_force_axis_closed_form():
    """Eq. (multiphasecorrections) for psi = psi(r) only: F_axis,z = 0 and
    F_axis,r = 3 kappa [psi (psi'' / r - psi' / r^2) + 6A psi'^2 / r]; for a
    z-only psi the correction vanishes (psi_r = psi_rr = psi_rz = 0)."""
    kap, A, r = 0.11, -0.152, 4.5
    fz, fr = core.force_axis(kap, A, r, 0.6, 0.0, 0.03, -0.004, 0.0)
    assert fz == 0.0
    assert fr == pytest.approx(3 * kap * (0.6 * (-0.004 / r - 0.03 / r**2) + 6 * A * 0.03**2 / r), rel=1e-14)
    fz, fr = core.force_axis(kap, A, r, 0.6, 0.05, 0.0, 0.0, 0.0)
    assert fz == 0.0 and fr == 0.0


def test_force_axis_is_the_cylindrical_part_of_the_taylor_force():
    """F_axis is what the Taylor form (Eq. taylorexpanssion) gains when the
    planar Laplacian is replaced by the cylindrical one, lap = lap_c + (1/r) d_r:
    3 c^4 [psi grad_c(psi_r / r) + 6A grad_c psi (psi_r / r)].  Checked
    numerically for psi(z, r) = exp(-(z^2 + r^2)/s) by differentiating
    psi_r/r with finite differences."""
    s, A, kap = 30.0, -0.152, 1 / 9
    z, r = 1.3, 2.7

    def psi(z, r):
        return 0.2 + np.exp(-(z * z + r * r) / s)

    h = 1e-4
    pz = (psi(z + h, r) - psi(z - h, r)) / (2 * h)
    pr = (psi(z, r + h) - psi(z, r - h)) / (2 * h)
    q = lambda zz, rr: (psi(zz, rr + h) - psi(zz, rr - h)) / (2 * h) / rr  # psi_r / r
    dq_dz = (q(z + h, r) - q(z - h, r)) / (2 * h)
    dq_dr = (q(z, r + h) - q(z, r - h)) / (2 * h)
    ez = 3 * kap * (psi(z, r) * dq_dz + 6 * A * pz * pr / r)
    er = 3 * kap * (psi(z, r) * dq_dr + 6 * A * pr * pr / r)
    prr = (psi(z, r + h) - 2 * psi(z, r) + psi(z, r - h)) / h**2
    prz = (psi(z + h, r + h) - psi(z + h, r - h) - psi(z - h, r + h) + psi(z - h, r - h)) / (4 * h * h)
    fz, fr = core.force_axis(kap, A, r, psi(z, r), pz, pr, prr, prz)
    assert fz == pytest.approx(ez, rel=1e-5)
    assert fr == pytest.approx(er, rel=1e-5)


def test_force_axis_exact_expansion_coefficient():
    """Reading of F_axis's A-term.  The discrete force's exact expansion on D2Q9
    (pinned for quadratic psi by test_kupershtokh_quadratic_psi) is
    F = 2 psi grad psi + (1/3) psi grad lap psi + (2A/3) grad psi lap psi + (2A/3) grad |grad psi|^2;
    the paper's Eq. (taylorexpanssion) prints 2A for the third coefficient.
    For an axisymmetric psi the 3D Laplacian is the planar one plus psi_r / r,
    and |grad psi|^2 is the same, so the cylindrical correction is
    (1/3) [psi grad(psi_r / r) + 2A (psi_r / r) grad psi]: F_axis with c = 2 at
    c^4 = 1/9.  (The two forms agree in 1D, where grad psi lap psi and
    grad |grad psi|^2 / 2 coincide, and differ in 2D.)"""
    s, A, kap = 30.0, -0.152, 1 / 9
    z, r = 1.3, 2.7

    def psi(z, r):
        return 0.2 + np.exp(-(z * z + r * r) / s)

    h = 1e-4
    pz = (psi(z + h, r) - psi(z - h, r)) / (2 * h)
    pr = (psi(z, r + h) - psi(z, r - h)) / (2 * h)
    q = lambda zz, rr: (psi(zz, rr + h) - psi(zz, rr - h)) / (2 * h) / rr  # psi_r / r
    dq_dz = (q(z + h, r) - q(z - h, r)) / (2 * h)
    dq_dr = (q(z, r + h) - q(z, r - h)) / (2 * h)
    ez = (psi(z, r) * dq_dz + 2 * A * pz * pr / r) / 3
    er = (psi(z, r) * dq_dr + 2 * A * pr * pr / r) / 3
    prr = (psi(z, r + h) - 2 * psi(z, r) + psi(z, r - h)) / h**2
    prz = (psi(z + h, r + h) - psi(z + h, r - h) - psi(z - h, r + h) + psi(z - h, r - h)) / (4 * h * h)
    fz, fr = core.force_axis(kap, A, r, psi(z, r), pz, pr, prr, prz, c=2.0)
    assert fz == pytest.approx(ez, rel=1e-5)
    assert fr == pytest.approx(er, rel=1e-5)
    # the 2D expansion's third coefficient, from the discrete force itself: a quadratic
    # psi with an isotropic Hessian separates 2A/3 (exact) from the printed 2A
    p = O.Params(nz=6, nr=5, A=A)
    ext = core.ext_from_function(p, lambda Z, R: 0.5 + 0.002 * (Z * Z + R * R))
    fzd, _ = core.force_kupershtokh(p, ext)
    Z, _ = np.meshgrid(np.arange(p.nz) + 0.5, np.arange(p.nr) + 0.5)
    ps = 0.5 + 0.002 * (Z * Z + (np.arange(p.nr)[:, None] + 0.5) ** 2)
    dz, lap = 0.004 * Z, 0.008
    a_part = fzd - 2 * ps * dz  # the A-dependent remainder of the discrete force
    exact = 2 * A / 3 * (dz * lap + 2 * 0.004 * dz)
    printed = 2 * A * dz * lap
    np.testing.assert_allclose(a_part, exact, rtol=1e-9, atol=1e-15)
    assert np.max(np.abs(a_part - printed)) > 0.1 * np.max(np.abs(printed))


@pytest.mark.parametrize("mode,expect", [(O.KAPPA_LATTICE, lambda c2: 1 / 9),
                                         (O.KAPPA_THERMO, lambda c2: c2 * c2),
                                         (O.KAPPA_MIXED, lambda c2: c2 / 3)])
def test_kappa_modes(mode, expect):
    p = O.Params(eos=O.EOS_VDW, T=0.8, lam=0.01, kappa=mode)
    for rho in (0.3, 1.0, 1.9):
        c2 = core.eos_dpdrho(p, rho)
        assert core.kappa(p, rho) == pytest.approx(expect(c2), rel=1e-15)


# ----------------------------------------------------------------- streaming --

@pytest.mark.parametrize("top", [O.TOP_FREESLIP, O.TOP_NOSLIP, O.TOP_PERIODIC])
@pytest.mark.parametrize("nz,nr", [(5, 4), (1, 3), (4, 1)])
def test_stream_is_a_permutation_with_the_boundary_rules(top, nz, nr):
    """Every (node, direction) slot receives exactly one population.  Rules:
    z periodic; at the axis (mid-grid specular) c_r flips and the node stays
    in row 0; at a free-slip top c_r flips; at a no-slip top the population
    returns to its own node reversed; periodic r wraps."""
    p = O.Params(nz=nz, nr=nr, top=top)
    seen = set()
    for i in range(9):
        for j in range(nr):
            for k in range(nz):
                kd, jd, idd = core.stream_dest(p, k, j, i)
                seen.add((kd, jd, idd))
                jj = j + CR[i]
                if 0 <= jj < nr or top == O.TOP_PERIODIC:
                    assert (kd, jd, idd) == ((k + CZ[i]) % nz, jj % nr, i)
                elif jj < 0:
                    assert (jd, CZ[idd], CR[idd]) == (0, CZ[i], -CR[i]) and kd == (k + CZ[i]) % nz
                elif top == O.TOP_FREESLIP:
                    assert (jd, CZ[idd], CR[idd]) == (nr - 1, CZ[i], -CR[i]) and kd == (k + CZ[i]) % nz
                else:
                    assert (kd, jd, CZ[idd], CR[idd]) == (k, j, -CZ[i], -CR[i])
    assert len(seen) == 9 * nz * nr


@pytest.mark.parametrize("seed", [5, 6])
def test_guo_source_moments(seed):
    """Guo forcing (Sec. II.A, second term read as (c_i.u)(c_i.F)/c_s^4): the
    source adds no mass, momentum (1 - 1/(2 tau)) F and second moment
    (1 - 1/(2 tau)) (u F + F u).  The printed (c_i - u).(c_i - F) term would
    put mass into the source and break the first of these."""
    rng = np.random.default_rng(seed)
    _, cz, cr = _lattice_from_feq()
    tau = rng.uniform(0.55, 2.0)
    uz, ur, Fz, Fr = rng.uniform(-0.1, 0.1, size=4)
    S = core.guo_source(tau, uz, ur, Fz, Fr)
    pre = 1 - 1 / (2 * tau)
    assert abs(S.sum()) < 1e-16
    assert (S * cz).sum() == pytest.approx(pre * Fz, rel=1e-13)
    assert (S * cr).sum() == pytest.approx(pre * Fr, rel=1e-13)
    assert (S * cz * cz).sum() == pytest.approx(pre * 2 * uz * Fz, rel=1e-12, abs=1e-17)
    assert (S * cr * cr).sum() == pytest.approx(pre * 2 * ur * Fr, rel=1e-12, abs=1e-17)
    assert (S * cz * cr).sum() == pytest.approx(pre * (uz * Fr + ur * Fz), rel=1e-12, abs=1e-17)


def _collision_moments(forcing, seed):
    """One collision of a multiphase state (plane mode, no h_i): per node the
    moments of f* - f, the pre-collision moments and the force F."""
    from paper_1512_01977_gb300 import inputs as I

    p = O.make_params(24, 20, 0.8, O.EOS_CS, 0.85, top=O.TOP_PERIODIC, axis=0, forcing=forcing)
    rv, rl = O.eos.maxwell_densities(p)
    rho, uz, ur = I.droplet_2d(24, 20, 6, rl, rv)
    _, vz, vr = I.random_state(24, 20, 1.0, 0.0, 2e-3, seed)
    o = O.Oracle(p).init(rho, vz, vr)
    d = o.moments(diagnostics=True)
    post = o.collide_only()
    _, cz, cr = _lattice_from_feq()
    c = [np.ones(9), cz, cr]
    dm = [[np.tensordot(a * b, post - o.f, axes=(0, 0)) for b in c] for a in c]
    m = [[np.tensordot(a * b, o.f, axes=(0, 0)) for b in c] for a in c]
    return p, d, dm, m


@pytest.mark.parametrize("forcing", [O.FORCING_EDM, O.FORCING_GUO])
def test_collision_moments_with_force(forcing):
    """Per node, one collision with either forcing keeps the mass and adds F
    to the momentum (both schemes give the fluid velocity u = u0 + F/(2 rho)).
    Second moment: EDM, Pi* = Pi + (Pi_eq(u0) - Pi)/tau + rho (u1 u1 - u0 u0),
    u1 = u0 + F/rho (the equilibrium shift of Sec. II.C); Guo,
    Pi* = Pi + (Pi_eq(u) - Pi)/tau + (1 - 1/(2 tau)) (u F + F u)."""
    p, d, dm, m = _collision_moments(forcing, 3)
    rho, jz, jr = m[0][0], m[0][1], m[0][2]
    Fz, Fr = d["Fz"], d["Fr"]
    assert np.max(np.abs(Fz)) > 1e-4  # the interface carries a real force
    assert np.max(np.abs(dm[0][0])) < 1e-15
    np.testing.assert_allclose(dm[0][1], Fz, rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(dm[0][2], Fr, rtol=1e-11, atol=1e-15)
    tau = p.tau
    if forcing == O.FORCING_EDM:
        vz, vr = jz / rho, jr / rho
        wz, wr = vz + Fz / rho, vr + Fr / rho
        extra = lambda a, b: rho * (a[1] * b[1] - a[0] * b[0])  # noqa: E731
        shift = {(1, 1): extra((vz, wz), (vz, wz)), (2, 2): extra((vr, wr), (vr, wr)),
                 (1, 2): extra((vz, wz), (vr, wr))}
    else:
        vz, vr = (jz + Fz / 2) / rho, (jr + Fr / 2) / rho
        pre = 1 - 1 / (2 * tau)
        shift = {(1, 1): pre * 2 * vz * Fz, (2, 2): pre * 2 * vr * Fr, (1, 2): pre * (vz * Fr + vr * Fz)}
    ueq = {1: vz, 2: vr}
    for (a, b), s in shift.items():
        pi_eq = rho * ueq[a] * ueq[b] + (rho / 3 if a == b else 0.0)
        expect = (pi_eq - m[a][b]) / tau + s
        np.testing.assert_allclose(dm[a][b], expect, rtol=1e-9, atol=1e-14)
