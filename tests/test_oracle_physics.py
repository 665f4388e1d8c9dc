"""Pins of the whole oracle update against textbook special cases, closed-form
flows, the paper's own validation laws and exact discrete invariants.

Readings these pins decide (each would fail under the alternative):
* H_r carries -u_r/r (the radial acoustic mode test; the printed +u_r/r is
  unstable), i.e. the viscous hoop term 2 mu d_r(u_r / r) of the target
  momentum equation.
* H_z's viscous hoop term (Hagen-Poiseuille; without it the profile is the
  planar one, twice as fast).
* the Kupershtokh force with A = -0.152 reproduces the vdW coexistence curve.
"""
import numpy as np
import pytest
from scipy import special

import oracle as O
from paper_1512_01977_gb300 import inputs as I

CZ = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CR = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _textbook_bgk(f, tau):
    """Plain periodic D2Q9 BGK (no force, no source) with np.roll streaming."""
    W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    rho = f.sum(0)
    uz = (f * CZ[:, None, None]).sum(0) / rho
    ur = (f * CR[:, None, None]).sum(0) / rho
    cu = CZ[:, None, None] * uz + CR[:, None, None] * ur
    feq = W[:, None, None] * rho * (1 + 3 * cu + 4.5 * cu**2 - 1.5 * (uz**2 + ur**2))
    post = f + (feq - f) / tau
    return np.stack([np.roll(np.roll(post[i], CZ[i], axis=1), CR[i], axis=0) for i in range(9)])


def test_reduces_to_textbook_bgk():
    """Force, axisymmetric terms off and periodic walls: one step of the oracle
    is one step of plain D2Q9 BGK."""
    p = O.Params(nz=12, nr=10, tau=0.7, multiphase=0, axis=0, top=O.TOP_PERIODIC)
    rng = np.random.default_rng(7)
    o = O.Oracle(p).init(*I.random_state(12, 10, 1.0, 0.05, 0.05, 11))
    o.f += rng.uniform(-1e-3, 1e-3, size=o.f.shape) * o.f
    expect = _textbook_bgk(o.f.copy(), p.tau)
    o.step(1)
    np.testing.assert_allclose(o.f, expect, rtol=1e-14, atol=1e-16)


def _fit(series):
    t = np.arange(len(series))
    return O.analytic.fit_damped_cosine(t, np.array(series))


def test_shear_wave_decay():
    """u_z = U sin(k r) in a periodic box decays as exp(-nu k^2 t), nu = (tau - 1/2)/3."""
    nr, tau, U = 32, 0.9, 1e-4
    p = O.Params(nz=1, nr=nr, tau=tau, multiphase=0, axis=0, top=O.TOP_PERIODIC)
    o = O.Oracle(p).init(*I.shear_wave(1, nr, 1.0, U))
    k = 2 * np.pi / nr
    a0 = o.moments()["uz"][:, 0] @ np.sin(k * (np.arange(nr) + 0.5))
    o.step(400)
    a1 = o.moments()["uz"][:, 0] @ np.sin(k * (np.arange(nr) + 0.5))
    rate = -np.log(a1 / a0) / 400
    assert rate == pytest.approx((tau - 0.5) / 3 * k * k, rel=5e-3)


def test_plane_sound_wave():
    """Planar acoustic wave: angular frequency c_s k and amplitude decay nu k^2."""
    nz, tau = 64, 0.8
    p = O.Params(nz=nz, nr=1, tau=tau, multiphase=0, axis=0, top=O.TOP_PERIODIC)
    k = 2 * np.pi / nz
    Z, _ = I.grid(nz, 1)
    o = O.Oracle(p).init(1.0 + 1e-4 * np.cos(k * Z))
    ys = []
    for _ in range(600):
        ys.append(o.moments()["rho"][0, 0])
        o.step(1)
    w, c = _fit(ys)
    assert w == pytest.approx(k / np.sqrt(3), rel=2e-3)
    assert c == pytest.approx((tau - 0.5) / 3 * k * k, rel=3e-2)


def _radial_mode(hr_sign, top, steps=600, h_eval=O.H_LOCAL):
    nr, tau = 64, 0.8
    k = special.jn_zeros(1, 1)[0] / nr  # J1(k R) = 0: u_r = 0 at the wall r = R
    p = O.Params(nz=1, nr=nr, tau=tau, multiphase=0, axis=1, hr_sign=hr_sign, top=top, h_eval=h_eval)
    o = O.Oracle(p).init(*I.radial_mode(1, nr, 1.0, 1e-4, k))
    ys = []
    for _ in range(steps):
        ys.append(o.moments()["rho"][0, 0])
        o.step(1)
    w, c = _fit(ys)
    return w / (k / np.sqrt(3)), c / ((tau - 0.5) / 3 * k * k)


@pytest.mark.parametrize("top", [O.TOP_FREESLIP, O.TOP_NOSLIP])
def test_radial_acoustic_mode(top):
    """Axisymmetric source terms (mass sink + H): the standing mode
    rho = rho0 (1 + e J0(k r)) of a cylinder oscillates at c_s k and decays at
    nu k^2, exactly like the planar wave with the same k (irrotational flow:
    the vector Laplacian equals grad div in both geometries)."""
    w, c = _radial_mode(-1, top)
    assert w == pytest.approx(1.0, abs=2e-3)
    assert c == pytest.approx(1.0, abs=3e-2)


@pytest.mark.parametrize("top", [O.TOP_FREESLIP, O.TOP_NOSLIP])
def test_link_averaged_source_misses_acoustic_damping(top):
    """h_i averaged over the two ends of its link at time t keeps the
    frequency but not the damping of the same mode (about 0.7 nu k^2): the
    half-link shift adds (1/2) c_i . grad h_i, whose moments (1/2) div H and
    (1/2) c_s^2 grad(-rho u_r / r) are of the viscous order, with no matching
    (1/2) d_t h_i.  This is why h_i is evaluated at the node by default."""
    w, c = _radial_mode(-1, top, h_eval=O.H_LINK_AVG)
    assert w == pytest.approx(1.0, abs=2e-3)
    assert c < 0.8


def test_radial_mode_rejects_printed_hr_sign():
    """With +u_r/r inside H_r (as printed) the same mode is unstable or wrong."""
    try:
        w, c = _radial_mode(+1, O.TOP_FREESLIP, steps=400)
    except O.OracleError:
        return
    assert abs(w - 1) > 0.05 or abs(c - 1) > 0.5


@pytest.mark.parametrize("h_eval", [O.H_LOCAL, O.H_LINK_AVG])
def test_hagen_poiseuille(h_eval):
    """Pipe flow driven by a body acceleration g (top = no-slip wall at r = nr):
    u_z(r) = g (R^2 - r^2) / (4 nu).  Without H_z the profile would be the
    planar g (R^2 - r^2) / (2 nu)."""
    nr, tau, g = 16, 1.0, 1e-6
    p = O.Params(nz=2, nr=nr, tau=tau, multiphase=0, axis=1, top=O.TOP_NOSLIP, gz=g, h_eval=h_eval)
    o = O.Oracle(p).init(*I.uniform(2, nr, 1.0))
    o.step(6000)
    uz = o.moments()["uz"][:, 0]
    r = np.arange(nr) + 0.5
    nu = (tau - 0.5) / 3
    ua = O.analytic.hagen_poiseuille(g, nr, nu, r)
    assert np.max(np.abs(uz - ua)) < 3e-3 * ua.max()
    assert np.max(np.abs(uz - O.analytic.plane_poiseuille(g, nr, nu, r))) > 0.3 * ua.max()


def test_radial_density_wave_bessel():
    """Sec. III.C (Eq. analyticdensityprop): a ring-shaped density bump in a
    1 x 2000 channel (vdW, lambda = 0.01, T = 0.8, rho0 = 1.8, A = 0, tau = 0.6)
    splits into waves towards and away from the axis that follow the Bessel
    series of the inviscid cylindrical wave equation.  The bump's width and
    amplitude are not printed; w_d = 20 and rho_p = 1e-3 rho0 are used."""
    nr, rho0, wd = 2000, 1.8, 20.0
    rp = 1e-3 * rho0
    p = O.Params(nz=1, nr=nr, tau=0.6, A=0.0, eos=O.EOS_VDW, T=0.8, lam=0.01, axis=1, top=O.TOP_NOSLIP)
    ck = np.sqrt(O.eos.sound_speed_sq(p, rho0))
    o = O.Oracle(p).init(*I.radial_bump(1, nr, rho0, rp, wd))
    m0 = o.mass_rweighted()
    r = np.arange(nr) + 0.5
    done = 0
    sel = slice(800, 1200)  # the analytic series is evaluated where the waves are
    for tw in (1.0, 2.0, 3.0):
        steps = int(round(tw * wd / ck))
        o.step(steps - done)
        done = steps
        rho1 = o.moments()["rho"][:, 0] - rho0
        ana = O.analytic.bessel_wave(lambda x: rp * np.exp(-(((x - nr / 2) / wd) ** 2)), nr, ck, steps, r[sel],
                                     n_terms=400)
        assert np.max(np.abs(rho1[sel] - ana)) < 0.06 * rp
        assert np.max(np.abs(rho1[:800])) < 1e-3 * rp and np.max(np.abs(rho1[1200:])) < 1e-3 * rp
    # the waves have not reached the walls: r-weighted mass is conserved
    assert o.mass_rweighted() == pytest.approx(m0, rel=1e-12)


@pytest.mark.parametrize("T", [0.7, 0.8, 0.9])
def test_vdw_coexistence_with_kupershtokh_A(T):
    """Sec. II.C / Fig. 2: with A = -0.152 the flat-interface densities follow
    the vdW coexistence curve (Maxwell construction); with A = 0 the vapour
    density is visibly off."""
    nz = 128

    def run(A):
        p = O.make_params(nz, 1, 1.0, O.EOS_VDW, T, A=A, lam=0.01, top=O.TOP_PERIODIC, axis=0)
        rv, rl = O.eos.maxwell_densities(p)
        o = O.Oracle(p).init(*I.slab(nz, 1, rl, rv))
        o.step(12000)
        rho = o.moments()["rho"][0]
        return rho[nz // 2] / rl - 1, rho[0] / rv - 1

    el, ev = run(-0.152)
    assert abs(el) < 3e-3 and abs(ev) < 3e-3
    el0, ev0 = run(0.0)
    assert abs(ev0) > 1e-2


def test_cs_coexistence_liquid_branch():
    """CS (not in the paper; A = -0.152 is tuned for vdW): the liquid branch
    still matches Maxwell within 0.2 %; the vapour branch is only loosely
    pinned (measured 1.5 % at T = 0.9 Tc, 5 % at 0.8 Tc)."""
    nz = 128
    for T, vap_tol in ((0.9, 0.03), (0.8, 0.08)):
        p = O.make_params(nz, 1, 1.0, O.EOS_CS, T, top=O.TOP_PERIODIC, axis=0)
        rv, rl = O.eos.maxwell_densities(p)
        o = O.Oracle(p).init(*I.slab(nz, 1, rl, rv))
        o.step(5000)
        rho = o.moments()["rho"][0]
        assert abs(rho[nz // 2] / rl - 1) < 2e-3
        assert abs(rho[0] / rv - 1) < vap_tol


def _droplet_oracle(T=0.8, R0=12, nz=48, nr=32, kappa=O.KAPPA_THERMO, h_eval=O.H_LOCAL, physical=False):
    p = O.make_params(nz, nr, 1.0, O.EOS_CS, T, kappa=kappa, top=O.TOP_FREESLIP, axis=1, h_eval=h_eval)
    rv, rl = O.eos.maxwell_densities(p)
    return O.Oracle(p).init(*I.droplet(nz, nr, R0, rl, rv), physical=physical), rv, rl


@pytest.mark.parametrize("h_eval", [O.H_LOCAL, O.H_LINK_AVG])
def test_rweighted_mass_budget_identity(h_eval):
    """Exact discrete budget of one step: with r_j = j + 1/2,
    M_r(t+1) - M_r(t) = sum_x [F_r/2 + H_r] + sum_{j=0, c_r=-1} f*_i - sum_{j=nr-1, c_r=+1} f*_i,
    because the collision keeps mass, the source's zeroth and first moments
    are -rho u_r / r and H, and streaming moves f*_i by c_ir except where the
    axis or the free-slip top reflects it.  With h_i at the link midpoint the
    departure half brings -rho u_r / (2r) and H/2, and the arrival half adds
    -rho u_r / (2r) at the arrival node, so H_r/2 replaces H_r."""
    o, _, _ = _droplet_oracle(h_eval=h_eval, physical=True)
    o.step(30)
    d = o.moments(diagnostics=True)
    post = o.collide_only()
    m0 = o.mass_rweighted()
    budget = np.sum(d["Fr"] / 2 + (0.5 if h_eval == O.H_LINK_AVG else 1.0) * d["Hr"])
    budget += post[CR == -1][:, 0, :].sum() - post[CR == 1][:, -1, :].sum()
    o.step(1)
    assert o.mass_rweighted() - m0 == pytest.approx(budget, rel=1e-9, abs=1e-13 * m0)


def test_mass_exact_in_plane_mode():
    """Axis terms off, periodic: sum rho is conserved to round-off (EDM and BGK
    conserve mass, streaming is a permutation)."""
    p = O.make_params(40, 40, 1.0, O.EOS_CS, 0.8, top=O.TOP_PERIODIC, axis=0)
    rv, rl = O.eos.maxwell_densities(p)
    o = O.Oracle(p).init(*I.droplet_2d(40, 40, 10, rl, rv))
    m0 = o.mass()
    o.step(200)
    assert o.mass() == pytest.approx(m0, rel=1e-13)


def test_droplet_keeps_z_mirror_symmetry():
    """A droplet centred at z = nz/2 stays mirror-symmetric in z; a mixed-up
    z/r index or a wrong sign of c_z in any stencil breaks this."""
    o, _, _ = _droplet_oracle()
    o.step(200)
    m = o.moments()
    np.testing.assert_allclose(m["rho"], m["rho"][:, ::-1], rtol=1e-11)
    np.testing.assert_allclose(m["uz"], -m["uz"][:, ::-1], atol=1e-13)
    np.testing.assert_allclose(m["ur"], m["ur"][:, ::-1], atol=1e-13)


def _laplace(m, rv, rl, R_guess, axis, zc, rc=0.0):
    nr, nz = m["rho"].shape
    Z, Rr = I.grid(nz, nr)
    if axis:
        r = np.arange(nr) + 0.5
        V = 2 * np.pi * np.sum(r[:, None] * (m["rho"] - rv) / (rl - rv))
        R = (3 * V / (4 * np.pi)) ** (1 / 3)
    else:
        R = np.sqrt(np.sum((m["rho"] - rv) / (rl - rv)) / np.pi)
    d = np.sqrt((Z - zc) ** 2 + (Rr - rc) ** 2)
    return R, m["p"][d < R / 2].mean() - m["p"][d > R + 8].mean()


@pytest.mark.slow
def test_young_laplace_sphere_lattice_kappa():
    """Young-Laplace for a sphere (dp = 2 sigma / R) against the planar droplet
    (dp = sigma / R) of the same fluid: with F_axis at the lattice c_s^4 the
    two surface tensions agree within 10 % (CS, T = 0.8 Tc, R = 16)."""
    p = O.make_params(64, 48, 1.0, O.EOS_CS, 0.8, kappa=O.KAPPA_LATTICE, top=O.TOP_FREESLIP, axis=1)
    rv, rl = O.eos.maxwell_densities(p)
    o = O.Oracle(p).init(*I.droplet(64, 48, 16, rl, rv))
    o.step(3000)
    R, dp = _laplace(o.moments(), rv, rl, 16, True, 32)
    sig_axis = dp * R / 2
    q = O.make_params(64, 64, 1.0, O.EOS_CS, 0.8, top=O.TOP_PERIODIC, axis=0)
    o2 = O.Oracle(q).init(*I.droplet_2d(64, 64, 16, rl, rv))
    o2.step(3000)
    R2, dp2 = _laplace(o2.moments(), rv, rl, 16, False, 32, 32)
    sig_2d = dp2 * R2
    assert sig_axis == pytest.approx(sig_2d, rel=0.10)
    # without F_axis the axisymmetric droplet would show the planar jump sigma/R
    assert dp * R > 1.6 * sig_2d


@pytest.mark.slow
def test_table1_axis_matches_2d_with_ck_substitution():
    """Table 1 (vdW, lambda = 0.01, T = 0.8, A = 0, tau = 1.5): with the paper's
    c_s -> c_k substitution in F_axis, sigma from the printed law dp = sigma/R
    agrees between the axisymmetric and the fully periodic 2D droplet within the
    paper's 3.2 % (here at R0 = 16 instead of 150)."""
    R0 = 16
    p = O.make_params(4 * R0, 2 * R0, 1.5, O.EOS_VDW, 0.8, A=0.0, lam=0.01, kappa=O.KAPPA_THERMO,
                      top=O.TOP_FREESLIP, axis=1)
    rv, rl = O.eos.maxwell_densities(p)
    o = O.Oracle(p).init(*I.droplet(4 * R0, 2 * R0, R0, rl, rv, width=8.0))
    o.step(4000)
    R, dp = _laplace(o.moments(), rv, rl, R0, True, 2 * R0)
    q = O.make_params(4 * R0, 4 * R0, 1.5, O.EOS_VDW, 0.8, A=0.0, lam=0.01, top=O.TOP_PERIODIC, axis=0)
    o2 = O.Oracle(q).init(*I.droplet_2d(4 * R0, 4 * R0, R0, rl, rv, width=8.0))
    o2.step(4000)
    R2, dp2 = _laplace(o2.moments(), rv, rl, R0, False, 2 * R0, 2 * R0)
    assert dp * R == pytest.approx(dp2 * R2, rel=0.032)


def test_damped_cosine_fit_recovers_frequency_over_a_drift():
    """The oscillation-period fit: a known damped cosine on a linearly
    drifting mean, sampled over about one period, gives back its frequency
    and decay rate (the zero-crossing start alone locks onto the drift)."""
    t = np.arange(0, 12000, 100.0)
    w, c = 8.4e-4, 4.0e-4
    y = 120 + 7 * np.exp(-c * t) * np.cos(w * t + 0.3) - 2e-4 * t
    wf, cf = O.analytic.fit_damped_cosine(t, y, w_guess=1.1 * w)
    assert wf == pytest.approx(w, rel=1e-6) and cf == pytest.approx(c, rel=1e-5)
    wf, _ = O.analytic.fit_damped_cosine(t, y + 1e-3 * np.sin(0.37 * t))
    assert wf == pytest.approx(w, rel=1e-3)


def test_init_physical_is_plain_init_for_uniform_density():
    """A uniform density exerts no force (every stencil sum of a constant psi
    cancels), so starting with a physical velocity is starting with that bare
    velocity -- up to the rounding of rho = sum_i f_i^eq(rho, u), which leaves
    psi constant only to an ulp."""
    nz, nr = 24, 12
    p = O.make_params(nz, nr, 0.8, O.EOS_VDW, 0.8)
    rho = np.full((nr, nz), 1.3)
    _, uz, ur = I.random_state(nz, nr, 1.0, 0.0, 0.03, 5)
    a = O.Oracle(p).init(rho, uz, ur)
    b = O.Oracle(p).init(rho, uz, ur, physical=True)
    np.testing.assert_allclose(b.f, a.f, rtol=1e-14, atol=0)


def test_init_physical_starts_a_droplet_at_rest():
    """With physical=True and u = 0 the fluid velocity u0 + F/(2 rho) of the
    first state vanishes (Sec. II.A), while the bare start leaves F/(2 rho),
    of order 1e-2 in the interface."""
    nz, nr = 64, 32
    p = O.make_params(nz, nr, 0.7, O.EOS_VDW, 0.8, A=0.0)
    rv, rl = O.eos.maxwell_densities(p)
    rho, _, _ = I.droplet(nz, nr, 12, rl, rv)
    m = O.Oracle(p).init(rho, physical=True).moments()
    assert np.abs(m["uz"]).max() < 1e-14 and np.abs(m["ur"]).max() < 1e-14
    mb = O.Oracle(p).init(rho).moments()
    assert np.hypot(mb["uz"], mb["ur"]).max() > 1e-3


def test_oscillation_settings_run_from_rest():
    """The oscillating-droplet settings of Sec. III (vdW, T = 0.8 T_c, A = 0,
    tau = 0.7, density ratio about 10): started at rest the droplet relaxes
    with spurious currents below 1e-2; started from the bare velocity, the
    force F/(2 rho) of the sharp initial interface feeds the mass source
    -rho u_r / r and the run goes unphysical within a few hundred steps."""
    nz, nr = 160, 80
    p = O.make_params(nz, nr, 0.7, O.EOS_VDW, 0.8, A=0.0)
    rv, rl = O.eos.maxwell_densities(p)
    rho, _, _ = I.droplet(nz, nr, 32, rl, rv)
    o = O.Oracle(p).init(rho, physical=True).step(600)
    m = o.moments()
    assert np.hypot(m["uz"], m["ur"]).max() < 1e-2
    with pytest.raises(O.OracleError):
        O.Oracle(p).init(rho).step(600)
