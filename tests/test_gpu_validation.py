"""The GPU path against the physics of Sec. III at the paper's scale.

* Table 1: surface tension from the printed Young-Laplace law, Eq.
  (laplacepressure), for an axisymmetric droplet and a fully periodic 2D
  droplet (vdW, lambda = 0.01, R0 = 150, 500 x 200, tau = 1.5).
* Young-Laplace for a sphere, dp = 2 sigma / R, over several radii.
* The mode-2 oscillation of an ellipsoidal drop against the Miller-Scriven
  frequency, Eq. (oscillatingfreq), for both readings of the c^4 factor of
  F_axis, and its FP32 period error.
* The radial density wave of Sec. III.C (1 x 2000, no-slip top) against the
  Bessel series, Eq. (analyticdensityprop), in FP32, and against the oracle.
* Fig. 2: flat-interface coexistence densities against the vdW Maxwell
  construction for A = -0.152 and A = 0 (150 x 100, tau = 1).

Every test prints what it measured; the bars are stated in each test.
"""
import numpy as np
import pytest

import oracle as O
from paper_1512_01977_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LAM = 0.01


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_01977_gb300 import build, lbm as L

    build.build()
    L.lib()
    return L


def _axis_state(rho):
    """Equal-volume radius of an axisymmetric droplet centred on the axis,
    with its inner (axis, centre) and outer (top corner) densities."""
    nr, nz = rho.shape
    rl, rv = rho[0, nz // 2], rho[-1, 0]
    r = np.arange(nr) + 0.5
    V = 2 * np.pi * np.sum(r[:, None] * (rho - rv) / (rl - rv))
    return (3 * V / (4 * np.pi)) ** (1 / 3), rl, rv


def _plane_state(rho):
    n = rho.shape[0]
    rl, rv = rho[n // 2, rho.shape[1] // 2], rho[0, 0]
    return np.sqrt(np.sum((rho - rv) / (rl - rv)) / np.pi), rl, rv


def _half_extent(row, rl, rv):
    """Half the distance between the two crossings of (rho_l + rho_v)/2 on
    the axis row (linear interpolation); nan if the liquid touches an end."""
    mid = 0.5 * (rl + rv)
    z = np.arange(len(row)) + 0.5
    idx = np.nonzero(row > mid)[0]
    if len(idx) == 0 or idx[0] == 0 or idx[-1] >= len(row) - 1:
        return float("nan")
    i0, i1 = idx[0], idx[-1]
    zh = z[i1] + (mid - row[i1]) / (row[i1 + 1] - row[i1])
    zl = z[i0 - 1] + (mid - row[i0 - 1]) / (row[i0] - row[i0 - 1])
    return 0.5 * (zh - zl)


# ------------------------------------------------------------- Table 1 --

# Table 1 (sigma / lambda): (T, A) -> (2D, axis)
TABLE1 = {(0.9, 0.0): (0.305, 0.304), (0.8, 0.0): (0.928, 0.928), (0.7, 0.0): (1.983, 2.009),
          (0.9, -0.152): (0.371, 0.383), (0.8, -0.152): (1.146, 1.158), (0.7, -0.152): (2.285, 2.318)}


def _laplace_printed(lbm, T, A, axis, steps=100000, R0=150):
    """sigma / lambda = dp R / lambda (printed law) after `steps` steps, FP32,
    with the outer average taken beyond R + 8 and beyond R + 24."""
    eos = lbm.make_eos(lbm.EOS_VDW, T, lam=LAM)
    rv, rl = lbm.lbm_eos_coexistence(eos)
    if axis:
        nz, nr = 500, 200
        s = lbm.Solver(nz, nr, 1.5, eos=eos, A=A, precision=32, rho_ref=rv)
        s.init(*I.droplet(nz, nr, R0, rl, rv, width=8.0), physical=True)
    else:
        nz = nr = 500
        s = lbm.Solver(nz, nr, 1.5, eos=eos, A=A, precision=32, rho_ref=rv, top=lbm.TOP_PERIODIC, axis=0)
        s.init(*I.droplet_2d(nz, nr, R0, rl, rv, width=8.0), physical=True)
    s.step(steps)
    rho = s.moments()["rho"]
    R, _, _ = _axis_state(rho) if axis else _plane_state(rho)
    rc = 0.0 if axis else nr / 2
    out = [s.pressure_jump(nz / 2, rc, R / 2, R + gap) * R / LAM for gap in (8, 24)]
    s.close()
    return R, out


@pytest.mark.parametrize("A", [0.0, -0.152])
@pytest.mark.parametrize("T", [0.7, 0.8, 0.9])
def test_table1_axis_vs_2d(lbm, T, A):
    """Table 1's comparison at its own scale: with the paper's c_s -> c_k
    substitution in F_axis (default), sigma from the printed law agrees
    between the axisymmetric and the 2D droplet within the paper's 3.2 %.
    The vapour average is taken beyond R + 24: at 0.9 T_c the interface is
    wide enough that a shell at R + 8 still sits in its tail (ratio about
    0.89 there).  The absolute values come out 1.5-1.9 times Table 1's."""
    Ra, sa = _laplace_printed(lbm, T, A, True)
    R2, s2 = _laplace_printed(lbm, T, A, False)
    p2d, pax = TABLE1[(T, A)]
    print("Table 1 T %.1f A %+.3f: axis R %.2f sigma/lam %.4f (R+24: %.4f) | 2D R %.2f sigma/lam %.4f (R+24: %.4f) | "
          "ratio %.4f (R+24: %.4f) | paper 2D %.3f axis %.3f" % (T, A, Ra, sa[0], sa[1], R2, s2[0], s2[1],
                                                                   sa[0] / s2[0], sa[1] / s2[1], p2d, pax))
    assert sa[1] / s2[1] == pytest.approx(1.0, abs=0.032)


# ---------------------------------------------------- Young-Laplace (1/R) --

def test_young_laplace_sphere_over_radii(lbm):
    """dp = 2 sigma / R for axisymmetric droplets of radius 32 .. 64 (CS,
    T = 0.8 T_c, tau = 1, c_s^4 in F_axis): dp R is the same for every
    radius within 6 %, and sigma = dp R / 2 is the planar droplet's within
    10 %.  (A drop of radius 24 in its box evaporates into the vapour.)"""
    eos = lbm.make_eos(lbm.EOS_CS, 0.8)
    rv, rl = lbm.lbm_eos_coexistence(eos)
    s = lbm.Solver(256, 256, 1.0, eos=eos, A=-0.152, precision=64, top=lbm.TOP_PERIODIC, axis=0)
    s.init(*I.droplet_2d(256, 256, 48, rl, rv), physical=True)
    s.step(20000)
    R2, _, _ = _plane_state(s.moments()["rho"])
    sig2d = s.pressure_jump(128, 128, R2 / 2, R2 + 12) * R2
    s.close()
    sig = []
    for R0 in (32, 40, 48, 64):
        nz, nr = 4 * R0 + 64, 2 * R0 + 48
        s = lbm.Solver(nz, nr, 1.0, eos=eos, A=-0.152, precision=64, kappa=lbm.KAPPA_LATTICE)
        s.init(*I.droplet(nz, nr, R0, rl, rv), physical=True)
        s.step(20000)
        R, _, _ = _axis_state(s.moments()["rho"])
        sig.append(s.pressure_jump(nz / 2, 0, R / 2, R + 12) * R / 2)
        s.close()
    print("Young-Laplace sphere: sigma(R) =", np.round(sig, 6).tolist(), "sigma_2D = %.6f" % sig2d)
    assert max(sig) / min(sig) < 1.06
    for x in sig:
        assert x == pytest.approx(sig2d, rel=0.10)


# ----------------------------------------------------- mode-2 oscillation --

def _oscillation(lbm, kappa, precision=64, shape=(62, 76), steps=25000, every=100, forcing=0, axis_a_term=0):
    """Mode-2 frequency of an ellipsoidal drop (CS, T = 0.8 T_c, A = -0.152,
    tau = 1, 500 x 250, free-slip top) and the Miller-Scriven value for its
    measured radius and densities, with sigma from a planar droplet."""
    nz, nr, tau, A = 500, 250, 1.0, -0.152
    eos = lbm.make_eos(lbm.EOS_CS, 0.8)
    rv0, rl0 = lbm.lbm_eos_coexistence(eos)
    # planar droplet: sigma of the scheme (no F_axis, so the same for both kappa readings)
    s = lbm.Solver(320, 320, tau, eos=eos, A=A, precision=64, top=lbm.TOP_PERIODIC, axis=0, forcing=forcing)
    s.init(*I.droplet_2d(320, 320, 64, rl0, rv0), physical=True)
    s.step(30000)
    R2, _, _ = _plane_state(s.moments()["rho"])
    sig2d = s.pressure_jump(160, 160, R2 / 2, R2 + 12) * R2
    s.close()
    # the spherical drop of the same volume at rest: its equilibrium radius and densities
    Ra, Rz = shape
    R0 = (Ra * Ra * Rz) ** (1 / 3)
    s = lbm.Solver(nz, nr, tau, eos=eos, A=A, precision=64, kappa=kappa, forcing=forcing, axis_a_term=axis_a_term)
    s.init(*I.droplet(nz, nr, R0, rl0, rv0), physical=True)
    s.step(20000)
    Rs, rl, rv = _axis_state(s.moments()["rho"])
    s.close()
    # the ellipsoid, scaled to that radius, at rest
    k = Rs / R0
    s = lbm.Solver(nz, nr, tau, eos=eos, A=A, precision=precision, kappa=kappa,
                   rho_ref=rv if precision == 32 else 0.0, forcing=forcing, axis_a_term=axis_a_term)
    s.init(*I.ellipsoid(nz, nr, Ra * k, Rz * k, rl, rv), physical=True)
    m_start = s.mass()[0]
    ts, ext, rad, dens = [], [], [], []
    for i in range(steps // every):
        rho = lbm.lbm_axi_moments(s.h, nz, nr, want=("rho",))["rho"]
        R, a, b = _axis_state(rho)
        ts.append(i * every)
        ext.append(_half_extent(rho[0], a, b))
        rad.append(R)
        dens.append((a, b))
        s.step(every)
    drift = s.mass()[0] / m_start - 1
    s.close()
    ts, ext = np.array(ts[3:]), np.array(ext[3:])
    Rm = float(np.mean(rad[3:]))
    rlm, rvm = np.mean([d[0] for d in dens[3:]]), np.mean([d[1] for d in dens[3:]])
    nu = (tau - 0.5) / 3
    w_ms = O.analytic.miller_scriven_omega2(sig2d, Rm, rlm, rvm, nu, nu)
    w, c = O.analytic.fit_damped_cosine(ts, ext, w_guess=w_ms)
    return dict(omega=w, decay=c, omega_ms=w_ms, err=w / w_ms - 1, R=Rm, sigma_2d=sig2d, mass_drift=drift,
                ext=ext, rho_l=rlm, rho_v=rvm)


def test_mode2_oscillation_lattice_kappa(lbm):
    """With c_s^4 = 1/9 in F_axis the drop's mode-2 frequency is the
    Miller-Scriven value within 5 % (the paper reports 6-8 % for its runs)."""
    r = _oscillation(lbm, lbm.KAPPA_LATTICE)
    print("mode 2, kappa c_s^4: omega %.4e MS %.4e err %+.4f R %.2f decay %.2e M_r drift %.1e"
          % (r["omega"], r["omega_ms"], r["err"], r["R"], r["decay"], r["mass_drift"]))
    assert abs(r["err"]) <= 0.05


def test_mode2_oscillation_thermo_kappa(lbm):
    """With the paper's c_s -> c_k substitution (c_k^4, default) the same
    drop oscillates slower than Miller-Scriven: by 5-20 % here."""
    r = _oscillation(lbm, lbm.KAPPA_THERMO)
    print("mode 2, kappa c_k^4: omega %.4e MS %.4e err %+.4f R %.2f decay %.2e M_r drift %.1e"
          % (r["omega"], r["omega_ms"], r["err"], r["R"], r["decay"], r["mass_drift"]))
    assert -0.20 <= r["err"] <= -0.05


def test_mode2_period_fp32(lbm):
    """FP32 (deviations about rho_v) against FP64 for the same oscillation:
    period within 1e-3, axis extent within 0.1 node, r-weighted mass drift
    within 2e-4."""
    r64 = _oscillation(lbm, lbm.KAPPA_LATTICE, precision=64, steps=15000)
    r32 = _oscillation(lbm, lbm.KAPPA_LATTICE, precision=32, steps=15000)
    dper = r64["omega"] / r32["omega"] - 1
    dext = float(np.nanmax(np.abs(r64["ext"] - r32["ext"])))
    print("mode 2 FP32 vs FP64: period error %.2e, max extent difference %.2e, M_r drift FP64 %.1e FP32 %.1e"
          % (dper, dext, r64["mass_drift"], r32["mass_drift"]))
    assert abs(dper) <= 1e-3 and dext <= 0.1 and abs(r32["mass_drift"]) <= 2e-4


# -------------------------------------------------------- radial wave --

def test_radial_density_wave_fp32(lbm):
    """Sec. III.C at its scale (1 x 2000, vdW T = 0.8, lambda = 0.01,
    rho0 = 1.8, A = 0, tau = 0.6, no-slip top) in FP32: a Gaussian ring
    (w_d = 20, rho_p = 1e-3 rho0, centred at r = 120, started at rest)
    splits into an inward and an outward wave.  Up to t_w = 3.98 they follow
    the Bessel series, each mode damped at nu k^2, within 6 % of rho_p (the
    inviscid series within 10 %); at t_w = 5 the inward wave focuses on the
    axis (printed only).  FP32 (deviations about rho0) matches the FP64
    oracle within 1e-2 rho_p (1e-5 of rho0; measured 1.3e-3 at t_w = 1
    growing to 8e-3 as the wave focuses on the axis, where the 1/r terms
    are largest) and keeps the r-weighted mass to 1e-7."""
    nr, rho0, wd, rc = 2000, 1.8, 20.0, 120.0
    rp = 1e-3 * rho0
    p = O.Params(nz=1, nr=nr, tau=0.6, A=0.0, eos=O.EOS_VDW, T=0.8, lam=LAM, axis=1, top=O.TOP_NOSLIP)
    ck = np.sqrt(O.eos.sound_speed_sq(p, rho0))
    nu = (0.6 - 0.5) / 3
    fields = I.radial_bump(1, nr, rho0, rp, wd, r_c=rc)
    o = O.Oracle(p).init(*fields, physical=True)
    eos = lbm.make_eos(lbm.EOS_VDW, 0.8, lam=LAM)
    s = lbm.Solver(1, nr, 0.6, eos=eos, A=0.0, precision=32, rho_ref=rho0, top=lbm.TOP_NOSLIP)
    s.init(*fields, physical=True)
    m0 = s.mass()[0]
    r = np.arange(nr) + 0.5
    sel = slice(0, 400)
    done = 0
    for tw in (1.0, 2.0, 3.98, 5.0):
        steps = int(round(tw * wd / ck))
        o.step(steps - done)
        s.step(steps - done)
        done = steps
        g = s.moments()["rho"][:, 0] - rho0
        ref = o.moments()["rho"][:, 0] - rho0
        bump = lambda x: rp * np.exp(-(((x - rc) / wd) ** 2))  # noqa: E731
        e_vis = np.max(np.abs(g[sel] - O.analytic.bessel_wave(bump, nr, ck, steps, r[sel], 800, nu))) / rp
        e_inv = np.max(np.abs(g[sel] - O.analytic.bessel_wave(bump, nr, ck, steps, r[sel], 800))) / rp
        e_orc = np.max(np.abs(g - ref)) / rp
        print("radial wave t_w %.2f: vs damped series %.3e, vs inviscid %.3e, FP32 vs oracle %.3e (of rho_p); "
              "peak near the axis %.3f rho_p" % (tw, e_vis, e_inv, e_orc, g[:20].max() / rp))
        assert e_orc <= 1e-2
        if tw < 4:
            assert e_vis <= 0.06 and e_inv <= 0.10
    assert s.mass()[0] == pytest.approx(m0, rel=1e-7)
    s.close()


# ------------------------------------------------------------- Fig. 2 --

def _slab_coexistence(lbm, T, A):
    eos = lbm.make_eos(lbm.EOS_VDW, T, lam=LAM)
    rv, rl = lbm.lbm_eos_coexistence(eos)
    s = lbm.Solver(150, 100, 1.0, eos=eos, A=A, precision=64)
    s.init(*I.slab(150, 100, rl, rv, width=4.0), physical=True)
    s.step(40000)
    rho = s.moments()["rho"]
    s.close()
    return rho[:, 75].mean() / rl - 1, rho[:, 0].mean() / rv - 1, rho[:, 75].mean() / rho[:, 0].mean()


def test_fig2_coexistence_curve(lbm):
    """Fig. 2 (150 x 100, tau = 1, vdW lambda = 0.01, a liquid slab started at
    rest, 40000 steps): with A = -0.152 the flat-interface densities follow the
    Maxwell construction -- liquid within 1e-4, vapour within 5e-3 down to
    0.4 T_c and 2e-2 at 0.35 T_c, where the density ratio passes 10^3 --
    while with A = 0 the vapour density is off by more than 2 % (its error
    grows from 2.7 % at 0.9 T_c to 95 % at 0.5 T_c)."""
    for T in (0.35, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9):
        el, ev, ratio = _slab_coexistence(lbm, T, -0.152)
        print("Fig. 2 A = -0.152, T %.2f: liquid %+.2e, vapour %+.2e of Maxwell, ratio %.0f" % (T, el, ev, ratio))
        assert abs(el) <= 1e-4 and abs(ev) <= (2e-2 if T < 0.4 else 5e-3)
        if T == 0.35:
            assert ratio > 1000
    for T in (0.6, 0.7, 0.8, 0.9):
        el, ev, _ = _slab_coexistence(lbm, T, 0.0)
        print("Fig. 2 A = 0, T %.2f: liquid %+.2e, vapour %+.2e of Maxwell" % (T, el, ev))
        assert ev < -2e-2


_VDW_PREP = {}


def _vdw_prep(lbm, kappa, tau, A, T, R0):
    """sigma of the scheme (planar droplet) and the densities a static drop of
    radius R0 keeps in the 500 x 250 box.  At density ratio ~9 the large vapour
    volume evaporates a drop started at the flat-interface densities (R 66 ->
    46), so a first static run measures the 1/R (Kelvin) shift of both
    densities and the drop starts from the densities it has at its own radius."""
    key = (kappa, tau, A, T, round(R0, 6))
    if key in _VDW_PREP:
        return _VDW_PREP[key]
    nz, nr = 500, 250
    eos = lbm.make_eos(lbm.EOS_VDW, T, lam=LAM)
    rv0, rl0 = lbm.lbm_eos_coexistence(eos)
    s = lbm.Solver(256, 16, tau, eos=eos, A=A, precision=64, top=lbm.TOP_PERIODIC, axis=0)
    s.init(*I.slab(256, 16, rl0, rv0, width=4.0), physical=True)
    s.step(40000)
    m = s.moments()["rho"]
    lv, ll = float(m[:, 0].mean()), float(m[:, 128].mean())
    s.close()
    s = lbm.Solver(320, 320, tau, eos=eos, A=A, precision=64, top=lbm.TOP_PERIODIC, axis=0)
    s.init(*I.droplet_2d(320, 320, 64, ll, lv), physical=True)
    s.step(30000)
    R2, _, _ = _plane_state(s.moments()["rho"])
    sig2d = s.pressure_jump(160, 160, R2 / 2, R2 + 12) * R2
    s.close()
    s = lbm.Solver(nz, nr, tau, eos=eos, A=A, precision=64, kappa=kappa)
    s.init(*I.droplet(nz, nr, R0, ll, lv), physical=True)
    s.step(20000)
    R1, rl1, rv1 = _axis_state(s.moments()["rho"])
    s.close()
    s = lbm.Solver(nz, nr, tau, eos=eos, A=A, precision=64, kappa=kappa)
    s.init(*I.droplet(nz, nr, R0, ll + (rl1 - ll) * R1 / R0, lv + (rv1 - lv) * R1 / R0), physical=True)
    s.step(20000)
    Rs, rl, rv = _axis_state(s.moments()["rho"])
    s.close()
    _VDW_PREP[key] = (sig2d, R1, Rs, rl, rv)
    return _VDW_PREP[key]


def _oscillation_vdw(lbm, kappa, tau=0.8, A=0.0, T=0.8, shape=(62, 76), steps=25000, every=100):
    """Mode-2 frequency of an ellipsoidal drop with the paper's vdW fluid
    (lambda = 0.01, A = 0, T = 0.8 T_c, density ratio about 9; tau = 0.8, the
    smallest at which this drop runs from rest, the paper's being 0.7), and the
    Miller-Scriven value for its measured radius and densities.  The ellipsoid
    (semi-axes Ra radially, Rz along z) is scaled to the equilibrium radius of
    the static drop of equal volume and started at rest with its densities."""
    nz, nr = 500, 250
    eos = lbm.make_eos(lbm.EOS_VDW, T, lam=LAM)
    Ra, Rz = shape
    R0 = (Ra * Ra * Rz) ** (1 / 3)
    sig2d, R1, Rs, rl, rv = _vdw_prep(lbm, kappa, tau, A, T, R0)
    k = Rs / R0
    s = lbm.Solver(nz, nr, tau, eos=eos, A=A, precision=64, kappa=kappa)
    s.init(*I.ellipsoid(nz, nr, Ra * k, Rz * k, rl, rv), physical=True)
    ts, ext, rad, dens = [], [], [], []
    for i in range(steps // every):
        rho = lbm.lbm_axi_moments(s.h, nz, nr, want=("rho",))["rho"]
        R, a, b = _axis_state(rho)
        ts.append(i * every)
        ext.append(_half_extent(rho[0], a, b))
        rad.append(R)
        dens.append((a, b))
        s.step(every)
    s.close()
    ts, ext = np.array(ts[3:]), np.array(ext[3:])
    Rm = float(np.mean(rad[3:]))
    rlm, rvm = np.mean([d[0] for d in dens[3:]]), np.mean([d[1] for d in dens[3:]])
    nu = (tau - 0.5) / 3
    w_ms = O.analytic.miller_scriven_omega2(sig2d, Rm, rlm, rvm, nu, nu)
    w, c = O.analytic.fit_damped_cosine(ts, ext, w_guess=w_ms)
    return dict(omega=w, omega_ms=w_ms, err=w / w_ms - 1, R=Rm, R_flat_start=R1, R_equilibrated=Rs)


def test_mode2_oscillation_vdw(lbm):
    """The paper's fluid (vdW, A = 0, ratio about 9): with c_s^4 in F_axis the
    mode-2 frequency is Miller-Scriven's within 5 %; with the paper's c_k^4 it
    is 3-15 % low (measured -9 %; the paper reports 6-8 % errors)."""
    out = {}
    for kappa in (lbm.KAPPA_LATTICE, lbm.KAPPA_THERMO):
        r = _oscillation_vdw(lbm, kappa)
        out[kappa] = r
        print("mode 2 vdW, kappa %d: omega %.4e MS %.4e err %+.4f R %.2f (flat-density start %.1f, equilibrated %.1f)"
              % (kappa, r["omega"], r["omega_ms"], r["err"], r["R"], r["R_flat_start"], r["R_equilibrated"]))
    assert abs(out[lbm.KAPPA_LATTICE]["err"]) <= 0.05
    assert -0.15 <= out[lbm.KAPPA_THERMO]["err"] <= -0.03


# Fig. 3's four ellipsoids (aspect ratios not printed): equal volume, the
# radius of the (62, 76) drop, Rz / Ra = 0.8, 1.1, 76/62 and 1.4.
FIG3_SHAPES = [(66.3 * q ** (-1 / 3), 66.3 * q ** (2 / 3)) for q in (0.8, 1.1, 76 / 62, 1.4)]


def test_fig3_four_ellipsoids_vdw(lbm):
    """Fig. 3 (Sec. III.B): four initial ellipsoids of the paper's fluid; the
    paper finds mode-2 frequency errors of 6 % (min) to 8 % (max) against
    Miller-Scriven, Eq. (oscillatingfreq).  Here, per reading of the c^4 factor
    of F_axis: with c_k^4 (the paper's statement) every shape is 3-15 % low
    (measured 6.5-11 %, the paper's range widened by the shapes); with c_s^4
    every shape is within 6 %; the spread over the four shapes stays within
    6 points for either reading."""
    out = {}
    for kappa in (lbm.KAPPA_THERMO, lbm.KAPPA_LATTICE):
        errs = []
        for shape in FIG3_SHAPES:
            r = _oscillation_vdw(lbm, kappa, shape=shape)
            errs.append(r["err"])
            print("Fig. 3 vdW kappa %d shape (%.1f, %.1f): omega %.4e MS %.4e err %+.4f R %.2f"
                  % (kappa, shape[0], shape[1], r["omega"], r["omega_ms"], r["err"], r["R"]))
        a = np.abs(errs)
        print("Fig. 3 vdW kappa %d: |error| min %.3f max %.3f (paper: 0.06 .. 0.08)" % (kappa, a.min(), a.max()))
        out[kappa] = errs
    for kappa, lo, hi in ((lbm.KAPPA_THERMO, -0.15, -0.03), (lbm.KAPPA_LATTICE, -0.06, 0.06)):
        errs = out[kappa]
        assert all(lo <= e <= hi for e in errs), (kappa, errs)
        assert max(errs) - min(errs) <= 0.06, (kappa, errs)


# ------------------------------------------- Table 1: absolute values --

def _slab_profile(lbm, T, A, forcing, tau=1.5, nz=256, nr=8, steps=30000):
    """Relaxed flat interface (fully periodic box, slab normal to z), FP64:
    the density profile along z averaged over r."""
    eos = lbm.make_eos(lbm.EOS_VDW, T, lam=LAM)
    rv, rl = lbm.lbm_eos_coexistence(eos)
    s = lbm.Solver(nz, nr, tau, eos=eos, A=A, precision=64, top=lbm.TOP_PERIODIC, axis=0, forcing=forcing)
    s.init(*I.slab(nz, nr, rl, rv, width=8.0), physical=True)
    s.step(steps)
    rho = s.moments()["rho"].mean(axis=0)
    s.close()
    return rho


def _mechanical_sigma(rho, T, A, edm):
    """Surface tension of a flat interface as the excess of normal over
    tangential pressure, per interface (the profile holds two).  The Taylor
    expansion of the discrete force of Eq. (kupershtokhforcing) (exact for
    quadratic psi, pinned on the oracle) is
    F = 2 psi grad psi + (1/3) psi grad lap psi + (2A/3) grad psi lap psi + (2A/3) grad |grad psi|^2,
    the divergence of a tensor with P_N - P_T = (1 - 2A)/3 psi'^2 across a flat
    interface.  The EDM adds F F / (4 rho) to the momentum flux of the lattice
    fluid (the second moment of its equilibrium shift is rho u1 u1 - rho u0 u0,
    not that of the mean velocity); Guo forcing adds nothing.  So
    sigma = int [(1 - 2A)/3 psi'^2 + F_z^2 / (4 rho)] dz (EDM), without the last term (Guo).
    psi' by the isotropic stencil of Eq. (fifthorderaccuratefinitedifference)
    on a z-only profile (the 4th-order central difference); F_z the discrete
    force of Eq. (kupershtokhforcing) on that profile."""
    p = O.Params(nz=len(rho), nr=1, eos=O.EOS_VDW, T=T, lam=LAM, A=A)
    pk = np.array([O.core.eos_p(p, x) for x in rho])
    psi = np.sqrt(rho / 3 - pk)
    up, dn = np.roll(psi, -1), np.roll(psi, 1)
    d = (2 / 3) * (up - dn) - (1 / 12) * (np.roll(psi, -2) - np.roll(psi, 2))
    fz = A * (up * up - dn * dn) + (1 - 2 * A) * psi * (up - dn)
    s = (1 - 2 * A) / 3 * np.sum(d * d) / 2
    return s + (np.sum(fz * fz / (4 * rho)) / 2 if edm else 0.0)


def _laplace_2d(lbm, T, A, forcing, n=320, R0=64, steps=40000):
    eos = lbm.make_eos(lbm.EOS_VDW, T, lam=LAM)
    rv, rl = lbm.lbm_eos_coexistence(eos)
    s = lbm.Solver(n, n, 1.5, eos=eos, A=A, precision=64, top=lbm.TOP_PERIODIC, axis=0, forcing=forcing)
    s.init(*I.droplet_2d(n, n, R0, rl, rv, width=8.0), physical=True)
    s.step(steps)
    R, _, _ = _plane_state(s.moments()["rho"])
    sig = s.pressure_jump(n / 2, n / 2, R / 2, R + 24) * R
    s.close()
    return sig


@pytest.mark.parametrize("A", [0.0, -0.152])
@pytest.mark.parametrize("T", [0.7, 0.8, 0.9])
def test_table1_sigma_mechanics_and_forcing(lbm, T, A):
    """Where Table 1's absolute values part from this build's.  For each
    forcing scheme the surface tension from the printed law (planar droplet,
    dp R, vdW lambda = 0.01, tau = 1.5, FP64) is the flat interface's mechanical
    surface tension within 5 % (measured 0.4-0.7 % EDM, 2-4 % Guo): with the
    EDM it carries the scheme's F F / (4 rho) stress, about half of it, which
    Guo forcing (named in Sec. II.A) lacks.  Guo's values are Table 1's
    printed ones within 6 % (measured -1.1 % .. +5.1 %, five of six within
    1.5 %), the EDM's 1.46-1.90 times them: the paper's Table 1 was computed
    with Guo forcing."""
    out = {}
    for name, forcing in (("EDM", lbm.FORCING_EDM), ("Guo", lbm.FORCING_GUO)):
        rho = _slab_profile(lbm, T, A, forcing)
        sm = _mechanical_sigma(rho, T, A, edm=forcing == lbm.FORCING_EDM)
        sl = _laplace_2d(lbm, T, A, forcing)
        out[name] = (sl, sm)
    paper = TABLE1[(T, A)][0]
    print("Table 1 trace T %.1f A %+.3f: sigma/lam EDM Laplace %.4f mechanical %.4f | Guo Laplace %.4f mechanical "
          "%.4f | paper 2D %.3f | EDM/paper %.3f Guo/paper %.3f"
          % (T, A, out["EDM"][0] / LAM, out["EDM"][1] / LAM, out["Guo"][0] / LAM, out["Guo"][1] / LAM, paper,
             out["EDM"][0] / LAM / paper, out["Guo"][0] / LAM / paper))
    for name, (sl, sm) in out.items():
        assert sl / sm == pytest.approx(1.0, abs=0.05), (name, sl, sm)
    assert out["Guo"][0] / LAM == pytest.approx(paper, rel=0.06)
    assert out["EDM"][0] / LAM > 1.4 * paper


# ------------------------------------------------ Guo forcing vs the EDM --

def _flat_coexistence(lbm, T, forcing, tau=1.0, steps=40000):
    """Flat-interface densities relative to Maxwell's, or the step at which the
    run went unphysical."""
    eos = lbm.make_eos(lbm.EOS_VDW, T, lam=LAM)
    rv, rl = lbm.lbm_eos_coexistence(eos)
    s = lbm.Solver(150, 16, tau, eos=eos, A=-0.152, precision=64, top=lbm.TOP_PERIODIC, axis=0, forcing=forcing)
    s.init(*I.slab(150, 16, rl, rv, width=4.0), physical=True)
    done = 0
    try:
        while done < steps:
            s.step(1000)
            done += 1000
    except lbm.LbmError:
        s.close()
        return None, done
    rho = s.moments()["rho"]
    s.close()
    return (rho[:, 75].mean() / rl - 1, rho[:, 0].mean() / rv - 1), done


def test_guo_vs_edm_laplace_and_oscillation(lbm):
    """The forcing variant of Sec. II.A (Guo) beside the default EDM on the
    coexistence pin (vdW, A = -0.152, flat interface, tau = 1), Young-Laplace
    (P9) and the mode-2 oscillation (P10, CS 0.8 T_c, c_s^4 in F_axis).
    A = -0.152 is Kupershtokh's value for the EDM: the EDM keeps the Maxwell
    densities from 0.9 down to 0.6 T_c, while Guo forcing leaves them by more
    and, at 0.6 T_c, does not keep the flat interface at all (the run goes
    unphysical; printed).  The planar surface tension and the oscillation are
    reported for both; Guo's sigma is the EDM's less its F F / (4 rho) stress
    (see the Table 1 trace), so it is smaller, and its mode-2 frequency stays
    within 15 % of Miller-Scriven's with its own sigma."""
    for T in (0.6, 0.8, 0.9):
        edm, _ = _flat_coexistence(lbm, T, lbm.FORCING_EDM)
        guo, n_guo = _flat_coexistence(lbm, T, lbm.FORCING_GUO)
        print("coexistence vdW T %.1f A -0.152: EDM liquid %+.2e vapour %+.2e | Guo %s"
              % (T, edm[0], edm[1], "liquid %+.2e vapour %+.2e (of Maxwell)" % guo if guo
                 else "unphysical by step %d" % n_guo))
        assert abs(edm[0]) <= 1e-3 and abs(edm[1]) <= 5e-3
        if T >= 0.8:
            assert guo is not None
    r_e = _oscillation(lbm, lbm.KAPPA_LATTICE, steps=20000)
    r_g = _oscillation(lbm, lbm.KAPPA_LATTICE, steps=20000, forcing=lbm.FORCING_GUO)
    for name, r in (("EDM", r_e), ("Guo", r_g)):
        print("CS 0.8 Tc, %s: planar sigma %.5e, mode-2 omega %.4e, Miller-Scriven %.4e, error %+.4f, "
              "R %.2f, rho_l %.5f, rho_v %.5f" % (name, r["sigma_2d"], r["omega"], r["omega_ms"], r["err"], r["R"],
                                                   r["rho_l"], r["rho_v"]))
    assert abs(r_e["err"]) <= 0.05 and abs(r_g["err"]) <= 0.15
    assert r_g["sigma_2d"] < r_e["sigma_2d"]


# ------------------------------------------- F_axis: the A-term coefficient --

def _sphere_over_planar(lbm, forcing, term, radii=(32, 48, 64)):
    """sigma from dp = 2 sigma / R of axisymmetric droplets over sigma from the
    planar droplet (dp = sigma / R) of the same fluid (CS 0.8 T_c, A = -0.152,
    tau = 1, c^4 = c_s^4 in F_axis, FP64)."""
    eos = lbm.make_eos(lbm.EOS_CS, 0.8)
    rv, rl = lbm.lbm_eos_coexistence(eos)
    s = lbm.Solver(256, 256, 1.0, eos=eos, A=-0.152, precision=64, top=lbm.TOP_PERIODIC, axis=0, forcing=forcing)
    s.init(*I.droplet_2d(256, 256, 48, rl, rv), physical=True)
    s.step(20000)
    R2, _, _ = _plane_state(s.moments()["rho"])
    sig2d = s.pressure_jump(128, 128, R2 / 2, R2 + 12) * R2
    s.close()
    sig = []
    for R0 in radii:
        nz, nr = 4 * R0 + 64, 2 * R0 + 48
        s = lbm.Solver(nz, nr, 1.0, eos=eos, A=-0.152, precision=64, kappa=lbm.KAPPA_LATTICE, forcing=forcing,
                       axis_a_term=term)
        s.init(*I.droplet(nz, nr, R0, rl, rv), physical=True)
        s.step(20000)
        R, _, _ = _axis_state(s.moments()["rho"])
        sig.append(s.pressure_jump(nz / 2, 0, R / 2, R + 12) * R / 2)
        s.close()
    return np.array(sig) / sig2d, sig2d


def test_axis_a_term_young_laplace_and_oscillation(lbm):
    """F_axis's A-term with the printed coefficient (6A) and the exact
    expansion's (2A), at c^4 = c_s^4 (CS, 0.8 T_c, A = -0.152, tau = 1): the
    spherical Young-Laplace law dp = 2 sigma / R over R = 32..64 against the
    planar droplet's sigma, for the EDM and for Guo forcing, and the EDM's
    mode-2 frequency against Miller-Scriven.  F_axis corrects the psi terms of
    the force for the hoop curvature; the EDM's F F / (4 rho) stress, about
    half of its sigma, gets no such correction, so with the EDM the sphere
    reads low by about a quarter with the exact 2A (measured 0.79), and the
    printed 6A over-corrects the psi terms into 0.93.  Guo forcing has no
    such stress, and with the exact 2A its sphere obeys dp = 2 sigma / R with
    the planar sigma within 0.5 % (6A: 24 % high).  dp R is constant over R
    within 6 % for every combination."""
    res = {}
    for fname, forcing in (("EDM", lbm.FORCING_EDM), ("Guo", lbm.FORCING_GUO)):
        for tname, term in (("6A", lbm.AXIS_A_PRINTED), ("2A", lbm.AXIS_A_EXPANSION)):
            ratio, sig2d = _sphere_over_planar(lbm, forcing, term)
            res[(fname, tname)] = ratio
            print("F_axis A-term %s, %s: sphere sigma(R = 32, 48, 64) / planar sigma %.5e = %s"
                  % (tname, fname, sig2d, np.round(ratio, 4).tolist()))
            assert ratio.max() / ratio.min() < 1.06
    for tname, term in (("6A", lbm.AXIS_A_PRINTED), ("2A", lbm.AXIS_A_EXPANSION)):
        r = _oscillation(lbm, lbm.KAPPA_LATTICE, steps=20000, axis_a_term=term)
        print("F_axis A-term %s, EDM: mode-2 omega %.4e, Miller-Scriven %.4e, error %+.4f"
              % (tname, r["omega"], r["omega_ms"], r["err"]))
        res[("osc", tname)] = r["err"]
    assert np.all(np.abs(res[("EDM", "6A")] - 0.93) <= 0.03)
    assert np.all(np.abs(res[("EDM", "2A")] - 0.79) <= 0.03)
    assert abs(res[("osc", "6A")]) <= 0.02 and abs(res[("osc", "2A")]) <= 0.07
    # Guo forcing has no F F / (4 rho) stress: the exact 2A makes the sphere's
    # Laplace law the planar one's (measured 0.999 .. 1.005); 6A over-corrects (1.24)
    assert np.all(np.abs(res[("Guo", "2A")] - 1.0) <= 0.02)
    assert np.all(np.abs(res[("Guo", "6A")] - 1.245) <= 0.03)
