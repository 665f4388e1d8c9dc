"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 bar, after the stated steps (only the rounding order differs between the
two): max |gpu - oracle| / max |oracle| <= 1e-12 for rho and P_k; for each
velocity component c, max |u_gpu - u_oracle| / max(max |u_c|, 1e-3) <= 1e-12,
and the same for the velocity vector.  A velocity's FP64 rounding error is
absolute (populations of size w_i rho summed into rho u), so below 1e-3 the
bar is the absolute 1e-15, ten units of that rounding.  States are chosen
with disturbances large enough that the discrete force -- a difference of
nearly equal psi values -- is not dominated by cancellation.  FP32 bars are
per result and stated in test_gpu_fp32.py.
"""
import numpy as np
import pytest

import oracle as O
from paper_1512_01977_gb300 import inputs as I
from tests._cases import Case, component_errs, rel_err, run_gpu, run_oracle, vel_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _library():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_01977_gb300 import build, lbm

    build.build()
    lbm.lib()


def _droplet_fields(case, R, du=0.0, seed=0, eps=0.0):
    rv, rl = case.coexistence()
    rho, uz, ur = I.droplet(case.nz, case.nr, R, rl, rv, eps=eps)
    if du:
        _, vz, vr = I.random_state(case.nz, case.nr, 1.0, 0.0, du, seed)
        uz, ur = vz, vr * (np.arange(case.nr) + 0.5)[:, None] / case.nr  # u_r -> 0 at the axis
    return rho, uz, ur


def _check(mg, mo, tol=TOL64):
    errs = {k: rel_err(mg[k], mo[k]) for k in ("rho", "p")}
    errs["u"] = vel_err(mg, mo)
    errs.update(component_errs(mg, mo))
    for k, e in errs.items():
        assert e <= tol, (k, errs)
    return errs


def _compare(case, fields, steps, tol=TOL64, tuning=None):
    o = run_oracle(case, fields, steps)
    s = run_gpu(case, fields, steps, tuning=tuning)
    mo, mg = o.moments(), s.moments()
    s.close()
    return _check(mg, mo, tol)


@pytest.mark.parametrize("tuning", [(1, 0), (1, 4), (1, 20), (1, 64), (2, 16)])
@pytest.mark.parametrize("top", [O.TOP_FREESLIP, O.TOP_NOSLIP, O.TOP_PERIODIC])
def test_fused_and_split_paths_fp64(tuning, top):
    """The single-pass kernel (path 1) with several chunk heights (chunk seams
    inside the droplet) and the two-kernel path (2) against the oracle."""
    c = Case(70, 44, top=top, axis=0 if top == O.TOP_PERIODIC else 1)
    _compare(c, _droplet_fields(c, 13, du=2e-3, seed=9), 80, tuning=tuning)


@pytest.mark.parametrize("top", [O.TOP_FREESLIP, O.TOP_NOSLIP, O.TOP_PERIODIC])
@pytest.mark.parametrize("nz,nr", [(200, 40), (290, 37)])
def test_fp64_grids_wider_than_a_strip(nz, nr, top):
    """The fused FP64 kernel on grids that span several z-strips (strip seams,
    a ragged last strip) against the oracle, with every top boundary."""
    c = Case(nz, nr, top=top, axis=0 if top == O.TOP_PERIODIC else 1)
    rv, rl = c.coexistence()
    rho, uz, ur = I.droplet(nz, nr, 12, rl, rv)
    _, vz, vr = I.random_state(nz, nr, 1.0, 0.0, 2e-3, nz + nr)
    ur = vr * (np.arange(nr) + 0.5)[:, None] / nr
    # a second droplet across the periodic z seam
    rho2, _, _ = I.droplet(nz, nr, 9, rl, rv)
    rho = np.maximum(rho, np.roll(rho2, nz // 2 - 3, axis=1))
    _compare(c, (rho, vz, ur), 64)


@pytest.mark.parametrize("rows_per_cta", [0, 16])
def test_fp64_wide_grid_balanced_and_chunked(rows_per_cta):
    """A 290 x 37 droplet pair through the balanced one-wave grid (the batched
    kernel's single-solve form) and through 16-row chunks of the chunked kernel."""
    c = Case(290, 37)
    rv, rl = c.coexistence()
    rho, _, _ = I.droplet(290, 37, 11, rl, rv)
    rho = np.maximum(rho, np.roll(rho, 140, axis=1))
    _, vz, vr = I.random_state(290, 37, 1.0, 0.0, 2e-3, 5)
    from paper_1512_01977_gb300 import lbm

    _compare(c, (rho, vz, vr * (np.arange(37) + 0.5)[:, None] / 37), 70, tuning=(lbm.PATH_FUSED, rows_per_cta))


@pytest.mark.parametrize("path", ["fused", "split"])
@pytest.mark.parametrize("top", [O.TOP_FREESLIP, O.TOP_NOSLIP])
def test_guo_forcing_fp64(top, path):
    """Guo forcing against the oracle, through the fused kernel's Guo form (the
    default with the force and the axis terms on) and the two-kernel path: a
    droplet started at rest with a random flow, and a single-phase channel driven
    by a body force (two-kernel path: the fused forms need the force on)."""
    from paper_1512_01977_gb300 import lbm

    c = Case(45, 27, top=top, forcing=O.FORCING_GUO)
    fields = _droplet_fields(c, 10, du=2e-3, seed=41)
    o = O.Oracle(c.oracle_params()).init(*fields, physical=True).step(80)
    s = c.solver().init(*fields, physical=True)
    assert lbm.lbm_axi_get_tuning(s.h)[0] == lbm.PATH_FUSED
    with pytest.raises(lbm.LbmError):
        lbm.lbm_axi_set_tuning(s.h, lbm.PATH_FUSED, 16)  # chunked grids have the EDM form only
    with pytest.raises(lbm.LbmError):
        lbm.Batch([s])
    if path == "split":
        lbm.lbm_axi_set_tuning(s.h, lbm.PATH_SPLIT, 0)
    s.step(80)
    mg = s.moments()
    s.close()
    _check(mg, o.moments())
    c = Case(8, 16, multiphase=0, top=O.TOP_NOSLIP, gz=1e-5, forcing=O.FORCING_GUO)
    s = c.solver()
    assert lbm.lbm_axi_get_tuning(s.h)[0] == lbm.PATH_SPLIT
    with pytest.raises(lbm.LbmError):
        lbm.lbm_axi_set_tuning(s.h, lbm.PATH_FUSED, 0)
    s.close()
    _compare(c, I.random_state(8, 16, 1.0, 0.01, 1e-3, 6), 200)


@pytest.mark.parametrize("top", [O.TOP_FREESLIP, O.TOP_NOSLIP])
@pytest.mark.parametrize("forcing,h_eval", [(O.FORCING_GUO, O.H_LOCAL), (O.FORCING_EDM, O.H_LINK_AVG),
                                            (O.FORCING_GUO, O.H_LINK_AVG)])
def test_collision_forms_wide_grid_fp64(forcing, h_eval, top):
    """The fused kernel's Guo and link-source forms on a 230 x 33 grid (three
    z-strips, a ragged last one; a droplet pair, one across the periodic z seam)
    against the oracle, with both wall tops."""
    from paper_1512_01977_gb300 import lbm

    nz, nr = 230, 33
    c = Case(nz, nr, top=top, forcing=forcing, h_eval=h_eval)
    s = c.solver()
    assert lbm.lbm_axi_get_tuning(s.h)[0] == lbm.PATH_FUSED
    s.close()
    rv, rl = c.coexistence()
    rho, _, _ = I.droplet(nz, nr, 10, rl, rv)
    rho = np.maximum(rho, np.roll(rho, nz // 2 + 1, axis=1))
    _, vz, vr = I.random_state(nz, nr, 1.0, 0.0, 2e-3, 77)
    ur = vr * (np.arange(nr) + 0.5)[:, None] / nr
    # the given velocity is the physical one (with EDM and the link source a start
    # at u0 = u leaves the coexistence state within ~15 steps, in the oracle too)
    o = O.Oracle(c.oracle_params()).init(rho, vz, ur, physical=True).step(60)
    s = c.solver().init(rho, vz, ur, physical=True).step(60)
    mg = s.moments()
    s.close()
    _check(mg, o.moments())


def test_init_moments_roundtrip():
    """f = f^eq(rho, u) then moments: rho back exactly, u = u0 + F/(2 rho)."""
    c = Case(40, 24)
    fields = _droplet_fields(c, 9, du=1e-3)
    o = O.Oracle(c.oracle_params()).init(*fields)
    s = c.solver().init(*fields)
    mg, mo = s.moments(), o.moments()
    np.testing.assert_allclose(mg["rho"], fields[0], rtol=1e-15, atol=0)
    assert rel_err(mg["rho"], mo["rho"]) <= 1e-13
    assert vel_err(mg, mo) <= 1e-13
    assert rel_err(mg["p"], mo["p"]) <= TOL64
    s.close()


def test_droplet_fp64_ragged_tiles():
    """Droplet with a random velocity field on a grid that is not a multiple
    of the tile in either direction (ragged last tiles)."""
    c = Case(45, 27)
    _compare(c, _droplet_fields(c, 10, du=2e-3, seed=1), 150)


@pytest.mark.parametrize("top", [O.TOP_FREESLIP, O.TOP_NOSLIP, O.TOP_PERIODIC])
def test_boundaries_fp64(top):
    c = Case(36, 20, top=top, axis=0 if top == O.TOP_PERIODIC else 1)
    _compare(c, _droplet_fields(c, 8, du=2e-3, seed=2), 60)


@pytest.mark.parametrize("kappa", [O.KAPPA_THERMO, O.KAPPA_LATTICE, O.KAPPA_MIXED])
def test_kappa_modes_fp64(kappa):
    c = Case(40, 24, kappa=kappa)
    _compare(c, _droplet_fields(c, 9, du=1e-3, seed=3), 60)


@pytest.mark.parametrize("tuning", [(1, 0), (2, 0)])
@pytest.mark.parametrize("kappa", [O.KAPPA_LATTICE, O.KAPPA_THERMO])
def test_axis_a_expansion_fp64(kappa, tuning):
    """F_axis with the exact expansion's A-coefficient (c = 2), fused and
    two-kernel paths, against the oracle."""
    c = Case(45, 27, kappa=kappa, axis_a=2.0)
    _compare(c, _droplet_fields(c, 10, du=2e-3, seed=13), 60, tuning=tuning)


def test_vdw_fp64():
    c = Case(48, 28, tau=1.5, eos=O.EOS_VDW, A=0.0, T_over_Tc=0.8)
    _compare(c, _droplet_fields(c, 10, du=1e-3, seed=4), 60)


def test_printed_hr_sign_fp64():
    """The +u_r/r reading of H_r (as printed; unstable over long runs) is
    selectable and matches the oracle's over a short single-phase run."""
    from scipy import special

    c = Case(3, 32, multiphase=0, tau=0.8, hr_sign=+1)
    fields = I.radial_mode(3, 32, 1.0, 1e-2, special.jn_zeros(1, 1)[0] / 32)
    _compare(c, fields, 10)


def test_single_phase_body_force_fp64():
    c = Case(8, 16, multiphase=0, top=O.TOP_NOSLIP, gz=1e-5)
    rho, uz, ur = I.random_state(8, 16, 1.0, 0.01, 1e-3, 6)
    _compare(c, (rho, uz, ur), 200)


@pytest.mark.parametrize("nz,nr", [(1, 1), (1, 7), (5, 1), (3, 3), (33, 9), (31, 17)])
def test_tiny_and_thin_grids_fp64(nz, nr):
    """Grids thinner than the stencil halo (multiple reflections, wraps)."""
    c = Case(nz, nr, multiphase=1, T_over_Tc=0.9)
    rho, uz, ur = I.random_state(nz, nr, 0.2, 0.01, 1e-3, nz * 100 + nr)
    _compare(c, (rho, uz, ur), 30)


def test_radial_wave_channel_fp64():
    """The paper's 1 x N_r wave channel (nz = 1), vdW, no-slip top."""
    c = Case(1, 400, tau=0.6, eos=O.EOS_VDW, A=0.0, T_over_Tc=0.8, top=O.TOP_NOSLIP)
    fields = I.radial_bump(1, 400, 1.8, 0.05 * 1.8, 10.0)
    _compare(c, fields, 300)


def test_droplet_64x64_full_fp64():
    """64 x 64 droplet (CS, T = 0.8 Tc, A = -0.152, tau = 1, R = 16, tanh width 2),
    the full 2000 steps."""
    c = Case(64, 64)
    errs = _compare(c, _droplet_fields(c, 16), 2000)
    print("64x64 droplet parity", errs)


def test_mass_and_pressure_jump_fp64():
    c = Case(64, 40)
    fields = _droplet_fields(c, 12)
    o = run_oracle(c, fields, 100)
    s = run_gpu(c, fields, 100)
    mr, m = s.mass()
    assert mr == pytest.approx(o.mass_rweighted(), rel=1e-13)
    assert m == pytest.approx(o.mass(), rel=1e-13)
    mo = o.moments()
    Z, Rr = I.grid(64, 40)
    d = np.sqrt((Z - 32) ** 2 + Rr**2)
    dp_o = mo["p"][d < 6].mean() - mo["p"][d > 20].mean()
    assert s.pressure_jump(32.0, 0.0, 6.0, 20.0) == pytest.approx(dp_o, rel=1e-12)
    s.close()


def test_step_chunking_is_invisible():
    """n steps in one call (CUDA-graph chunks + tail) equal n single-step calls."""
    c = Case(40, 24)
    fields = _droplet_fields(c, 9, du=1e-3)
    a = run_gpu(c, fields, 301)
    b = c.solver().init(*fields)
    for _ in range(301):
        b.step(1)
    ma, mb = a.moments(), b.moments()
    for k in ma:
        np.testing.assert_array_equal(ma[k], mb[k])
    a.close()
    b.close()


def test_unphysical_state_is_reported():
    from paper_1512_01977_gb300 import lbm

    c = Case(16, 8)
    rho = np.full((8, 16), 0.2)
    rho[3, 5] = -0.1
    s = c.solver().init(rho)
    with pytest.raises(lbm.LbmError) as e:
        s.step(5)
    assert e.value.code == lbm.ERR_UNPHYSICAL
    s.init(np.full((8, 16), 0.2))  # recoverable: re-init and continue
    s.step(5)
    s.close()


def test_invalid_calls():
    from paper_1512_01977_gb300 import lbm

    with pytest.raises(lbm.LbmError):
        lbm.Solver(0, 4, 1.0, eos=lbm.make_eos())
    with pytest.raises(lbm.LbmError):
        lbm.Solver(4, 4, 0.4, eos=lbm.make_eos())
    s = lbm.Solver(4, 4, 1.0, eos=lbm.make_eos())
    with pytest.raises(lbm.LbmError) as e:
        s.step(1)
    assert e.value.code == lbm.ERR_STATE
    s.close()


def test_torch_allocator_and_stream():
    import torch

    from paper_1512_01977_gb300 import lbm

    c = Case(40, 24)
    fields = _droplet_fields(c, 9, du=1e-3)
    ref = run_gpu(c, fields, 50).moments()
    lbm.use_torch_allocator()
    try:
        st = torch.cuda.Stream()
        eos = lbm.make_eos(c.eos, c.T_over_Tc)
        s = lbm.Solver(c.nz, c.nr, c.tau, eos=eos, A=c.A, stream=st.cuda_stream)
        s.init(*fields).step(50)
        m = s.moments()
        s.close()
    finally:
        lbm.use_cuda_allocator()
    for k in ref:
        np.testing.assert_array_equal(m[k], ref[k])


def test_device_init_and_moments():
    import torch

    from paper_1512_01977_gb300 import lbm

    c = Case(40, 24)
    fields = _droplet_fields(c, 9, du=1e-3)
    host = run_gpu(c, fields, 40).moments()
    s = c.solver()
    d = [torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda") for a in fields]
    lbm.lbm_axi_init_device(s.h, *d)
    s.step(40)
    out = [torch.empty(24 * 40, dtype=torch.float64, device="cuda") for _ in range(4)]
    lbm.lbm_axi_moments_device(s.h, *out)
    torch.cuda.synchronize()
    for k, t in zip(("rho", "uz", "ur", "p"), out):
        np.testing.assert_array_equal(t.cpu().numpy().reshape(24, 40), host[k])
    s.close()


@pytest.mark.parametrize("device_arrays", [False, True])
def test_init_physical_fp64(device_arrays):
    """lbm_axi_init_physical(_device): the first state's fluid velocity is the
    given u (the droplet starts at rest plus a random flow), equal to the
    oracle's start, and a run from it at the oscillating-droplet settings
    (vdW, T = 0.8 T_c, A = 0, tau = 0.7) follows the oracle."""
    import torch

    from paper_1512_01977_gb300 import lbm

    c = Case(45, 27, tau=0.7, eos=O.EOS_VDW, A=0.0, T_over_Tc=0.8)
    fields = _droplet_fields(c, 10, du=2e-3, seed=12)
    o = O.Oracle(c.oracle_params()).init(*fields, physical=True)
    mo0 = o.moments()
    s = c.solver()
    if device_arrays:
        d = [torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda") for a in fields]
        lbm.lbm_axi_init_physical_device(s.h, *d)
    else:
        s.init(*fields, physical=True)
    m0 = s.moments()
    assert vel_err(m0, mo0) <= 1e-13
    assert vel_err(m0, {"uz": fields[1], "ur": fields[2]}) <= 1e-13
    assert rel_err(m0["rho"], mo0["rho"]) <= 1e-15
    o.step(150)
    s.step(150)
    mo, mg = o.moments(), s.moments()
    s.close()
    assert rel_err(mg["rho"], mo["rho"]) <= TOL64 and vel_err(mg, mo) <= TOL64 and rel_err(mg["p"], mo["p"]) <= TOL64


def test_init_physical_reports_unphysical_density():
    from paper_1512_01977_gb300 import lbm

    c = Case(16, 8)
    rho = np.full((8, 16), 0.2)
    rho[3, 5] = -0.1
    s = c.solver()
    with pytest.raises(lbm.LbmError) as e:
        s.init(rho, physical=True)
    assert e.value.code == lbm.ERR_UNPHYSICAL
    s.init(np.full((8, 16), 0.2), physical=True).step(3)
    s.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_checkpoint_resume_is_exact(precision):
    """Save after an odd number of steps (the other population buffer is
    current), load into a fresh solve, step on: bitwise the uninterrupted run."""
    from paper_1512_01977_gb300 import lbm

    c = Case(45, 27)
    rv, _ = c.coexistence()
    rr = rv if precision == 32 else 0.0
    fields = _droplet_fields(c, 10, du=2e-3, seed=21)
    a = c.solver(precision, rr).init(*fields)
    a.step(37)
    blob = a.save()
    assert len(blob) == lbm.lbm_axi_state_bytes(a.h)
    a.step(40)
    ref = a.moments()
    b = c.solver(precision, rr).load(blob)
    b.step(40)
    m = b.moments()
    for k in ("rho", "uz", "ur", "p"):
        np.testing.assert_array_equal(m[k], ref[k])
    assert b.mass() == a.mass()
    # a blob of another grid, precision, rho_ref or dynamics (tau, temperature, A, boundary,
    # kappa, forcing) is refused; a fresh solve cannot be saved
    others = [Case(45, 28).solver(precision, rr), c.solver(96 - precision, rv if precision == 64 else 0.0),
              c.solver(precision, rr + 0.25)]
    for kw in ({"tau": 0.9}, {"T_over_Tc": 0.81}, {"A": 0.0}, {"top": O.TOP_NOSLIP},
               {"kappa": O.KAPPA_LATTICE}, {"forcing": O.FORCING_GUO}):
        others.append(Case(45, 27, **kw).solver(precision, rr))
    for other in others:
        with pytest.raises(lbm.LbmError) as e:
            other.load(blob)
        assert e.value.code == lbm.ERR_INVALID_ARG
        with pytest.raises(lbm.LbmError) as e:
            other.save()
        assert e.value.code == lbm.ERR_STATE
        other.close()
    with pytest.raises(lbm.LbmError):
        b.load(blob[:100])
    a.close()
    b.close()


@pytest.mark.parametrize("path", ["fused", "split"])
@pytest.mark.parametrize("top", [O.TOP_FREESLIP, O.TOP_NOSLIP])
def test_link_midpoint_source_fp64(top, path):
    """h_eval = LINK_AVG against the oracle's link average, through the fused
    kernel's link form and the two-kernel path: a droplet from rest with a
    random flow, and the radial acoustic mode (single phase: two-kernel path)."""
    from scipy import special

    c = Case(45, 27, top=top, h_eval=O.H_LINK_AVG)
    fields = _droplet_fields(c, 10, du=2e-3, seed=31)
    o = O.Oracle(c.oracle_params()).init(*fields, physical=True).step(90)
    s = c.solver().init(*fields, physical=True)
    from paper_1512_01977_gb300 import lbm

    assert lbm.lbm_axi_get_tuning(s.h)[0] == lbm.PATH_FUSED
    if path == "split":
        lbm.lbm_axi_set_tuning(s.h, lbm.PATH_SPLIT, 0)
    s.step(90)
    mo, mg = o.moments(), s.moments()
    assert rel_err(mg["rho"], mo["rho"]) <= TOL64 and vel_err(mg, mo) <= TOL64 and rel_err(mg["p"], mo["p"]) <= TOL64
    assert mg["rho"].size and s.mass()[0] == pytest.approx(o.mass_rweighted(), rel=1e-12)
    s.close()
    c = Case(3, 32, multiphase=0, tau=0.8, top=top, h_eval=O.H_LINK_AVG)
    _compare(c, I.radial_mode(3, 32, 1.0, 1e-2, special.jn_zeros(1, 1)[0] / 32), 40)


def test_link_midpoint_source_limits():
    """A LINK_AVG solve refuses chunked fused grids and batches; its checkpoint
    carries the source planes (bitwise resume)."""
    from paper_1512_01977_gb300 import lbm

    c = Case(40, 24, h_eval=O.H_LINK_AVG)
    fields = _droplet_fields(c, 9, du=1e-3, seed=32)
    s = c.solver(32, c.coexistence()[0]).init(*fields, physical=True)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_axi_set_tuning(s.h, lbm.PATH_FUSED, 16)
    with pytest.raises(lbm.LbmError):
        lbm.Batch([s])
    s.step(11)
    blob = s.save()
    s.step(20)
    ref = s.moments()
    t = c.solver(32, c.coexistence()[0]).load(blob).step(20)
    np.testing.assert_array_equal(t.moments()["rho"], ref["rho"])
    # a LOCAL solve of the same grid refuses the blob
    u = Case(40, 24).solver(32, c.coexistence()[0])
    with pytest.raises(lbm.LbmError):
        u.load(blob)
    for x in (s, t, u):
        x.close()


def test_full_size_wave_sampled_windows_fp64():
    """The bench workload at full size (4096 x 2048) in FP64 through the same
    balanced tile plan: after 3 steps a node depends only on initial data
    within 7 per step (psi halo 6 + streaming 1), so the oracle reproduces
    windows of the lattice once their edges are farther away than that, here
    to the FP64 bar.  Windows: at the axis across the periodic z seam, in the
    bulk, at the free-slip top."""
    nz, nr, n_steps = 4096, 2048, 3
    c = Case(nz, nr, T_over_Tc=0.9, tau=0.6)
    _, rho0 = c.coexistence()
    rho, uz, ur = I.density_wave(nz, nr, rho0)
    _, vz, vr = I.random_state(nz, nr, 1.0, 0.0, 2e-3, 17)
    s = c.solver(precision=64)
    s.init(rho, vz, vr)
    s.step(n_steps)
    mg = s.moments()
    s.close()
    m = 7 * n_steps + 8
    wz, wr = 48, 40
    for (k0, j0, at_axis, at_top) in ((nz - 24, 0, True, False), (2500, 900, False, False),
                                      (3300, nr - wr, False, True)):
        ks = np.arange(k0 - m, k0 + wz + m) % nz
        lo = 0 if at_axis else j0 - m
        hi = nr if at_top else j0 + wr + m
        sub = lambda a: np.ascontiguousarray(a[lo:hi][:, ks])  # noqa: E731
        wc = Case(len(ks), hi - lo, T_over_Tc=0.9, tau=0.6, r0=float(lo))
        o = O.Oracle(wc.oracle_params()).init(sub(rho), sub(vz), sub(vr))
        o.step(n_steps)
        mo = o.moments()
        inner = (slice(0, wr) if at_axis else (slice(m, m + wr) if not at_top else slice(m, None)),
                 slice(m, m + wz))
        g = {k: mg[k][lo:hi][:, ks][inner] for k in ("rho", "uz", "ur", "p")}
        r = {k: mo[k][inner] for k in ("rho", "uz", "ur", "p")}
        _check(g, r)
