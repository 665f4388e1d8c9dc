"""Batched stepping (include/lbm_axi_batch.h): one launch advances many solves.

No arithmetic couples two solves and the per-node arithmetic of the fused
kernel does not depend on the strip width or on how the rows are cut, so a
solve's state after n batched steps is bitwise the state after n steps alone.
"""
import numpy as np
import pytest

import oracle as O
from paper_1512_01977_gb300 import inputs as I
from tests._cases import Case, component_errs, rel_err, run_oracle, vel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_01977_gb300 import build, lbm as L

    build.build()
    L.lib()
    return L


def _mix(seed=4, n=7, precision=64):
    """Droplets of uneven sizes and temperatures (the batched workload's size
    recipe, scaled down to 40x24 .. 120x72, at stable T = 0.85-0.89 T_c)."""
    specs = I.batch_droplets(n=n, seed=seed, lo=(40, 24), scale_max=3.0)
    out = []
    for sp in specs:
        c = Case(sp["nz"], sp["nr"], tau=1.0, T_over_Tc=0.8 + 0.1 * sp["T_over_Tc"])
        rv, rl = c.coexistence()
        fields = I.droplet(c.nz, c.nr, sp["R"], rl, rv)
        out.append((c, fields, rv if precision == 32 else 0.0))
    return out


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("strip", [64, 112])
def test_batch_equals_alone(lbm, precision, strip):
    """Same arithmetic alone (the single-solve form, strip 112) and in the batch:
    bitwise equal at strip 112; with strip 64 (another compiled form) FP32
    may differ in the last bits (FMA contraction), bounded here by 1e-6."""
    mix = _mix(precision=precision)
    alone = []
    for c, fields, rr in mix:
        s = c.solver(precision, rr).init(*fields)
        s.step(37)
        alone.append(s.moments())
        s.close()
    solvers = [c.solver(precision, rr).init(*fields) for c, fields, rr in mix]
    b = lbm.Batch(solvers)
    lbm.lbm_axi_batch_set_tuning(b.b, strip, 0)
    assert b.step(37) == lbm.OK
    assert b.status() == [lbm.OK] * len(solvers)
    for s, ref in zip(solvers, alone):
        m = s.moments()
        if strip == 112 or precision == 64:
            for k in ("rho", "uz", "ur", "p"):
                np.testing.assert_array_equal(m[k], ref[k])
        else:
            assert rel_err(m["rho"], ref["rho"]) <= 1e-6 and vel_err(m, ref) <= 1e-6
    b.close()
    for s in solvers:
        s.close()


def test_large_fp32_batch_equals_alone(lbm):
    """An FP32 batch of 260 solves, more than one kernel-argument table holds
    (256): the batched kernel then reads the descriptors from a device table;
    every solve still equals its run alone, bitwise."""
    n = 260
    specs = I.batch_droplets(n=n, seed=9, lo=(24, 16), scale_max=1.6)
    cases = []
    for sp in specs:
        c = Case(sp["nz"], sp["nr"], tau=1.0, T_over_Tc=0.85)
        rv, rl = c.coexistence()
        cases.append((c, I.droplet(c.nz, c.nr, min(sp["R"], 6.0), rl, rv), rv))
    solvers = [c.solver(32, rr).init(*fields) for c, fields, rr in cases]
    b = lbm.Batch(solvers)
    assert b.step(21) == lbm.OK
    assert b.status() == [lbm.OK] * n
    b.close()
    for k in range(0, n, 37):
        c, fields, rr = cases[k]
        s = c.solver(32, rr).init(*fields)
        s.step(21)
        ref = s.moments()
        s.close()
        m = solvers[k].moments()
        for key in ("rho", "uz", "ur", "p"):
            np.testing.assert_array_equal(m[key], ref[key])
    for s in solvers:
        s.close()


@pytest.mark.parametrize("strip", [64, 112])
def test_batch_fp64_matches_oracle(lbm, strip):
    """An FP64 batch whose mix holds grids wider than one strip (up to 230
    columns: several strips and a ragged last one) against the oracle."""
    mix = _mix(seed=11, n=4)
    for nz, nr in ((230, 30), (131, 41)):
        c = Case(nz, nr, tau=1.0, T_over_Tc=0.85)
        rv, rl = c.coexistence()
        rho, _, _ = I.droplet(nz, nr, 10, rl, rv)
        rho = np.maximum(rho, np.roll(rho, nz // 2, axis=1))
        _, vz, vr = I.random_state(nz, nr, 1.0, 0.0, 1e-3, nz)
        mix.append((c, (rho, vz, vr * (np.arange(nr) + 0.5)[:, None] / nr), 0.0))
    solvers = [c.solver().init(*fields) for c, fields, _ in mix]
    b = lbm.Batch(solvers)
    lbm.lbm_axi_batch_set_tuning(b.b, strip, 0)
    b.step(60)
    for (c, fields, _), s in zip(mix, solvers):
        mo = run_oracle(c, fields, 60).moments()
        mg = s.moments()
        assert rel_err(mg["rho"], mo["rho"]) <= 1e-12
        assert vel_err(mg, mo) <= 1e-12
        for k, e in component_errs(mg, mo).items():
            assert e <= 1e-12, (c.nz, c.nr, k, e)
    b.close()
    for s in solvers:
        s.close()


def test_failed_solve_is_isolated(lbm):
    """A solve that goes unphysical is reported through its own status; the
    others keep their alone results bit for bit."""
    mix = _mix(seed=5, n=4)
    refs = []
    for c, fields, _ in mix:
        s = c.solver().init(*fields)
        s.step(20)
        refs.append(s.moments())
        s.close()
    solvers = [c.solver().init(*fields) for c, fields, _ in mix]
    bad_c = Case(40, 20)
    rho = np.full((20, 40), 0.2)
    rho[5, 7] = -0.1
    bad = bad_c.solver().init(rho)
    b = lbm.Batch(solvers[:2] + [bad] + solvers[2:])
    assert b.step(20) == lbm.ERR_UNPHYSICAL
    st = b.status()
    assert st[2] == lbm.ERR_UNPHYSICAL and st.count(lbm.OK) == 4
    for s, ref in zip(solvers, refs):
        m = s.moments()
        np.testing.assert_array_equal(m["rho"], ref["rho"])
    b.close()
    for s in solvers + [bad]:
        s.close()


def test_autotuners_are_non_destructive(lbm):
    mix = _mix(seed=6, n=5)
    ref = []
    for c, fields, _ in mix:
        s = c.solver().init(*fields)
        s.step(25)
        ref.append(s.moments()["rho"])
        s.close()
    solvers = [c.solver().init(*fields) for c, fields, _ in mix]
    b = lbm.Batch(solvers)
    b.step(10)
    strip, grid = b.autotune(trials=3)
    assert strip in (64, 112)
    b.step(15)
    for s, r in zip(solvers, ref):
        np.testing.assert_array_equal(s.moments()["rho"], r)
    b.close()
    # single-solve autotuner
    c, fields, _ = mix[0]
    s = c.solver().init(*fields)
    s.step(10)
    path, rows = lbm.lbm_axi_autotune(s.h, trials=3)
    assert path in (lbm.PATH_FUSED, lbm.PATH_SPLIT)
    s.step(15)
    np.testing.assert_allclose(s.moments()["rho"], ref[0], rtol=1e-13)  # paths agree to rounding
    s.close()
    for x in solvers:
        x.close()


def test_batch_rejects_mismatched_solves(lbm):
    a = Case(32, 20).solver(64).init(np.full((20, 32), 0.3))
    f32 = Case(32, 20).solver(32).init(np.full((20, 32), 0.3))
    thin = Case(32, 8).solver(64).init(np.full((8, 32), 0.3))
    for group in ([a, f32], [a, thin], [a, a]):
        with pytest.raises(lbm.LbmError):
            lbm.Batch(group)
    for s in (a, f32, thin):
        s.close()


def test_failed_solve_stays_failed_and_skipped(lbm):
    """Once a solve goes unphysical the batched kernel leaves it alone: its
    status stays failed through further steps and an autotune (whose trial
    launches do not clear it), and the other solves keep their alone results
    bit for bit."""
    mix = _mix(seed=8, n=3)
    refs = []
    for c, fields, _ in mix:
        s = c.solver().init(*fields)
        s.step(40)
        refs.append(s.moments()["rho"])
        s.close()
    solvers = [c.solver().init(*fields) for c, fields, _ in mix]
    bad_c = Case(40, 20)
    rho = np.full((20, 40), 0.2)
    rho[5, 7] = -0.1
    bad = bad_c.solver().init(rho)
    b = lbm.Batch([bad] + solvers)
    assert b.step(10) == lbm.ERR_UNPHYSICAL
    b.autotune(trials=2)
    assert b.status()[0] == lbm.ERR_UNPHYSICAL
    b.step(30)
    st = b.status()
    assert st[0] == lbm.ERR_UNPHYSICAL and st[1:] == [lbm.OK] * 3
    for s, r in zip(solvers, refs):
        np.testing.assert_array_equal(s.moments()["rho"], r)
    b.close()
    for s in solvers + [bad]:
        s.close()
