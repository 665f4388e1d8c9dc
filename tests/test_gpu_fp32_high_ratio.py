"""FP32 error at density ratios of about 10^3, stated per result.

The FP32 path stores populations as deviations f_i - w_i rho_ref and computes
in FP32; the r-weighted mass is reduced in FP64.  At a density ratio of 10^3
the choice of rho_ref decides which phase keeps its resolution: a vapour
stored against rho_ref = rho_l keeps only about eps_32 rho_l / rho_v of
relative resolution.  Each result is measured against the FP64 GPU path on
the same input (the FP64 path matches the oracle within 1e-12, see
test_gpu_parity.py):

* Fig. 2's flat interface (vdW, lambda = 0.01, A = -0.152, 150 x 100, tau = 1,
  40000 steps from rest) at 0.35, 0.4 and 0.5 T_c (density ratios 1549, 770,
  113 -- the paper's "10^3 and beyond"), with rho_ref = rho_v and rho_ref = rho_l:
  relative density error of each phase, velocity error, r-weighted mass drift.
* The mode-2 droplet of a Carnahan-Starling fluid at 0.5 T_c (ratio about
  725): 512 x 256, tau = 0.8, A = -0.152, R0 = 64 with a P2(cos theta)
  perturbation of 0.05 R0, started at rest, 40000 steps: oscillation period
  of the axis extent, density and mass drift, FP32 against FP64.

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


def _slab(lbm, T, precision, rho_ref, steps=40000):
    eos = lbm.make_eos(lbm.EOS_VDW, T, lam=LAM)
    rv, rl = lbm.lbm_eos_coexistence(eos)
    s = lbm.Solver(150, 100, 1.0, eos=eos, A=-0.152, precision=precision, rho_ref=rho_ref)
    s.init(*I.slab(150, 100, rl, rv, width=4.0), physical=True)
    m0 = s.mass()[0]
    s.step(steps)
    m = s.moments()
    drift = s.mass()[0] / m0 - 1
    s.close()
    return m, drift, rv, rl


def _crossings(row, mid):
    """z positions (k + 1/2) where a row crosses `mid`, by linear interpolation."""
    z = np.arange(len(row)) + 0.5
    out = []
    for k in range(len(row) - 1):
        a, b = row[k] - mid, row[k + 1] - mid
        if a == 0 or a * b < 0:
            out.append(z[k] + a / (a - b))
    return np.array(out)


def _slab_metrics(m, rv, rl):
    rho = m["rho"]
    z = np.arange(rho.shape[1]) + 0.5
    core = np.abs(z - 75) < 20
    far = np.abs(z - 75) > 60
    return rho[:, core].mean(), rho[:, far].mean(), _crossings(rho[0], 0.5 * (rl + rv))


# rho_ref -> bars (liquid plateau, vapour plateau, interface shift in nodes, |u_32 - u_64| in
# lattice units, |mass drift_32 - mass drift_64|), about 3x the largest of the three temperatures
# measured on a GB300 (rho_v: 5.8e-7, 9.5e-6, 0.028, 2.8e-6, 2.0e-4; rho_l: 3.1e-7, 9.7e-4, 0.13,
# 4.5e-4, 1.7e-4).  The mass drift, ~5e-9 per step, is FP32 rounding that repeats identically at
# every node of a uniform plateau (the same operands everywhere), so it does not average out.
SLAB_BARS = {
    "rho_v": (2e-6, 3e-5, 0.1, 1e-5, 6e-4),
    "rho_l": (1e-6, 3e-3, 0.4, 1.5e-3, 6e-4),
}


@pytest.mark.parametrize("ref", ["rho_v", "rho_l"])
@pytest.mark.parametrize("T", [0.35, 0.4, 0.5])
def test_fig2_slab_fp32_vs_fp64(lbm, T, ref):
    """Flat interface at density ratio 10^2..10^3: the plateau densities, the
    interface position, the spurious velocity and the r-weighted mass drift of
    FP32 against FP64."""
    m64, d64, rv, rl = _slab(lbm, T, 64, 0.0)
    m32, d32, _, _ = _slab(lbm, T, 32, rv if ref == "rho_v" else rl)
    l64, v64, x64 = _slab_metrics(m64, rv, rl)
    l32, v32, x32 = _slab_metrics(m32, rv, rl)
    e_l, e_v = abs(l32 / l64 - 1), abs(v32 / v64 - 1)
    assert len(x64) == len(x32) == 2
    e_x = float(np.max(np.abs(x32 - x64)))
    e_u = float(np.max(np.hypot(m32["uz"] - m64["uz"], m32["ur"] - m64["ur"])))
    umax = float(np.max(np.hypot(m64["uz"], m64["ur"])))
    print("FP32 slab T %.2f (plateau ratio %.0f) rho_ref %s: liquid %.2e, vapour %.2e, interface %.2e nodes, "
          "|du| %.2e (FP64 max|u| %.1e), mass drift FP64 %.1e FP32 %.1e"
          % (T, l64 / v64, ref, e_l, e_v, e_x, e_u, umax, d64, d32))
    bl, bv, bx, bu, bm = SLAB_BARS[ref]
    assert e_l <= bl and e_v <= bv and e_x <= bx and e_u <= bu and abs(d32 - d64) <= bm


def _c2_droplet(lbm, precision, steps=40000, every=100):
    """The mode-2 droplet at the high-ratio settings; the axis half-extent
    every `every` steps (crossings of (rho_l + rho_v)/2 on row 0)."""
    nz, nr, tau, A, R0 = 512, 256, 0.8, -0.152, 64.0
    eos = lbm.make_eos(lbm.EOS_CS, 0.5)
    rv, rl = lbm.lbm_eos_coexistence(eos)
    s = lbm.Solver(nz, nr, tau, eos=eos, A=A, precision=precision, rho_ref=rv if precision == 32 else 0.0)
    s.init(*I.droplet(nz, nr, R0, rl, rv, eps=0.05), physical=True)
    m0 = s.mass()[0]
    ext, failed = [], None
    mid = 0.5 * (rl + rv)
    for i in range(steps // every):
        x = _crossings(lbm.lbm_axi_moments(s.h, nz, nr, want=("rho",))["rho"][0], mid)
        ext.append(0.5 * (x[-1] - x[0]))
        try:
            s.step(every)
        except lbm.LbmError as e:
            failed = (i * every, e.code)
            break
    m = s.moments() if failed is None else None
    drift = s.mass()[0] / m0 - 1 if failed is None else float("nan")
    s.close()
    return np.array(ext), m, drift, failed, (rv, rl)


def test_c2_high_ratio_droplet_fp32_vs_fp64(lbm):
    """CS 0.5 T_c, 512 x 256, tau = 0.8, P2 perturbation 0.05, 40000 steps, from
    rest, FP64 and FP32 (deviations about rho_v).  Both runs complete; FP32
    against FP64: oscillation period of the axis extent within 1e-3 (measured
    1.9e-4), mean extent within 0.05 node (5e-3), liquid-core and far-vapour
    densities within 1e-3 (5.5e-5, 1.4e-5), r-weighted mass drift within
    5e-4 of FP64's (1.4e-4; FP64 itself drifts -2.8e-4 over the run, the
    scheme's r-weighted mass budget at spurious currents of 0.026)."""
    e64, m64, d64, f64, (rv, rl) = _c2_droplet(lbm, 64)
    e32, m32, d32, f32, _ = _c2_droplet(lbm, 32)
    print("C2 droplet: FP64 failed %s, FP32 failed %s" % (f64, f32))
    assert f64 is None and f32 is None
    t = np.arange(len(e64)) * 100.0
    sel = slice(5, None)
    w64, c64 = O.analytic.fit_damped_cosine(t[sel], e64[sel])
    w32, c32 = O.analytic.fit_damped_cosine(t[sel], e32[sel], w_guess=w64)
    Z, Rr = I.grid(512, 256)
    d = np.hypot(Z - 256, Rr)
    core, far = d < 32, d > 150
    l64, l32 = m64["rho"][core].mean(), m32["rho"][core].mean()
    v64, v32 = m64["rho"][far].mean(), m32["rho"][far].mean()
    umax = float(np.max(np.hypot(m64["uz"], m64["ur"])))
    print("C2 droplet (ratio %.0f): period FP64 %.2f FP32 %.2f steps (rel %.2e), mean half-extent FP64 %.4f "
          "FP32 %.4f, liquid core %.2e, far vapour %.2e, max|u| FP64 %.3f, mass drift FP64 %.2e FP32 %.2e"
          % (l64 / v64, 2 * np.pi / w64, 2 * np.pi / w32, w64 / w32 - 1, e64.mean(), e32.mean(),
             abs(l32 / l64 - 1), abs(v32 / v64 - 1), umax, d64, d32))
    assert abs(w64 / w32 - 1) <= 1e-3
    assert abs(e64.mean() - e32.mean()) <= 0.05
    assert abs(l32 / l64 - 1) <= 1e-3 and abs(v32 / v64 - 1) <= 1e-3
    assert abs(d32 - d64) <= 5e-4
