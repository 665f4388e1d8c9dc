"""The allocation-free mass reduction (lbm_axi_mass_field_noalloc) against the
handle-based lbm_axi_mass, through the C ABI.

The entry point exists for callers that cannot let a library allocate device
memory for them (a fixed pre-reserved arena, a framework allocator that must
see every byte): its scratch is a static device array, and the caller owns the
input field and the output buffer.  This file is collected last so that a run
stopping at the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1512_01977_gb300 import inputs as I
from tests._cases import Case

pytestmark = pytest.mark.gpu

TOL_MASS = 1e-13  # the relative tolerance of the other FP64 mass checks


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_01977_gb300 import build, lbm as L

    build.build()
    L.lib()
    return L


def test_noalloc_mass_matches_lbm_axi_mass_twice(lbm):
    import torch

    c = Case(96, 64)
    rv, rl = c.coexistence()
    s = c.solver()
    s.init(*I.droplet(96, 64, 20, rl, rv))
    s.step(40)
    ref_rw, ref_plain = s.mass()

    # caller-owned input (the density field on the device) and output buffer
    d_rho = torch.empty(96 * 64, dtype=torch.float64, device="cuda")
    lbm.lbm_axi_moments_device(s.h, rho=d_rho)
    torch.cuda.synchronize()
    d_out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    for _ in range(2):  # the second call reuses the static scratch left by the first
        d_out.fill_(float("nan"))
        torch.cuda.synchronize()
        lbm.lbm_axi_mass_field_noalloc(d_rho, 96, 64, d_out, stream)
        stream.synchronize()
        got = d_out.cpu().numpy()
        assert got[0] == pytest.approx(ref_rw, rel=TOL_MASS)
        assert got[1] == pytest.approx(ref_plain, rel=TOL_MASS)
    s.close()


def test_noalloc_mass_on_another_field_size(lbm):
    """A smaller field after a larger one: only the launched blocks' partial
    slots are read, so the stale contents of the others never leak in."""
    import torch

    for nz, nr in ((4096, 2048), (33, 17)):
        rho = np.random.default_rng(nz).uniform(0.1, 1.0, size=nz * nr)
        d_rho = torch.tensor(rho, dtype=torch.float64, device="cuda")
        d_out = torch.empty(2, dtype=torch.float64, device="cuda")
        lbm.lbm_axi_mass_field_noalloc(d_rho, nz, nr, d_out, None)
        torch.cuda.synchronize()
        j = np.repeat(np.arange(nr) + 0.5, nz)
        got = d_out.cpu().numpy()
        assert got[0] == pytest.approx(float(np.sum(j * rho)), rel=TOL_MASS)
        assert got[1] == pytest.approx(float(np.sum(rho)), rel=TOL_MASS)


def test_noalloc_rejects_fields_beyond_the_maximum(lbm):
    import torch

    d_rho = torch.zeros(16, dtype=torch.float64, device="cuda")
    d_out = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = lbm.lib().lbm_axi_mass_field_noalloc(C.c_void_p(d_rho.data_ptr()), 4096, 2049,
                                              C.c_void_p(d_out.data_ptr()), None)
    assert rc == lbm.ERR_INVALID_ARG
    with pytest.raises(lbm.LbmError, match="exceeds the maximum"):
        lbm.lbm_axi_mass_field_noalloc(d_rho, 4097, 2048, d_out)
