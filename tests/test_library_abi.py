"""CPU checks of the C ABI library: it loads without a GPU, exports every
function include/lbm_axi.h declares, and its host-side EOS helpers agree with
the oracle's independent ones."""
import os
import re

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    from paper_1512_01977_gb300 import build, lbm as L

    build.build()
    L.lib()
    return L


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lbm):
    L = lbm.lib()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name
    assert set(lbm.exported_symbols()) <= declared


def test_strerror_and_defaults(lbm):
    assert lbm.lbm_axi_strerror(0) == "ok"
    assert "unphysical" in lbm.lbm_axi_strerror(-4)
    o = lbm.lbm_axi_default_opts()
    assert (o.precision, o.top_bc, o.axis_terms, o.multiphase, o.kappa_mode, o.hr_sign) == (64, 0, 1, 1, 0, -1)


def test_footprint(lbm):
    # 2 x 9 population planes + 4 field planes (pitch 4096) + moments staging
    n = 4096 * 2048
    assert lbm.lbm_axi_footprint(4096, 2048, 32) >= (22 * 4 + 32) * n
    assert lbm.lbm_axi_footprint(4096, 2048, 64) >= (22 * 8 + 32) * n


@pytest.mark.parametrize("kind,T", [(O.EOS_CS, 0.5), (O.EOS_CS, 0.8), (O.EOS_CS, 0.9), (O.EOS_VDW, 0.7),
                                    (O.EOS_VDW, 0.9)])
def test_host_eos_matches_oracle(lbm, kind, T):
    p = O.make_params(8, 8, 1.0, kind, T, lam=0.01)
    rv, rl = O.eos.maxwell_densities(p)
    e = lbm.make_eos(kind, T, lam=0.01)
    gv, gl = lbm.lbm_eos_coexistence(e)
    assert gv == pytest.approx(rv, rel=1e-11)
    assert gl == pytest.approx(rl, rel=1e-11)
    Tc, _ = O.eos.critical_point(p)
    assert lbm.lbm_eos_critical_temperature(e) == pytest.approx(Tc, rel=1e-13)
    for rho in (0.5 * rv, rv, 0.5 * (rv + rl), rl):
        pg, dg = lbm.lbm_eos_pressure(e, rho)
        assert pg == pytest.approx(O.core.eos_p(p, rho), rel=1e-10, abs=1e-16)
        assert dg == pytest.approx(O.core.eos_dpdrho(p, rho), rel=1e-10, abs=1e-15)


def test_invalid_eos_rejected(lbm):
    with pytest.raises(lbm.LbmError):
        lbm.lbm_eos_coexistence(lbm.make_eos(O.EOS_CS, 1.2))


@pytest.mark.parametrize("nz,nr", [(16, 8388608), (1, 1 << 27), (4096, 1 << 16)])
def test_create_refuses_grids_beyond_32bit_offsets(lbm, nz, nr):
    """Grids whose population buffer (9 planes of pitch x nr, pitch = nz
    rounded up to 32) reaches 2^31 elements, or that exceed 2^27 nodes, are
    refused before any device call."""
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_axi_create(nz, nr, 1.0, lbm.make_eos(), -0.152)
    assert e.value.code == lbm.ERR_INVALID_ARG
