"""The oracle's two builds of one source: the parity build (one thread) and the
OpenMP timing build (all host cores) give bitwise the same populations, so a
CPU baseline timed with the second is the first's computation."""
import numpy as np
import pytest

import oracle as O
from oracle import core
from paper_1512_01977_gb300 import inputs as I


@pytest.mark.parametrize("forcing", [O.FORCING_EDM, O.FORCING_GUO])
def test_openmp_build_is_bitwise_the_parity_build(forcing):
    p = O.make_params(40, 33, 0.9, O.EOS_CS, 0.8, top=O.TOP_FREESLIP, forcing=forcing)
    rv, rl = O.eos.maxwell_densities(p)
    fields = I.droplet(40, 33, 9, rl, rv)
    a = O.Oracle(p).init(*fields, physical=True)
    b = O.Oracle(p, omp=True).init(*fields, physical=True)
    prev = core.threads(0)
    try:
        core.threads(4)
        a.step(25)
        b.step(25)
    finally:
        core.threads(prev)
    np.testing.assert_array_equal(a.f, b.f)


def test_openmp_build_reports_unphysical_states():
    p = O.make_params(16, 8, 1.0, O.EOS_CS, 0.8)
    rho = np.full((8, 16), 0.2)
    rho[3, 5] = -0.1
    o = O.Oracle(p, omp=True).init(rho)
    with pytest.raises(O.OracleError):
        o.step(2)
