"""FP64 CPU oracle of the axisymmetric multiphase D2Q9 update (arXiv:1512.01977).

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
leg of bench.py may import this package; the library never does, and the two
share no code.  The update itself is plain C (lbm_oracle.c); this package
binds it and adds the EOS helpers (critical point, Maxwell construction) and
the paper's analytic results used as pins (analytic.py).
"""
from .core import (  # noqa: F401
    EOS_CS, EOS_VDW, FORCING_EDM, FORCING_GUO, H_LINK_AVG, H_LOCAL, KAPPA_LATTICE, KAPPA_MIXED, KAPPA_THERMO, Oracle, OracleError, Params, Q, TOP_FREESLIP,
    TOP_NOSLIP, TOP_PERIODIC,
)
from . import analytic, core, eos  # noqa: F401


def make_params(nz, nr, tau, eos_kind, T_over_Tc, A=-0.152, **kw):
    """Params with the absolute EOS temperature computed from T/T_c."""
    p = Params(nz=nz, nr=nr, tau=tau, eos=eos_kind, A=A, **kw)
    Tc, _ = eos.critical_point(p)
    return p.replace(T=T_over_Tc * Tc)
