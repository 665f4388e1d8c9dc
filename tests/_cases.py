"""Test cases expressed once and turned into both an oracle solve and a CUDA
solve with the same numbers.  Inputs come from paper_1512_01977_gb300.inputs;
coexistence densities for initial states come from the oracle."""
import dataclasses

import numpy as np

import oracle as O


@dataclasses.dataclass
class Case:
    nz: int
    nr: int
    tau: float = 1.0
    eos: int = O.EOS_CS
    T_over_Tc: float = 0.8
    A: float = -0.152
    lam: float = 0.01
    top: int = O.TOP_FREESLIP
    axis: int = 1
    multiphase: int = 1
    kappa: int = O.KAPPA_THERMO
    hr_sign: int = -1
    gz: float = 0.0
    r0: float = 0.0  # oracle only: radial offset of a window cut from a larger lattice
    h_eval: int = O.H_LOCAL
    forcing: int = O.FORCING_EDM
    axis_a: float = 6.0  # 6: F_axis A-term as printed; 2: from the exact expansion

    def oracle_params(self):
        p = O.Params(nz=self.nz, nr=self.nr, tau=self.tau, A=self.A, eos=self.eos, lam=self.lam, top=self.top,
                     axis=self.axis, multiphase=self.multiphase, kappa=self.kappa, hr_sign=self.hr_sign,
                     gz=self.gz, r0=self.r0, h_eval=self.h_eval, forcing=self.forcing,
                     axis_a=self.axis_a)
        Tc, _ = O.eos.critical_point(p)
        return p.replace(T=self.T_over_Tc * Tc)

    def coexistence(self):
        return O.eos.maxwell_densities(self.oracle_params())

    def solver(self, precision=64, rho_ref=0.0):
        from paper_1512_01977_gb300 import lbm

        eos = lbm.make_eos(self.eos, self.T_over_Tc, lam=self.lam) if self.multiphase else None
        return lbm.Solver(self.nz, self.nr, self.tau, eos=eos, A=self.A, precision=precision, top=self.top,
                          axis=self.axis, multiphase=self.multiphase, kappa=self.kappa, hr_sign=self.hr_sign,
                          rho_ref=rho_ref, g_z=self.gz, h_eval=self.h_eval, forcing=self.forcing,
                          axis_a_term=lbm.AXIS_A_EXPANSION if self.axis_a == 2.0 else lbm.AXIS_A_PRINTED)


def run_oracle(case, fields, steps):
    o = O.Oracle(case.oracle_params()).init(*fields)
    o.step(steps)
    return o


def run_gpu(case, fields, steps, precision=64, rho_ref=0.0, tuning=None):
    s = case.solver(precision, rho_ref)
    if tuning is not None:
        from paper_1512_01977_gb300 import lbm

        lbm.lbm_axi_set_tuning(s.h, *tuning)
    s.init(*fields)
    s.step(steps)
    return s


def rel_err(a, b):
    """max |a - b| / max |b| (b the reference)."""
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0))


# Lattice velocity scale below which velocity errors are measured absolutely.  A velocity is
# sum_i c_i f_i / rho over populations of size w_i rho, so its FP64 rounding error is absolute
# (about eps_64 = 1.1e-16 per evaluation in lattice units, grown over the steps), not relative
# to u: a flow of magnitude |u| cannot be reproduced to better than ~eps_64 / |u| relative.
# Below |u| = 1e-3 the bar 1e-12 becomes the absolute 1e-15, ten units of that rounding.
U_FLOOR = 1e-3


def vel_err(mg, mo):
    """max |u_gpu - u_oracle| (both components) / max(max |u_oracle|, U_FLOOR).

    Velocities are compared as a vector against their own scale; the floor
    keeps states whose velocity has decayed to round-off (or is zero by
    symmetry) from turning rounding noise into a large relative error."""
    du = max(np.max(np.abs(mg["uz"] - mo["uz"])), np.max(np.abs(mg["ur"] - mo["ur"])))
    umax = np.max(np.hypot(mo["uz"], mo["ur"]))
    return float(du / max(umax, U_FLOOR))


def component_errs(mg, mo):
    """Per velocity component c: max |u_gpu - u_oracle| / max(max |u_c|, U_FLOOR),
    i.e. relative to the component's own scale wherever that exceeds the
    rounding floor of a lattice velocity (a tighter check than vel_err for a
    component much slower than the other)."""
    out = {}
    for k in ("uz", "ur"):
        scale = max(float(np.max(np.abs(mo[k]))), U_FLOOR)
        out[k] = float(np.max(np.abs(mg[k] - mo[k])) / scale)
    return out
