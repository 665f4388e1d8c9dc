"""ctypes binding of the FP64 CPU oracle (oracle/lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py, never by the library.
"""
import ctypes as C
import dataclasses

import numpy as np

from . import build as _build

Q = 9
TOP_FREESLIP, TOP_NOSLIP, TOP_PERIODIC = 0, 1, 2
EOS_VDW, EOS_CS = 0, 1
KAPPA_THERMO, KAPPA_LATTICE, KAPPA_MIXED = 0, 1, 2
H_LOCAL, H_LINK_AVG = 0, 1
FORCING_EDM, FORCING_GUO = 0, 1
ERR_UNPHYSICAL = -4


class _CParams(C.Structure):
    _fields_ = [
        ("nz", C.c_int), ("nr", C.c_int), ("tau", C.c_double), ("A", C.c_double),
        ("eos", C.c_int), ("T", C.c_double), ("a", C.c_double), ("b", C.c_double),
        ("R", C.c_double), ("lam", C.c_double), ("top", C.c_int), ("axis", C.c_int),
        ("multiphase", C.c_int), ("kappa", C.c_int), ("hr_sign", C.c_int), ("gz", C.c_double),
        ("r0", C.c_double), ("h_eval", C.c_int), ("forcing", C.c_int), ("axis_a", C.c_double),
    ]


@dataclasses.dataclass(frozen=True)
class Params:
    """Parameters of one solve.  T is the absolute EOS temperature."""

    nz: int = 1
    nr: int = 1
    tau: float = 1.0
    A: float = -0.152
    eos: int = EOS_CS
    T: float = 0.0
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    lam: float = 0.01
    top: int = TOP_FREESLIP
    axis: int = 1
    multiphase: int = 1
    kappa: int = KAPPA_THERMO
    hr_sign: int = -1
    gz: float = 0.0
    r0: float = 0.0
    h_eval: int = H_LOCAL
    forcing: int = FORCING_EDM
    axis_a: float = 6.0  # c of the c A psi_r grad psi / r term of F_axis (6 printed, 2 exact expansion)

    def replace(self, **kw):
        return dataclasses.replace(self, **kw)

    def c(self):
        return _CParams(*[getattr(self, f.name) for f in dataclasses.fields(self)])


_libs = {}
_D = C.POINTER(C.c_double)


def lib(omp=False):
    """The parity build of the oracle, or with omp=True the OpenMP timing build
    of the same source (bitwise the same results, all host cores)."""
    if omp not in _libs:
        L = C.CDLL(_build.build(omp=omp))
        P = C.POINTER(_CParams)
        sig = {
            "orc_eos_p": (C.c_double, [P, C.c_double]),
            "orc_eos_dpdrho": (C.c_double, [P, C.c_double]),
            "orc_feq": (None, [C.c_double, C.c_double, C.c_double, _D]),
            "orc_fill_ghosts": (None, [P, _D, C.c_int, C.c_int]),
            "orc_grad": (None, [P, _D, _D, _D]),
            "orc_force_kupershtokh": (None, [P, _D, _D, _D]),
            "orc_kappa": (C.c_double, [P, C.c_double]),
            "orc_force_axis": (None, [C.c_double] * 9 + [_D, _D]),
            "orc_source_H": (None, [C.c_double] * 8 + [C.c_int, _D, _D]),
            "orc_source_h": (None, [C.c_double] * 5 + [_D]),
            "orc_guo_source": (None, [C.c_double] * 5 + [_D]),
            "orc_stream_dest": (None, [P, C.c_int, C.c_int, C.c_int] + [C.POINTER(C.c_int)] * 3),
            "orc_stream": (None, [P, _D, _D]),
            "orc_run": (C.c_int, [P, _D, C.c_long]),
            "orc_init": (None, [P, _D, _D, _D, _D]),
            "orc_init_physical": (C.c_int, [P, _D, _D, _D, _D]),
            "orc_moments": (C.c_int, [P, _D] + [_D] * 8),
            "orc_collide_only": (C.c_int, [P, _D, _D]),
            "orc_mass_rweighted": (C.c_double, [P, _D]),
            "orc_ghost_width": (C.c_int, []),
            "orc_ext_index": (C.c_long, [P, C.c_int, C.c_int]),
            "orc_threads": (C.c_int, [C.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _libs[omp] = L
    return _libs[omp]


def threads(n=0, omp=True):
    """Set (n > 0) and return the thread count of the OpenMP build."""
    return lib(omp).orc_threads(int(n))


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


class OracleError(RuntimeError):
    pass


# ------------------------------------------------------------------ scalars --

def eos_p(params, rho):
    return lib().orc_eos_p(C.byref(params.c()), float(rho))


def eos_dpdrho(params, rho):
    return lib().orc_eos_dpdrho(C.byref(params.c()), float(rho))


def feq(rho, uz, ur):
    out = np.zeros(Q)
    lib().orc_feq(rho, uz, ur, _ptr(out))
    return out


def kappa(params, rho):
    return lib().orc_kappa(C.byref(params.c()), float(rho))


def force_axis(kappa_, A, r, psi, psi_z, psi_r, psi_rr, psi_rz, c=6.0):
    fz, fr = C.c_double(), C.c_double()
    lib().orc_force_axis(kappa_, A, c, r, psi, psi_z, psi_r, psi_rr, psi_rz, C.byref(fz), C.byref(fr))
    return fz.value, fr.value


def source_H(r, rho, mu, uz, ur, duz_dr, dur_dz, dur_dr, hr_sign):
    hz, hr = C.c_double(), C.c_double()
    lib().orc_source_H(r, rho, mu, uz, ur, duz_dr, dur_dz, dur_dr, hr_sign, C.byref(hz), C.byref(hr))
    return hz.value, hr.value


def source_h(r, rho, ur, Hz, Hr):
    out = np.zeros(Q)
    lib().orc_source_h(r, rho, ur, Hz, Hr, _ptr(out))
    return out


def guo_source(tau, uz, ur, Fz, Fr):
    out = np.zeros(Q)
    lib().orc_guo_source(tau, uz, ur, Fz, Fr, _ptr(out))
    return out


def stream_dest(params, k, j, i):
    kd, jd, idd = C.c_int(), C.c_int(), C.c_int()
    lib().orc_stream_dest(C.byref(params.c()), k, j, i, C.byref(kd), C.byref(jd), C.byref(idd))
    return kd.value, jd.value, idd.value


# ----------------------------------------------------------- ghosted fields --

def ghost_width():
    return lib().orc_ghost_width()


def ext_shape(params):
    g = ghost_width()
    return (params.nr + 2 * g, params.nz + 2 * g)


def ext_from_function(params, fn):
    """Extended field whose every node (ghosts included) holds fn(z_k, r_j),
    with z_k = k + 1/2 and r_j = j + 1/2 (k, j may be negative)."""
    g = ghost_width()
    nr_e, nz_e = ext_shape(params)
    k = np.arange(nz_e) - g
    j = np.arange(nr_e) - g
    Z, R = np.meshgrid(k + 0.5, j + 0.5)
    return np.ascontiguousarray(fn(Z, R), dtype=np.float64)


def interior(params, ext):
    g = ghost_width()
    return ext[g:g + params.nr, g:g + params.nz]


def fill_ghosts(params, ext, sign_axis, sign_top):
    lib().orc_fill_ghosts(C.byref(params.c()), _ptr(ext), sign_axis, sign_top)


def grad(params, ext):
    dz = np.zeros_like(ext)
    dr = np.zeros_like(ext)
    lib().orc_grad(C.byref(params.c()), _ptr(ext), _ptr(dz), _ptr(dr))
    return interior(params, dz).copy(), interior(params, dr).copy()


def force_kupershtokh(params, psi_ext):
    fz = np.zeros_like(psi_ext)
    fr = np.zeros_like(psi_ext)
    lib().orc_force_kupershtokh(C.byref(params.c()), _ptr(psi_ext), _ptr(fz), _ptr(fr))
    return interior(params, fz).copy(), interior(params, fr).copy()


# ---------------------------------------------------------------- the solve --

class Oracle:
    """One solve on the CPU: pre-collision populations f[9, nr, nz].
    omp=True steps with the OpenMP timing build (same results, all cores)."""

    def __init__(self, params, omp=False):
        self.params = params
        self.omp = omp
        self.f = np.zeros((Q, params.nr, params.nz))

    def init(self, rho, uz=None, ur=None, physical=False):
        """f = f^eq(rho, u).  physical=False: u is the bare velocity u0;
        physical=True: u is the fluid velocity u0 + F/(2 rho) (at rest for u = 0)."""
        p = self.params
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(p.nr, p.nz)
        uz = np.zeros_like(rho) if uz is None else np.ascontiguousarray(uz, dtype=np.float64).reshape(rho.shape)
        ur = np.zeros_like(rho) if ur is None else np.ascontiguousarray(ur, dtype=np.float64).reshape(rho.shape)
        if physical:
            rc = lib().orc_init_physical(C.byref(p.c()), _ptr(rho), _ptr(uz), _ptr(ur), _ptr(self.f))
            if rc != 0:
                raise OracleError("oracle init failed with code %d" % rc)
        else:
            lib().orc_init(C.byref(p.c()), _ptr(rho), _ptr(uz), _ptr(ur), _ptr(self.f))
        return self

    def step(self, n=1):
        rc = lib(self.omp).orc_run(C.byref(self.params.c()), _ptr(self.f), int(n))
        if rc != 0:
            raise OracleError("oracle step failed with code %d" % rc)
        return self

    def moments(self, diagnostics=False):
        p = self.params
        out = [np.zeros((p.nr, p.nz)) for _ in range(8)]
        rc = lib().orc_moments(C.byref(p.c()), _ptr(self.f), *[_ptr(a) for a in out])
        if rc != 0:
            raise OracleError("oracle moments failed with code %d" % rc)
        keys = ["rho", "uz", "ur", "p", "Fz", "Fr", "Hz", "Hr"]
        d = dict(zip(keys, out))
        if not diagnostics:
            for k in keys[4:]:
                d.pop(k)
        return d

    def collide_only(self):
        out = np.zeros_like(self.f)
        rc = lib().orc_collide_only(C.byref(self.params.c()), _ptr(self.f), _ptr(out))
        if rc != 0:
            raise OracleError("oracle collision failed with code %d" % rc)
        return out

    def mass_rweighted(self):
        return lib().orc_mass_rweighted(C.byref(self.params.c()), _ptr(self.f))

    def mass(self):
        return float(self.f.sum())
