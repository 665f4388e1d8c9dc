"""ctypes binding of the C ABI in include/lbm_axi.h (argument marshalling only).

Every step of the update runs in the CUDA kernels of liblbm_axi.so; this module
converts numpy arrays and torch tensors to pointers and raises LbmError on a
non-zero return code.  There is no fallback: if the compiled library is
missing, loading fails with an error that says how to build it.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm_axi.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_UNPHYSICAL, ERR_TIMEOUT, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
EOS_VDW, EOS_CS = 0, 1
TOP_FREESLIP, TOP_NOSLIP, TOP_PERIODIC = 0, 1, 2
KAPPA_THERMO, KAPPA_LATTICE, KAPPA_MIXED = 0, 1, 2


class lbm_eos(C.Structure):
    _fields_ = [("kind", C.c_int), ("T_over_Tc", C.c_double), ("a", C.c_double), ("b", C.c_double),
                ("R", C.c_double), ("lam", C.c_double)]


class lbm_axi_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("top_bc", C.c_int), ("axis_terms", C.c_int), ("multiphase", C.c_int),
                ("kappa_mode", C.c_int), ("hr_sign", C.c_int), ("rho_ref", C.c_double), ("g_z", C.c_double),
                ("stream", C.c_void_p), ("h_eval", C.c_int), ("forcing", C.c_int), ("axis_a_term", C.c_int)]


H_LOCAL, H_LINK_AVG = 0, 1
FORCING_EDM, FORCING_GUO = 0, 1
AXIS_A_PRINTED, AXIS_A_EXPANSION = 0, 1


PATH_FUSED, PATH_SPLIT = 1, 2


class lbm_axi_tuning(C.Structure):
    _fields_ = [("path", C.c_int), ("rows_per_cta", C.c_int)]


class lbm_axi_batch_tuning(C.Structure):
    _fields_ = [("strip", C.c_int), ("grid", C.c_int)]


class LbmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, lbm_axi_strerror(code), code))


_D = C.POINTER(C.c_double)
_H = C.c_void_p
_lib = None

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_SIGS = {
    "lbm_axi_default_opts": (None, [C.POINTER(lbm_axi_opts)]),
    "lbm_axi_create": (C.c_int, [C.c_int, C.c_int, C.c_double, C.POINTER(lbm_eos), C.c_double,
                                 C.POINTER(lbm_axi_opts), C.POINTER(_H)]),
    "lbm_axi_init": (C.c_int, [_H, _D, _D, _D]),
    "lbm_axi_init_device": (C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_axi_init_physical": (C.c_int, [_H, _D, _D, _D]),
    "lbm_axi_init_physical_device": (C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_axi_step": (C.c_int, [_H, C.c_longlong]),
    "lbm_axi_step_async": (C.c_int, [_H, C.c_longlong]),
    "lbm_axi_sync": (C.c_int, [_H]),
    "lbm_axi_time_kernels": (C.c_int, [_H, C.c_longlong, _D]),
    "lbm_axi_moments": (C.c_int, [_H, _D, _D, _D, _D]),
    "lbm_axi_moments_device": (C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_axi_mass": (C.c_int, [_H, _D, _D]),
    "lbm_axi_state_bytes": (C.c_int, [_H, C.POINTER(C.c_size_t)]),
    "lbm_axi_save": (C.c_int, [_H, C.c_void_p, C.c_size_t]),
    "lbm_axi_load": (C.c_int, [_H, C.c_void_p, C.c_size_t]),
    "lbm_axi_pressure_jump": (C.c_int, [_H, C.c_double, C.c_double, C.c_double, C.c_double, _D]),
    "lbm_axi_destroy": (None, [_H]),
    "lbm_axi_temperature": (C.c_int, [_H, _D, _D]),
    "lbm_axi_get_tuning": (C.c_int, [_H, C.POINTER(lbm_axi_tuning)]),
    "lbm_axi_set_tuning": (C.c_int, [_H, C.POINTER(lbm_axi_tuning)]),
    "lbm_axi_device_bytes": (C.c_int, [_H, C.POINTER(C.c_size_t)]),
    "lbm_axi_footprint": (C.c_size_t, [C.c_int, C.c_int, C.c_int]),
    "lbm_eos_critical_temperature": (C.c_int, [C.POINTER(lbm_eos), _D]),
    "lbm_eos_coexistence": (C.c_int, [C.POINTER(lbm_eos), _D, _D]),
    "lbm_eos_pressure": (C.c_int, [C.POINTER(lbm_eos), C.c_double, _D, _D]),
    "lbm_axi_set_allocator": (C.c_int, [ALLOC_FN, RELEASE_FN, C.c_void_p]),
    "lbm_axi_strerror": (C.c_char_p, [C.c_int]),
    "lbm_axi_mass_field_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    # include/lbm_axi_batch.h
    "lbm_axi_batch_create": (C.c_int, [C.POINTER(_H), C.c_int, C.c_void_p, C.POINTER(_H)]),
    "lbm_axi_batch_step": (C.c_int, [_H, C.c_longlong]),
    "lbm_axi_batch_step_async": (C.c_int, [_H, C.c_longlong]),
    "lbm_axi_batch_sync": (C.c_int, [_H]),
    "lbm_axi_batch_status": (C.c_int, [_H, C.POINTER(C.c_int)]),
    "lbm_axi_batch_steps": (C.c_int, [_H, C.POINTER(C.c_longlong)]),
    "lbm_axi_batch_get_tuning": (C.c_int, [_H, C.POINTER(lbm_axi_batch_tuning)]),
    "lbm_axi_batch_set_tuning": (C.c_int, [_H, C.POINTER(lbm_axi_batch_tuning)]),
    "lbm_axi_batch_autotune": (C.c_int, [_H, C.c_int, C.POINTER(lbm_axi_batch_tuning)]),
    "lbm_axi_autotune": (C.c_int, [_H, C.c_int, C.POINTER(lbm_axi_tuning)]),
    "lbm_axi_batch_destroy": (None, [_H]),
    "lbm_axi_tile_plan": (C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                    C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
}

NOALLOC_MAX_NODES = 8388608


def lib():
    """Load liblbm_axi.so (built by __graft_entry__.build() or
    paper_1512_01977_gb300/build.py).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("liblbm_axi.so not found at %s; build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(code, where):
    if code != OK:
        raise LbmError(code, where)


def _dptr(a):
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("expected a C-contiguous float64 numpy array")
    return a.ctypes.data_as(_D)


def _host(a, n):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size != n:
        raise ValueError("array of %d values, expected nz*nr = %d" % (a.size, n))
    return a


def _devptr(t):
    """Device pointer of a contiguous float64 CUDA tensor (or None)."""
    if t is None:
        return None
    import torch

    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


# ------------------------------------------------------------ C ABI names --

def lbm_axi_strerror(code):
    return lib().lbm_axi_strerror(code).decode()


def lbm_axi_default_opts():
    o = lbm_axi_opts()
    lib().lbm_axi_default_opts(C.byref(o))
    return o


def make_eos(kind=EOS_CS, T_over_Tc=0.8, a=1.0, b=4.0, R=1.0, lam=0.01):
    return lbm_eos(kind, T_over_Tc, a, b, R, lam)


def lbm_axi_create(nz, nr, tau, eos, A, opts=None):
    h = _H()
    rc = lib().lbm_axi_create(int(nz), int(nr), float(tau), C.byref(eos) if eos is not None else None, float(A),
                              C.byref(opts) if opts is not None else None, C.byref(h))
    _check(rc, "lbm_axi_create")
    return h


def lbm_axi_init(h, nz, nr, rho, u_z=None, u_r=None):
    n = nz * nr
    rho, u_z, u_r = _host(rho, n), _host(u_z, n), _host(u_r, n)
    _check(lib().lbm_axi_init(h, _dptr(rho), _dptr(u_z), _dptr(u_r)), "lbm_axi_init")


def lbm_axi_init_device(h, rho, u_z=None, u_r=None):
    _check(lib().lbm_axi_init_device(h, _devptr(rho), _devptr(u_z), _devptr(u_r)), "lbm_axi_init_device")


def lbm_axi_init_physical(h, nz, nr, rho, u_z=None, u_r=None):
    n = nz * nr
    rho, u_z, u_r = _host(rho, n), _host(u_z, n), _host(u_r, n)
    _check(lib().lbm_axi_init_physical(h, _dptr(rho), _dptr(u_z), _dptr(u_r)), "lbm_axi_init_physical")


def lbm_axi_init_physical_device(h, rho, u_z=None, u_r=None):
    _check(lib().lbm_axi_init_physical_device(h, _devptr(rho), _devptr(u_z), _devptr(u_r)),
           "lbm_axi_init_physical_device")


def lbm_axi_step(h, n):
    _check(lib().lbm_axi_step(h, int(n)), "lbm_axi_step")


def lbm_axi_step_async(h, n):
    _check(lib().lbm_axi_step_async(h, int(n)), "lbm_axi_step_async")


def lbm_axi_sync(h):
    _check(lib().lbm_axi_sync(h), "lbm_axi_sync")


def lbm_axi_time_kernels(h, n):
    """Summed device milliseconds of the n kernel-(a) and n kernel-(b) launches."""
    ms = (C.c_double * 2)()
    _check(lib().lbm_axi_time_kernels(h, int(n), ms), "lbm_axi_time_kernels")
    return ms[0], ms[1]


def lbm_axi_moments(h, nz, nr, want=("rho", "u_z", "u_r", "p")):
    out = {k: np.empty(nz * nr) for k in ("rho", "u_z", "u_r", "p") if k in want}
    rc = lib().lbm_axi_moments(h, *[_dptr(out.get(k)) for k in ("rho", "u_z", "u_r", "p")])
    _check(rc, "lbm_axi_moments")
    return {k: v.reshape(nr, nz) for k, v in out.items()}


def lbm_axi_moments_device(h, rho=None, u_z=None, u_r=None, p=None):
    _check(lib().lbm_axi_moments_device(h, _devptr(rho), _devptr(u_z), _devptr(u_r), _devptr(p)),
           "lbm_axi_moments_device")


def lbm_axi_mass(h):
    mr, m = C.c_double(), C.c_double()
    _check(lib().lbm_axi_mass(h, C.byref(mr), C.byref(m)), "lbm_axi_mass")
    return mr.value, m.value


def lbm_axi_state_bytes(h):
    n = C.c_size_t()
    _check(lib().lbm_axi_state_bytes(h, C.byref(n)), "lbm_axi_state_bytes")
    return n.value


def lbm_axi_save(h):
    """The solve's state as a bytes object (header + populations)."""
    n = lbm_axi_state_bytes(h)
    buf = C.create_string_buffer(n)
    _check(lib().lbm_axi_save(h, buf, n), "lbm_axi_save")
    return buf.raw


def lbm_axi_load(h, blob):
    blob = bytes(blob)
    _check(lib().lbm_axi_load(h, blob, len(blob)), "lbm_axi_load")


def lbm_axi_pressure_jump(h, z_c, r_c, r_in, r_out):
    dp = C.c_double()
    _check(lib().lbm_axi_pressure_jump(h, z_c, r_c, r_in, r_out, C.byref(dp)), "lbm_axi_pressure_jump")
    return dp.value


def lbm_axi_destroy(h):
    lib().lbm_axi_destroy(h)


def lbm_axi_temperature(h):
    T, Tc = C.c_double(), C.c_double()
    _check(lib().lbm_axi_temperature(h, C.byref(T), C.byref(Tc)), "lbm_axi_temperature")
    return T.value, Tc.value


def lbm_axi_get_tuning(h):
    t = lbm_axi_tuning()
    _check(lib().lbm_axi_get_tuning(h, C.byref(t)), "lbm_axi_get_tuning")
    return t.path, t.rows_per_cta


def lbm_axi_set_tuning(h, path, rows_per_cta):
    t = lbm_axi_tuning(path, rows_per_cta)
    _check(lib().lbm_axi_set_tuning(h, C.byref(t)), "lbm_axi_set_tuning")


def lbm_axi_device_bytes(h):
    b = C.c_size_t()
    _check(lib().lbm_axi_device_bytes(h, C.byref(b)), "lbm_axi_device_bytes")
    return b.value


def lbm_axi_footprint(nz, nr, precision):
    return lib().lbm_axi_footprint(nz, nr, precision)


def lbm_eos_critical_temperature(eos):
    Tc = C.c_double()
    _check(lib().lbm_eos_critical_temperature(C.byref(eos), C.byref(Tc)), "lbm_eos_critical_temperature")
    return Tc.value


def lbm_eos_coexistence(eos):
    rv, rl = C.c_double(), C.c_double()
    _check(lib().lbm_eos_coexistence(C.byref(eos), C.byref(rv), C.byref(rl)), "lbm_eos_coexistence")
    return rv.value, rl.value


def lbm_eos_pressure(eos, rho):
    p, dp = C.c_double(), C.c_double()
    _check(lib().lbm_eos_pressure(C.byref(eos), float(rho), C.byref(p), C.byref(dp)), "lbm_eos_pressure")
    return p.value, dp.value


def lbm_axi_mass_field_noalloc(d_rho, nz, nr, d_out, stream=None):
    """Allocation-free FP64 mass reduction over a caller-owned device density
    field (contiguous float64 CUDA tensor of nz*nr values) into a caller-owned
    float64 CUDA tensor of 2 values: [sum (j+1/2) rho, sum rho].  Enqueued on
    `stream` (a torch.cuda.Stream, a raw cudaStream_t or None); nothing is
    allocated.  Fields larger than NOALLOC_MAX_NODES are rejected."""
    if nz * nr > NOALLOC_MAX_NODES:
        raise LbmError(ERR_INVALID_ARG, "lbm_axi_mass_field_noalloc: nz*nr = %d exceeds the maximum %d"
                       % (nz * nr, NOALLOC_MAX_NODES))
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib().lbm_axi_mass_field_noalloc(_devptr(d_rho), int(nz), int(nr), _devptr(d_out), raw),
           "lbm_axi_mass_field_noalloc")


# ------------------------------------------------------------ batched API --

def lbm_axi_batch_create(handles, stream=None):
    arr = (_H * len(handles))(*[h.value if isinstance(h, _H) else h for h in handles])
    b = _H()
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib().lbm_axi_batch_create(arr, len(handles), raw, C.byref(b)), "lbm_axi_batch_create")
    return b


def lbm_axi_batch_step(b, n):
    _check(lib().lbm_axi_batch_step(b, int(n)), "lbm_axi_batch_step")


def lbm_axi_batch_step_async(b, n):
    _check(lib().lbm_axi_batch_step_async(b, int(n)), "lbm_axi_batch_step_async")


def lbm_axi_batch_sync(b):
    """Wait; returns LBM_OK or the first error code (per-solve detail: lbm_axi_batch_status)."""
    return lib().lbm_axi_batch_sync(b)


def lbm_axi_batch_status(b, n):
    st = (C.c_int * n)()
    rc = lib().lbm_axi_batch_status(b, st)
    if rc not in (OK, ERR_UNPHYSICAL):
        raise LbmError(rc, "lbm_axi_batch_status")
    return list(st)


def lbm_axi_batch_get_tuning(b):
    t = lbm_axi_batch_tuning()
    _check(lib().lbm_axi_batch_get_tuning(b, C.byref(t)), "lbm_axi_batch_get_tuning")
    return t.strip, t.grid


def lbm_axi_batch_set_tuning(b, strip, grid):
    t = lbm_axi_batch_tuning(strip, grid)
    _check(lib().lbm_axi_batch_set_tuning(b, C.byref(t)), "lbm_axi_batch_set_tuning")


def lbm_axi_batch_autotune(b, trials=5):
    t = lbm_axi_batch_tuning()
    _check(lib().lbm_axi_batch_autotune(b, int(trials), C.byref(t)), "lbm_axi_batch_autotune")
    return t.strip, t.grid


def lbm_axi_autotune(h, trials=5):
    t = lbm_axi_tuning()
    _check(lib().lbm_axi_autotune(h, int(trials), C.byref(t)), "lbm_axi_autotune")
    return t.path, t.rows_per_cta


def lbm_axi_batch_destroy(b):
    lib().lbm_axi_batch_destroy(b)


def lbm_axi_tile_plan(sizes, strip, slots):
    """Tile plan of a batched launch for solves of the given (nz, nr) sizes:
    (tiles as an (ntiles, 4) array of solve, strip, j0, jend in CTA order,
    first offsets per CTA, makespan in rows)."""
    n = len(sizes)
    nz = (C.c_int * n)(*[int(a) for a, _ in sizes])
    nr = (C.c_int * n)(*[int(b) for _, b in sizes])
    nt, nc, ms = C.c_int(), C.c_int(), C.c_longlong()
    rc = lib().lbm_axi_tile_plan(nz, nr, n, int(strip), int(slots), 0, None, None, C.byref(nt), C.byref(nc),
                                 C.byref(ms))
    if rc != ERR_INVALID_ARG or nt.value <= 0:
        _check(rc if rc != OK else ERR_INVALID_ARG, "lbm_axi_tile_plan")
    tiles = (C.c_int * (4 * nt.value))()
    first = (C.c_int * (int(slots) + 1))()
    _check(lib().lbm_axi_tile_plan(nz, nr, n, int(strip), int(slots), nt.value, tiles, first, C.byref(nt),
                                   C.byref(nc), C.byref(ms)), "lbm_axi_tile_plan")
    return np.array(tiles, dtype=np.int64).reshape(-1, 4), np.array(first[:nc.value + 1], dtype=np.int64), ms.value


class Batch:
    """Solves advanced together (one launch per step).  Borrows the Solver objects."""

    def __init__(self, solvers, stream=None):
        self.solvers = list(solvers)
        self.b = lbm_axi_batch_create([s.h for s in self.solvers], stream)

    def step(self, n):
        rc = lib().lbm_axi_batch_step(self.b, int(n))
        if rc not in (OK, ERR_UNPHYSICAL):
            raise LbmError(rc, "lbm_axi_batch_step")
        return rc

    def step_async(self, n):
        lbm_axi_batch_step_async(self.b, n)

    def sync(self):
        return lbm_axi_batch_sync(self.b)

    def status(self):
        return lbm_axi_batch_status(self.b, len(self.solvers))

    def autotune(self, trials=5):
        return lbm_axi_batch_autotune(self.b, trials)

    def close(self):
        if self.b:
            lbm_axi_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_alloc_keep = []


def use_torch_allocator(device=None):
    """Route the library's device allocations through torch's caching allocator
    (affects solves created afterwards)."""
    import torch

    dev = torch.cuda.current_device() if device is None else device

    @ALLOC_FN
    def _alloc(nbytes, ctx):
        return torch.cuda.caching_allocator_alloc(int(nbytes), dev)

    @RELEASE_FN
    def _release(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    _alloc_keep[:] = [_alloc, _release]
    _check(lib().lbm_axi_set_allocator(_alloc, _release, None), "lbm_axi_set_allocator")


def use_cuda_allocator():
    _check(lib().lbm_axi_set_allocator(ALLOC_FN(), RELEASE_FN(), None), "lbm_axi_set_allocator")
    _alloc_keep[:] = []


# ------------------------------------------------------------ convenience --

class Solver:
    """One solve: owns an lbm_axi handle."""

    def __init__(self, nz, nr, tau, eos=None, A=-0.152, precision=64, top=TOP_FREESLIP, axis=1, multiphase=1,
                 kappa=KAPPA_THERMO, hr_sign=-1, rho_ref=0.0, g_z=0.0, stream=None, h_eval=H_LOCAL,
                 forcing=FORCING_EDM, axis_a_term=AXIS_A_PRINTED):
        o = lbm_axi_default_opts()
        o.precision, o.top_bc, o.axis_terms, o.multiphase = precision, top, axis, multiphase
        o.kappa_mode, o.hr_sign, o.rho_ref, o.g_z = kappa, hr_sign, rho_ref, g_z
        o.stream, o.h_eval, o.forcing, o.axis_a_term = stream, h_eval, forcing, axis_a_term
        self.nz, self.nr = nz, nr
        self.eos = eos
        self.h = lbm_axi_create(nz, nr, tau, eos, A, o)

    def init(self, rho, u_z=None, u_r=None, physical=False):
        """f = f^eq: u is the bare velocity, or with physical=True the fluid
        velocity u0 + F/(2 rho) (at rest for u = 0)."""
        (lbm_axi_init_physical if physical else lbm_axi_init)(self.h, self.nz, self.nr, rho, u_z, u_r)
        return self

    def step(self, n=1):
        lbm_axi_step(self.h, n)
        return self

    def moments(self):
        m = lbm_axi_moments(self.h, self.nz, self.nr)
        return {"rho": m["rho"], "uz": m["u_z"], "ur": m["u_r"], "p": m["p"]}

    def mass(self):
        return lbm_axi_mass(self.h)

    def save(self):
        return lbm_axi_save(self.h)

    def load(self, blob):
        lbm_axi_load(self.h, blob)
        return self

    def pressure_jump(self, z_c, r_c, r_in, r_out):
        return lbm_axi_pressure_jump(self.h, z_c, r_c, r_in, r_out)

    def close(self):
        if self.h:
            lbm_axi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
