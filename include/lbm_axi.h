/*
 * lbm_axi.h — C ABI of the GB300 (sm_103a) axisymmetric multiphase lattice
 * Boltzmann engine.
 *
 * The method is the axisymmetric pseudopotential D2Q9 scheme of Reijers,
 * Gelderblom & Toschi, "Axisymmetric multiphase lattice Boltzmann method for
 * generic equations of state" (arXiv:1512.01977):
 *   - BGK evolution with a source term, Sec. II.A, Eq. (lbm);
 *   - Srivastava-type axisymmetric source h_i with H_z, H_r, Sec. II.B, Eq. (axihz);
 *   - pseudopotential psi = sqrt(rho/3 - P_k(rho)) and the Kupershtokh
 *     single-neighbour force with mixing parameter A, applied by the exact
 *     difference method (EDM), Sec. II.C, Eq. (kupershtokhforcing);
 *   - the cylindrical multiphase correction F_axis, Eq. (multiphasecorrections),
 *     with the isotropic finite differences of Eq. (fifthorderaccuratefinitedifference);
 *   - mid-grid specular reflection on the axis, periodic z, free-slip or
 *     no-slip wall at r = nr (Sec. III.A-C).
 *
 * Grid and layout.  The half-plane holds nz (along the axis) x nr (radial)
 * nodes (k, j) at z_k = k + 1/2, r_j = j + 1/2; dt = dx = 1, c_s^2 = 1/3.
 * Every host array passed through this interface is double, of length
 * nz * nr, indexed [j * nz + k] (z contiguous).  Host arrays are copied in or
 * out during the call and never retained.
 *
 * Ownership.  A handle owns all device memory of one solve (populations,
 * auxiliary fields, scratch); lbm_axi_destroy releases it.  There is no global
 * state apart from the optional allocator hook.  A handle is not thread-safe;
 * different handles may be used from different threads.
 *
 * Errors.  Every int-returning call returns LBM_OK (0) or a negative
 * LBM_ERR_* code; lbm_axi_strerror() names it.  After LBM_ERR_UNPHYSICAL or
 * LBM_ERR_CUDA the populations are undefined until lbm_axi_init is called.
 * No call aborts the process or traps on the device.
 */
#ifndef LBM_AXI_H
#define LBM_AXI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = -1, /* bad size, NULL handle/pointer, out-of-range option */
    LBM_ERR_OOM = -2,         /* device or pinned-host allocation failed */
    LBM_ERR_CUDA = -3,        /* a CUDA runtime call or launch failed */
    LBM_ERR_UNPHYSICAL = -4,  /* rho <= 0, psi^2 = rho/3 - P_k < 0, or a non-finite value */
    LBM_ERR_TIMEOUT = -5,     /* a bounded device wait gave up */
    LBM_ERR_STATE = -6        /* call out of order (e.g. step before init) */
};

/* Equation of state P_k(rho).
 *   LBM_EOS_VDW: P_k = lambda (8 rho T / (3 - rho) - 3 rho^2), reduced units,
 *                Eq. (kupershtokvdwpressure); T = T_over_Tc (T_c = 1).
 *   LBM_EOS_CS:  Carnahan-Starling p = rho R T (1 + e + e^2 - e^3)/(1 - e)^3 - a rho^2,
 *                e = b rho / 4 (not in the paper); T = T_over_Tc * T_c(a, b, R). */
typedef enum { LBM_EOS_VDW = 0, LBM_EOS_CS = 1 } lbm_eos_kind;

typedef struct {
    int kind;         /* lbm_eos_kind */
    double T_over_Tc; /* reduced temperature, (0, 1) for two-phase states */
    double a, b, R;   /* CS constants (ignored for vdW) */
    double lambda;    /* vdW pressure scale (ignored for CS) */
} lbm_eos;

enum { LBM_TOP_FREESLIP = 0, LBM_TOP_NOSLIP = 1, LBM_TOP_PERIODIC = 2 };

/* The c^4 factor of F_axis (Sec. II.C): the paper replaces the lattice c_s by
 * the thermodynamic c_k, c_k^2 = dP_k/drho at the local density. */
enum {
    LBM_KAPPA_THERMO = 0,  /* c_k^4 (the substitution as the paper states it; default) */
    LBM_KAPPA_LATTICE = 1, /* c_s^4 = 1/9 (the lattice moment of the Taylor expansion) */
    LBM_KAPPA_MIXED = 2    /* c_s^2 c_k^2 */
};

/* Where the axisymmetric source h_i, printed at the link midpoint (x + c_i/2,
 * t + 1/2) in Eq. (lbm), is evaluated:
 *   LBM_H_LOCAL     at the node, h_i(x, t) (default; every path);
 *   LBM_H_LINK_AVG  the mean of the link's two end nodes at time t: h_i(x)/2 at
 *                   the collision and h_i(y)/2 at the arrival node y, for the
 *                   direction the population arrives with.  Keeps two extra sets
 *                   of three planes (24 B per node more traffic per FP32 step).
 *                   The fused path has it with the force and the axis terms on
 *                   (balanced wave only, rows_per_cta = 0); otherwise the solve
 *                   runs the two-kernel path.  Such a solve cannot join a batch.
 *                   Its radial acoustic modes decay at about 0.7 nu k^2 instead
 *                   of nu k^2: the half-link shift has no matching half-step in
 *                   time. */
enum { LBM_H_LOCAL = 0, LBM_H_LINK_AVG = 1 };

/* How the force F enters the collision of Eq. (lbm):
 *   LBM_FORCING_EDM  the exact difference method, S_i = f^eq_i(rho, u0 + F/rho)
 *                    - f^eq_i(rho, u0), with f^eq at the bare velocity u0 (Sec. II.C,
 *                    the scheme the Kupershtokh force is defined with; default);
 *   LBM_FORCING_GUO  Guo forcing (Sec. II.A): f^eq at the fluid velocity
 *                    u = u0 + F/(2 rho) and S_i = w_i (1 - 1/(2 tau)) [(c_i - u).F / c_s^2
 *                    + (c_i.u)(c_i.F) / c_s^4] (the printed second term, (c_i - u).(c_i - F),
 *                    is read as Guo's (c_i.u)(c_i.F)).  Like LBM_H_LINK_AVG: on the
 *                    fused path with the force and the axis terms on (rows_per_cta
 *                    = 0), else on the two-kernel path; such a solve cannot join a
 *                    batch. */
enum { LBM_FORCING_EDM = 0, LBM_FORCING_GUO = 1 };

/* The A-term of F_axis, 3 kappa (c A / r) psi_r grad_c psi (Eq. multiphasecorrections):
 *   LBM_AXIS_A_PRINTED    c = 6, as printed (default); it follows from the paper's
 *                         Taylor form, Eq. (taylorexpanssion), whose A-term is 2A grad psi lap psi;
 *   LBM_AXIS_A_EXPANSION  c = 2, from the exact Taylor expansion of the discrete force
 *                         Eq. (kupershtokhforcing) on D2Q9, whose A-term is
 *                         (2A/3)(grad psi lap psi + grad |grad psi|^2). */
enum { LBM_AXIS_A_PRINTED = 0, LBM_AXIS_A_EXPANSION = 1 };

typedef struct {
    int precision;  /* 64: FP64 populations and arithmetic; 32: FP32 populations stored as
                       deviations f_i - w_i rho_ref, FP32 arithmetic, FP64 reductions */
    int top_bc;     /* LBM_TOP_*: wall at r = nr; PERIODIC makes r periodic (plain 2D box) */
    int axis_terms; /* 1: axisymmetric source h_i and F_axis; 0: plain 2D (z, r) plane */
    int multiphase; /* 1: pseudopotential force; 0: ideal single-phase fluid */
    int kappa_mode; /* LBM_KAPPA_* */
    int hr_sign;    /* sign of u_r/r inside H_r: -1 (default, the viscous hoop term
                       2 mu d_r(u_r/r)); +1 reproduces the printed formula */
    double rho_ref; /* reference density of the FP32 deviation storage (0 allowed) */
    double g_z;     /* constant body acceleration along z (0 in the paper's runs) */
    void* stream;   /* cudaStream_t to run on; NULL: the handle creates its own */
    int h_eval;     /* LBM_H_*: where h_i of Eq. (lbm) is evaluated (see above) */
    int forcing;    /* LBM_FORCING_*: how F enters the collision (see above) */
    int axis_a_term; /* LBM_AXIS_A_*: the coefficient of F_axis's A-term (see above) */
} lbm_axi_opts;

typedef struct lbm_axi lbm_axi;

/* Fill *opts with the defaults: FP64, free-slip top, axis terms and
 * multiphase on, LBM_KAPPA_THERMO, hr_sign -1, rho_ref 0, g_z 0, own stream,
 * LBM_H_LOCAL, LBM_FORCING_EDM, LBM_AXIS_A_PRINTED. */
void lbm_axi_default_opts(lbm_axi_opts* opts);

/* Create a solve on the current CUDA device.
 *   nz, nr >= 1 with nz * nr <= 2^27 nodes and 9 * pitch * nr < 2^31, pitch
 *   being nz rounded up to a multiple of 32 (the kernels address a population
 *   buffer with 32-bit offsets); tau > 1/2 (BGK relaxation time, nu = (tau - 1/2)/3);
 *   eos: required when opts->multiphase (else may be NULL); A: Kupershtokh
 *   mixing parameter (A = -0.152 recovers the vdW coexistence curve);
 *   opts: NULL for the defaults.
 * Allocates all device memory of the solve.  Returns LBM_ERR_INVALID_ARG for
 * bad arguments, LBM_ERR_OOM when memory runs out. */
int lbm_axi_create(int nz, int nr, double tau, const lbm_eos* eos, double A, const lbm_axi_opts* opts,
                   lbm_axi** out);

/* Set the populations to equilibrium, f_i = f_i^eq(rho, u) (Sec. II.A), with
 * u taken as the bare velocity sum_i c_i f_i / rho.  rho is required; u_z and
 * u_r may be NULL (zero).  Host arrays, nz*nr doubles.  Synchronous. */
int lbm_axi_init(lbm_axi* h, const double* rho, const double* u_z, const double* u_r);

/* Same as lbm_axi_init with device arrays (nz*nr doubles, [j*nz + k]). */
int lbm_axi_init_device(lbm_axi* h, const double* d_rho, const double* d_u_z, const double* d_u_r);

/* Set the populations so that the given u is the PHYSICAL (fluid) velocity
 * u = u0 + F/(2 rho) of Sec. II.A, where u0 = sum_i c_i f_i / rho is the bare
 * velocity and F = F_K + F_axis (+ rho g_z) the force of the density field
 * itself: f_i = f_i^eq(rho, u - F/(2 rho)).  With u = 0 the fluid starts at
 * rest, the start of the droplet tests of Sec. III (equilibrium densities, no
 * flow); lbm_axi_init instead leaves a spurious F/(2 rho) in every interface
 * at t = 0.  F is evaluated on f^eq(rho, u) (density rho up to rounding).
 * rho is required; u_z and u_r may be NULL (zero).  Host arrays, nz*nr
 * doubles; a temporary device copy is made.  Synchronous.  Returns
 * LBM_ERR_UNPHYSICAL (populations then hold f^eq(rho, u)) when psi^2 < 0 or
 * rho <= 0 somewhere, LBM_ERR_OOM when the temporary copy cannot be made. */
int lbm_axi_init_physical(lbm_axi* h, const double* rho, const double* u_z, const double* u_r);

/* Same as lbm_axi_init_physical with device arrays (nz*nr doubles,
 * [j*nz + k]); no allocation. */
int lbm_axi_init_physical_device(lbm_axi* h, const double* d_rho, const double* d_u_z, const double* d_u_r);

/* Advance n >= 0 time steps: gather (pull streaming with the boundary rules),
 * moments, psi, F = F_K + F_axis (+ rho g_z), EDM + BGK collision with the
 * axisymmetric source.  Waits for the stream and returns LBM_ERR_UNPHYSICAL
 * if any step met rho <= 0, psi^2 < 0 or a non-finite value. */
int lbm_axi_step(lbm_axi* h, long long n);

/* As lbm_axi_step, but only enqueues the work on the handle's stream; the
 * error status of the enqueued steps is returned by the next lbm_axi_sync. */
int lbm_axi_step_async(lbm_axi* h, long long n);

/* Wait for the handle's stream; return the sticky error status of the steps
 * enqueued since the previous sync (and clear it). */
int lbm_axi_sync(lbm_axi* h);

/* Measurement aid: advance n steps exactly like lbm_axi_step, but launch
 * kernel by kernel (no CUDA graph) with a CUDA event pair around every launch
 * on the handle's stream.  ms[1] receives the summed device time of the n
 * launches of the step's main kernel (the fused step kernel, or kernel (b) of
 * the split path); ms[0] that of the n kernel-(a) launches of the split path
 * (0 on the fused path).  Synchronous. */
int lbm_axi_time_kernels(lbm_axi* h, long long n, double* ms);

/* Kernel configuration of a solve (performance only).
 *   path: LBM_PATH_FUSED -- one kernel per step (gather, moments, psi, forces,
 *         collision in a single pass over the populations, 72 B per node in FP32);
 *         needs nr >= 16.  LBM_PATH_SPLIT -- kernel (a) (gather, rho, j, psi into
 *         field planes) then kernel (b) (forces + collision), 140 B per node.
 *   rows_per_cta: 0 -- one wave of CTAs, each marching an equal share of the
 *         (z-strip, row) space (default); > 0 -- fixed chunks of that many rows
 *         of one z-strip per CTA.
 * The default is FUSED (nr >= 16) with rows_per_cta = 0; a solve with
 * h_eval = LBM_H_LINK_AVG or forcing = LBM_FORCING_GUO defaults to FUSED only
 * when multiphase and axis_terms are both on (else SPLIT).  The paths agree to
 * rounding.  Setting waits for the handle's stream; it returns
 * LBM_ERR_INVALID_ARG for an unknown path, rows_per_cta < 0, FUSED when nr < 16,
 * and FUSED for a LBM_H_LINK_AVG or LBM_FORCING_GUO solve without both switches
 * or with rows_per_cta > 0. */
enum { LBM_PATH_FUSED = 1, LBM_PATH_SPLIT = 2 };
typedef struct {
    int path;
    int rows_per_cta;
} lbm_axi_tuning;
int lbm_axi_get_tuning(const lbm_axi* h, lbm_axi_tuning* t);
int lbm_axi_set_tuning(lbm_axi* h, const lbm_axi_tuning* t);

/* Macroscopic fields of the current state (host arrays, any may be NULL):
 * rho = sum_i f_i; physical velocity u = sum_i c_i f_i / rho + F / (2 rho)
 * (Sec. II.A); p = P_k(rho) (rho/3 for a single-phase run).  Synchronous. */
int lbm_axi_moments(lbm_axi* h, double* rho, double* u_z, double* u_r, double* p);

/* Same as lbm_axi_moments into device arrays (nz*nr doubles each, may be NULL). */
int lbm_axi_moments_device(lbm_axi* h, double* d_rho, double* d_u_z, double* d_u_r, double* d_p);

/* r-weighted mass sum_{k,j} (j + 1/2) rho(k, j) (the 2 pi of the volume
 * element omitted) and, if mass_plain != NULL, sum rho.  FP64 reduction with a
 * fixed summation order (bitwise reproducible).  Synchronous. */
int lbm_axi_mass(lbm_axi* h, double* mass_rweighted, double* mass_plain);

/* Young-Laplace pressure jump for a droplet centred at (z_c, r_c):
 * dp = <P_k>_{d < r_in} - <P_k>_{d > r_out}, d the distance of node (z_k, r_j)
 * from the centre (Sec. III.A, Eq. laplacepressure).  FP64 reduction.
 * Returns LBM_ERR_INVALID_ARG if either region holds no node. */
int lbm_axi_pressure_jump(lbm_axi* h, double z_c, double r_c, double r_in, double r_out, double* dp);

/* Allocation-free mass reduction.  No counterpart in the paper: it serves
 * callers that cannot let a library allocate device memory for them -- a
 * serving loop running out of a fixed, pre-reserved arena, or a framework
 * whose caching allocator must account for every device byte.  It computes
 * d_out[0] = sum_{k,j} (j + 1/2) rho[j*nz + k] and d_out[1] = sum rho over a
 * caller-owned device array of nz*nr doubles (e.g. the rho written by
 * lbm_axi_moments_device), with the FP64 warp-shuffle reduction of
 * lbm_axi_mass, and writes the two doubles to the caller-owned device buffer
 * d_out.  The reduction's per-block partial sums live in a 64 KB static device
 * array that every GPU loading the library holds until the process exits; the
 * call allocates nothing.  Limits and behaviour:
 *   - nz*nr must not exceed LBM_NOALLOC_MAX_NODES (8,388,608 = 4096 x 2048);
 *     larger fields, NULL pointers or nz, nr < 1 return LBM_ERR_INVALID_ARG;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call before any
 *     stream capture on that device;
 *   - work is enqueued on `stream` (a cudaStream_t, NULL = legacy default) and
 *     the call returns without waiting; the result is in d_out once the
 *     stream reaches it;
 *   - every call shares the one array, so calls whose work overlaps on the
 *     GPU (different streams, or threads without ordering) race and must be
 *     serialised by the caller. */
#define LBM_NOALLOC_MAX_NODES 8388608
int lbm_axi_mass_field_noalloc(const double* d_rho, int nz, int nr, double* d_out, void* stream);

/* Checkpoint and resume (no counterpart in the paper; an exact restart of a
 * long run).  The state is a host blob: a 64-byte header (magic "LBMAXIS1",
 * format version 1, precision, nz, nr, rho_ref, buffer parity) followed by
 * the 9 population planes, nr x nz each with z fastest, in the solve's
 * storage precision (FP32: deviations f_i - w_i rho_ref) and in the slot
 * order the next step reads.  Loading it into a solve of the same precision,
 * grid and rho_ref and stepping on gives bitwise the run that was saved.
 * The caller owns the buffer.  lbm_axi_state_bytes: the blob size.
 * lbm_axi_save: LBM_ERR_STATE before init, LBM_ERR_INVALID_ARG if bytes is
 * too small; synchronous.  lbm_axi_load: LBM_ERR_INVALID_ARG for a blob that
 * is truncated or does not match the solve (magic, version, precision, grid,
 * rho_ref, or any parameter of the dynamics); synchronous; clears the error word.  Do not load into a solve
 * while it belongs to a live batch (the batch keeps its own step parity). */
int lbm_axi_state_bytes(const lbm_axi* h, size_t* bytes);
int lbm_axi_save(lbm_axi* h, void* buf, size_t bytes);
int lbm_axi_load(lbm_axi* h, const void* buf, size_t bytes);

/* Release the solve.  NULL is a no-op.  Waits for the handle's stream. */
void lbm_axi_destroy(lbm_axi* h);

/* Absolute EOS temperature T and critical temperature T_c of a created solve. */
int lbm_axi_temperature(const lbm_axi* h, double* T, double* T_c);

/* Bytes of device memory the solve holds (populations, fields, scratch). */
int lbm_axi_device_bytes(const lbm_axi* h, size_t* bytes);

/* Device memory a solve of this size and precision would hold. */
size_t lbm_axi_footprint(int nz, int nr, int precision);

/* Host-side EOS helpers (no GPU): critical temperature T_c of the EOS and the
 * coexistence densities at eos->T_over_Tc from the Maxwell equal-area
 * construction, integral_{v_l}^{v_v} (P_k(v) - p_s) dv = 0 with v = 1/rho. */
int lbm_eos_critical_temperature(const lbm_eos* eos, double* T_c);
int lbm_eos_coexistence(const lbm_eos* eos, double* rho_v, double* rho_l);
/* P_k(rho) and dP_k/drho at the temperature of eos. */
int lbm_eos_pressure(const lbm_eos* eos, double rho, double* p, double* dpdrho);

/* Route the library's device allocations through a caller's allocator (for
 * example a framework's caching allocator).  Process-wide; affects handles
 * created afterwards.  Pass NULL, NULL to restore cudaMalloc/cudaFree.  alloc
 * returns a device pointer aligned to at least 256 bytes or NULL. */
int lbm_axi_set_allocator(void* (*alloc)(size_t bytes, void* ctx), void (*release)(void* ptr, void* ctx),
                          void* ctx);

/* Text for an LBM_* code (static storage). */
const char* lbm_axi_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* LBM_AXI_H */
