// Device building blocks of the axisymmetric multiphase D2Q9 update
// (arXiv:1512.01977): lattice, per-solve parameters, equation of state and
// the boundary index maps.  Written for sm_103a; no tensor cores (the update
// is a memory-bound stencil).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// ---------------------------------------------------------------- lattice --
// D2Q9, Sec. II.A.  Direction order used throughout the library:
//   0 rest; 1 (+1, 0); 2 (-1, 0); 3 (0, +1); 4 (0, -1);
//   5 (+1, +1); 6 (-1, -1); 7 (+1, -1); 8 (-1, +1)       (c_z, c_r)
// so that 2m-1 and 2m are opposite.  Weights 4/9, 1/9 (axes), 1/36 (diagonals).
constexpr int Q = 9;

__host__ __device__ constexpr int cz_of(int i) {
    return (i == 1 || i == 5 || i == 7) ? 1 : (i == 2 || i == 6 || i == 8) ? -1 : 0;
}
__host__ __device__ constexpr int cr_of(int i) {
    return (i == 3 || i == 5 || i == 8) ? 1 : (i == 4 || i == 6 || i == 7) ? -1 : 0;
}
template <typename R>
__host__ __device__ constexpr R w_of(int i) {
    return i == 0 ? R(4) / R(9) : (i <= 4 ? R(1) / R(9) : R(1) / R(36));
}
// FP32: 4/9 and 1/9 rounded to nearest, 1/36 rounded down (one unit in the
// last place), so that the nine weights sum to exactly 1.  Rounded to nearest
// all three lie 2^-27 (relative) high and sum to 1 + 2^-27, and every collision
// then adds 2^-27 omega (rho - rho_ref) of mass per node: a systematic drift of
// about 5e-4 over 40000 steps of a flat interface at density ratio ~500.
template <>
__host__ __device__ constexpr float w_of<float>(int i) {
    return i == 0 ? 0x1.c71c72p-2f : (i <= 4 ? 0x1.c71c72p-4f : 0x1.c71c70p-6f);
}
// Direction index of the velocity (cz, cr).
__host__ __device__ constexpr int dir_of(int cz, int cr) {
    return cr == 0 ? (cz == 0 ? 0 : (cz > 0 ? 1 : 2))
                   : (cz == 0 ? (cr > 0 ? 3 : 4)
                              : (cz > 0 ? (cr > 0 ? 5 : 7) : (cr > 0 ? 8 : 6)));
}

enum { TOP_FREESLIP = 0, TOP_NOSLIP = 1, TOP_PERIODIC = 2 };
enum { EOS_VDW = 0, EOS_CS = 1 };
enum { KAPPA_THERMO = 0, KAPPA_LATTICE = 1, KAPPA_MIXED = 2 };

// Error bits a kernel may raise in the device error word.
enum : int { ERRBIT_RHO = 1, ERRBIT_PSI = 2, ERRBIT_NONFINITE = 4 };

// ------------------------------------------------------------- parameters --
template <typename R>
struct Params {
    int nz, nr;        // grid
    int pitch;         // row pitch (elements) of every plane, >= nz, multiple of 32
    R axis_a;          // c of the c A psi_r grad psi / r term of F_axis (6 printed, 2 exact expansion)
    long long plane;   // elements per plane = pitch * nr
    R tau_inv;         // 1 / tau
    R nu;              // (tau - 1/2) / 3
    R A;               // Kupershtokh mixing parameter
    R rho_ref;         // deviation reference (0 in FP64 by default)
    R gz;              // body acceleration along z
    int eos;           // EOS_*
    R T, a, b, Rg, lambda;
    int top, axis, multiphase, kappa, hr_sign;
};

// h_i at the link midpoint: the step that reads the
// populations adds the arrival half h_i(y)/2 from src (the S0 = -rho u_r/r,
// H_z, H_r planes of the step that wrote them) and writes its own to dst.
// Null pointers: h_i at the node.
template <typename R>
struct LinkPlanes {
    const R* src;
    R* dst;
};

// One solve of a batched launch: its parameters and its two population buffers
// (even batch steps read f_a and write f_b, odd steps the reverse), and with
// the link-midpoint source its two sets of source planes, swapped the same way
// (null otherwise).
template <typename R>
struct BatchSolve {
    Params<R> p;
    const R* f_a;
    R* f_b;
    const R* h_a;
    R* h_b;
};

// The descriptors of a batch of at most N solves as one kernel argument
// (about 30 KB, under the 32 KB argument limit): the kernel reads a tile's
// parameters through the constant bank instead of staging them in shared
// memory.
template <typename R>
struct BatchTable {
    static constexpr int N = (30 * 1024) / (int)sizeof(BatchSolve<R>);
    BatchSolve<R> s[N];
};

// Compiled forms of the collision in the fused kernel (bit set): Guo forcing
// in place of the EDM shift, the link-midpoint source in place of h_i at the node.
enum { FV_GUO = 1, FV_LINK = 2 };

// --------------------------------------------------------------------- EOS --
// P_k(rho) of Eq. (kupershtokvdwpressure) or Carnahan-Starling.
template <typename R>
__device__ __forceinline__ R eos_p(const Params<R>& p, R rho) {
    if (p.eos == EOS_VDW) {
        return p.lambda * (R(8) * rho * p.T / (R(3) - rho) - R(3) * rho * rho);
    }
    R e = p.b * rho * R(0.25);
    R om = R(1) - e;
    R num = R(1) + e * (R(1) + e * (R(1) - e));
    return rho * p.Rg * p.T * num / (om * om * om) - p.a * rho * rho;
}

// dP_k/drho = c_k^2.  vdW: Eq. (kupershtokhspeedofsound) squared.  CS: the
// derivative of rho (1 + e + e^2 - e^3)/(1 - e)^3 with respect to rho is
// (1 + 4e + 4e^2 - 4e^3 + e^4)/(1 - e)^4.
template <typename R>
__device__ __forceinline__ R eos_dpdrho(const Params<R>& p, R rho) {
    if (p.eos == EOS_VDW) {
        R d = R(3) - rho;
        return p.lambda * (R(24) * p.T / (d * d) - R(6) * rho);
    }
    R e = p.b * rho * R(0.25);
    R om = R(1) - e;
    R om2 = om * om;
    R num = R(1) + e * (R(4) + e * (R(4) + e * (R(-4) + e)));
    return p.Rg * p.T * num / (om2 * om2) - R(2) * p.a * rho;
}

// c^4 factor of F_axis (Sec. II.C).
template <typename R>
__device__ __forceinline__ R kappa_of(const Params<R>& p, R rho) {
    if (p.kappa == KAPPA_LATTICE) return R(1) / R(9);
    R c2 = eos_dpdrho(p, rho);
    return p.kappa == KAPPA_MIXED ? c2 * (R(1) / R(3)) : c2 * c2;
}

// ------------------------------------------------------------- index maps --
__device__ __forceinline__ int wrap_small(int k, int n) {  // k in [-n, 2n)
    return k < 0 ? k + n : (k >= n ? k - n : k);
}
__device__ __forceinline__ int wrap_any(int k, int n) {
    k %= n;
    return k < 0 ? k + n : k;
}

// Row j outside [0, nr) -> the interior row whose value it mirrors, and the
// sign a field of parities (sa at the axis, st at the top wall) picks up.
// Axis: mid-grid mirror -1-m <-> m.  Top: nr+m <-> nr-1-m, or wrap if periodic.
template <typename R>
__device__ __forceinline__ int map_row(const Params<R>& p, int j, int sa, int st, int& sign) {
    int s = 1;
    while (j < 0 || j >= p.nr) {
        if (p.top == TOP_PERIODIC) {
            j = j < 0 ? j + p.nr : j - p.nr;
        } else if (j < 0) {
            j = -1 - j;
            s *= sa;
        } else {
            j = 2 * p.nr - 1 - j;
            s *= st;
        }
    }
    sign = s;
    return j;
}

// Pull streaming: the value of population i arriving at node (k, j) is the
// post-collision value of slot (ks, js, is) of the previous step.  Interior:
// (k - cz, j - cr, i).  Axis (mid-grid specular reflection): a population with
// c_r = +1 arriving at row 0 left row 0 with c_r = -1.  Free-slip top: c_r
// flips at row nr-1.  No-slip top (mid-grid bounce-back): it left the same
// node with the opposite velocity.  Periodic z (and r if TOP_PERIODIC).
template <typename R>
__device__ __forceinline__ long long pull_slot(const Params<R>& p, int k, int j, int i) {
    const int cz = cz_of(i), cr = cr_of(i);
    int ks = k - cz, js = j - cr, is = i;
    if (js < 0) {
        if (p.top == TOP_PERIODIC) {
            js += p.nr;
        } else {
            js = 0;
            is = dir_of(cz, -cr);
        }
    } else if (js >= p.nr) {
        if (p.top == TOP_PERIODIC) {
            js -= p.nr;
        } else if (p.top == TOP_FREESLIP) {
            js = p.nr - 1;
            is = dir_of(cz, -cr);
        } else {
            ks = k;
            js = j;
            is = dir_of(-cz, -cr);
        }
    }
    ks = wrap_small(ks, p.nz);
    return (long long)is * p.plane + (long long)js * p.pitch + ks;
}

}  // namespace lbm
