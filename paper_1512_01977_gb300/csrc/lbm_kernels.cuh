// Kernels of one time step of the axisymmetric multiphase D2Q9 update
// (arXiv:1512.01977), templated on the arithmetic type R (float or double).
//
// Storage (per solve, all planes with row pitch p.pitch, z contiguous):
//   f[2][9][nr][pitch]  populations, post-collision values of the previous
//                       step (pull streaming reads them shifted by -c_i);
//                       stored as deviations f_i - w_i rho_ref
//   aux[4][nr][pitch]   rho - rho_ref, j_z, j_r, psi of the current step
//
// One step = k_density (kernel a) + k_update (kernel b).  Reductions (kernel
// c) and the init/moments passes use the same maps.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// ------------------------------------------------- kernel (a): rho, j, psi --
// Pull-gather the nine populations of node (k, j) (Sec. II.A moments:
// rho = sum_i f_i, j = sum_i c_i f_i), evaluate psi = sqrt(rho/3 - P_k(rho))
// (Sec. II.C) and write rho - rho_ref, j_z, j_r, psi.  Raises error bits for
// rho <= 0, psi^2 < 0 and non-finite values; never traps.
template <typename R>
__global__ void __launch_bounds__(256) k_density(Params<R> p, const R* __restrict__ f, R* __restrict__ aux,
                                                 int* __restrict__ err, LinkPlanes<R> lk) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (k >= p.nz || j >= p.nr) return;
    R drho = R(0), jz = R(0), jr = R(0);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const R fi = f[pull_slot(p, k, j, i)];
        drho += fi;
        jz += R(cz_of(i)) * fi;
        jr += R(cr_of(i)) * fi;
    }
    if (lk.src) {
        // arrival halves h_i(y)/2: zeroth moment S0/2, first moment H/2
        const long long o = (long long)j * p.pitch + k;
        drho += R(0.5) * lk.src[o];
        jz += R(0.5) * lk.src[p.plane + o];
        jr += R(0.5) * lk.src[2 * p.plane + o];
    }
    const R rho = p.rho_ref + drho;
    R psi = R(0);
    int bad = 0;
    if (!(rho > R(0))) bad |= ERRBIT_RHO;
    if (!isfinite(jz) || !isfinite(jr)) bad |= ERRBIT_NONFINITE;
    if (p.multiphase) {
        const R arg = rho * (R(1) / R(3)) - eos_p(p, rho);
        if (!(arg >= R(0))) bad |= ERRBIT_PSI;
        psi = sqrt(arg > R(0) ? arg : R(0));
    }
    if (bad) atomicOr(err, bad);
    const long long o = (long long)j * p.pitch + k;
    aux[o] = drho;
    aux[p.plane + o] = jz;
    aux[2 * p.plane + o] = jr;
    aux[3 * p.plane + o] = psi;
}

// ------------------------------------------------------ stencil helpers --
// Isotropic derivative, Eq. (fifthorderaccuratefinitedifference), on a
// shared-memory tile of row width W centred at m:
// d_z = 1/36 [8 (sum of the 3 nodes at dz=+1 - those at dz=-1)
//            - (sum of the 3 nodes at +2 c_i with c_z=+1 - those with c_z=-1)].
template <typename R, int W>
__device__ __forceinline__ R fd_z(const R* m) {
    const R n1 = (m[1] + m[1 + W] + m[1 - W]) - (m[-1] + m[-1 + W] + m[-1 - W]);
    const R n2 = (m[2] + m[2 + 2 * W] + m[2 - 2 * W]) - (m[-2] + m[-2 + 2 * W] + m[-2 - 2 * W]);
    return (R(8) * n1 - n2) * (R(1) / R(36));
}
template <typename R, int W>
__device__ __forceinline__ R fd_r(const R* m) {
    const R n1 = (m[W] + m[W + 1] + m[W - 1]) - (m[-W] + m[-W + 1] + m[-W - 1]);
    const R n2 = (m[2 * W] + m[2 * W + 2] + m[2 * W - 2]) - (m[-2 * W] + m[-2 * W + 2] + m[-2 * W - 2]);
    return (R(8) * n1 - n2) * (R(1) / R(36));
}

// Kupershtokh force, Eq. (kupershtokhforcing) with dt = 1:
// F = 6 [A sum_i w_i psi^2(x+c_i) c_i + (1-2A) psi(x) sum_i w_i psi(x+c_i) c_i].
template <typename R, int W>
__device__ __forceinline__ void kupershtokh(const R* m, R A, R& fz, R& fr) {
    const R e = m[1], w = m[-1], n = m[W], s = m[-W];
    const R ne = m[W + 1], nw = m[W - 1], se = m[-W + 1], sw = m[-W - 1];
    const R c9 = R(1) / R(9), c36 = R(1) / R(36);
    const R s1z = c9 * (e - w) + c36 * ((ne + se) - (nw + sw));
    const R s1r = c9 * (n - s) + c36 * ((ne + nw) - (se + sw));
    const R s2z = c9 * (e * e - w * w) + c36 * ((ne * ne + se * se) - (nw * nw + sw * sw));
    const R s2r = c9 * (n * n - s * s) + c36 * ((ne * ne + nw * nw) - (se * se + sw * sw));
    const R b = (R(1) - R(2) * A) * m[0];
    fz += R(6) * (A * s2z + b * s1z);
    fr += R(6) * (A * s2r + b * s1r);
}

// ------------------------------------- kernel (b): the fused update step --
// One CTA owns a TZ x TR tile of nodes.  Staged in shared memory:
//   psi            tile + 6 (F on a 2-ring needs psi_rr, which needs psi_r on a 4-ring)
//   psi_z, psi_r   tile + 4
//   rho-rho_ref, j tile + 2
//   u (physical)   tile + 2 (velocity gradients of H)
//   F              tile
// Values of psi_z, psi_r and u beyond the axis or a wall are the mirror
// images of interior values with their parity (psi, psi_z, u_z even; psi_r,
// u_r odd; u_z odd at a no-slip wall), evaluated at the mirrored node.
// MOMENTS = true writes rho, physical u and P_k instead of colliding.
template <int TZ, int TR>
struct TileShape {
    static constexpr int PW = TZ + 12, PH = TR + 12;
    static constexpr int DW = TZ + 8, DH = TR + 8;
    static constexpr int UW = TZ + 4, UH = TR + 4;
    static constexpr int elems = PW * PH + 2 * DW * DH + 5 * UW * UH + 2 * TZ * TR;
};

// GUO: Guo forcing (Sec. II.A) in place of the EDM shift.
template <typename R, int TZ, int TR, bool MOMENTS, bool GUO = false>
__global__ void __launch_bounds__(256) k_update(Params<R> p, Params<double> pd, const R* __restrict__ f,
                                                R* __restrict__ fout, const R* __restrict__ aux,
                                                double* __restrict__ mout, LinkPlanes<R> lk) {
    using S = TileShape<TZ, TR>;
    constexpr int PW = S::PW, PH = S::PH, DW = S::DW, DH = S::DH, UW = S::UW, UH = S::UH;
    constexpr int NT = 256;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sPsi = reinterpret_cast<R*>(smem_raw);
    R* sPz = sPsi + PW * PH;
    R* sPr = sPz + DW * DH;
    R* sRho = sPr + DW * DH;
    R* sJz = sRho + UW * UH;
    R* sJr = sJz + UW * UH;
    R* sUz = sJr + UW * UH;
    R* sUr = sUz + UW * UH;
    R* sFz = sUr + UW * UH;
    R* sFr = sFz + TZ * TR;

    const int tid = threadIdx.x;
    const int k0 = blockIdx.x * TZ, j0 = blockIdx.y * TR;
    const int kn = min(TZ, p.nz - k0), jn = min(TR, p.nr - j0);
    const bool mp = p.multiphase != 0, ax = p.axis != 0;
    const int uz_top = p.top == TOP_NOSLIP ? -1 : 1;

    // Stage 0: load psi (ring 6) and rho - rho_ref, j (ring 2).
    if (mp) {
        for (int idx = tid; idx < PW * PH; idx += NT) {
            const int a = idx / PW, b = idx - a * PW;
            if (a >= jn + 12 || b >= kn + 12) continue;
            int s;
            const int jm = map_row(p, j0 - 6 + a, 1, 1, s);
            const int km = wrap_any(k0 - 6 + b, p.nz);
            sPsi[idx] = aux[3 * p.plane + (long long)jm * p.pitch + km];
        }
    }
    for (int idx = tid; idx < UW * UH; idx += NT) {
        const int a = idx / UW, b = idx - a * UW;
        if (a >= jn + 4 || b >= kn + 4) continue;
        int s;
        const int jm = map_row(p, j0 - 2 + a, 1, 1, s);
        const int km = wrap_any(k0 - 2 + b, p.nz);
        const long long o = (long long)jm * p.pitch + km;
        sRho[idx] = aux[o];
        sJz[idx] = aux[p.plane + o];
        sJr[idx] = aux[2 * p.plane + o];
    }
    __syncthreads();

    // Stage 1: psi_z, psi_r on the 4-ring (needed for psi_rr, psi_rz of F_axis).
    if (mp && ax) {
        for (int idx = tid; idx < DW * DH; idx += NT) {
            const int a = idx / DW, b = idx - a * DW;
            if (a >= jn + 8 || b >= kn + 8) continue;
            int s;
            const int jm = map_row(p, j0 - 4 + a, -1, -1, s);
            // mirrored rows are evaluated at their interior image; wrapped rows in place
            const int jl = p.top == TOP_PERIODIC ? j0 - 4 + a : jm;
            const R* m = sPsi + (jl - j0 + 6) * PW + (b + 2);
            sPz[idx] = fd_z<R, PW>(m);
            sPr[idx] = R(s) * fd_r<R, PW>(m);
        }
        __syncthreads();
    }

    // Stage 2: total force and physical velocity on the 2-ring.
    for (int idx = tid; idx < UW * UH; idx += NT) {
        const int a = idx / UW, b = idx - a * UW;
        if (a >= jn + 4 || b >= kn + 4) continue;
        int s_ur, s_uz;
        const int jm = map_row(p, j0 - 2 + a, -1, -1, s_ur);
        map_row(p, j0 - 2 + a, 1, uz_top, s_uz);
        const int jl = p.top == TOP_PERIODIC ? j0 - 2 + a : jm;  // see stage 1
        const int lu = (jl - j0 + 2) * UW + b;
        const R drho = sRho[lu];
        const R rho = p.rho_ref + drho;
        R fz = rho * p.gz, fr = R(0);
        if (mp) {
            const R* m = sPsi + (jl - j0 + 6) * PW + (b + 4);
            kupershtokh<R, PW>(m, p.A, fz, fr);
            if (ax) {
                // F_axis = 3 kappa [psi grad_c(psi_r / r) + (c A / r) psi_r grad_c psi],
                // Eq. (multiphasecorrections) (c = 6 as printed, 2 from the exact expansion);
                // psi_rr = D_r(psi_r), psi_rz = D_r(psi_z).
                const int ld = (jl - j0 + 4) * DW + (b + 2);
                const R psi = m[0], psz = sPz[ld], psr = sPr[ld];
                const R prr = fd_r<R, DW>(sPr + ld);
                const R prz = fd_r<R, DW>(sPz + ld);
                const R ir = R(1) / (R(jm) + R(0.5));
                const R k3 = R(3) * kappa_of(p, rho);
                const R a6 = p.axis_a * p.A * ir * psr;
                fz += k3 * (psi * prz * ir + a6 * psz);
                fr += k3 * (psi * (prr - psr * ir) * ir + a6 * psr);
            }
        }
        // u = j / rho + F / (2 rho)  (Sec. II.A, velocity with half-force shift)
        const R uz = (sJz[lu] + R(0.5) * fz) / rho;
        const R ur = (sJr[lu] + R(0.5) * fr) / rho;
        sUz[idx] = R(s_uz) * uz;
        sUr[idx] = R(s_ur) * ur;
        const int ti = a - 2, tk = b - 2;
        if (ti >= 0 && ti < jn && tk >= 0 && tk < kn) {
            sFz[ti * TZ + tk] = fz;
            sFr[ti * TZ + tk] = fr;
        }
    }
    __syncthreads();

    // Stage 3: collide the tile's own nodes.
    for (int idx = tid; idx < TZ * TR; idx += NT) {
        const int ti = idx / TZ, tk = idx - ti * TZ;
        if (ti >= jn || tk >= kn) continue;
        const int k = k0 + tk, j = j0 + ti;
        const int lu = (ti + 2) * UW + (tk + 2);
        const R drho = sRho[lu];
        const R rho = p.rho_ref + drho;
        const R uz = sUz[lu], ur = sUr[lu];
        if (MOMENTS) {
            const long long o = (long long)j * p.nz + k;
            const double rd = (double)pd.rho_ref + (double)drho;
            if (mout) {
                mout[o] = rd;
                mout[(long long)p.nz * p.nr + o] = (double)uz;
                mout[2LL * p.nz * p.nr + o] = (double)ur;
                mout[3LL * p.nz * p.nr + o] = mp ? eos_p(pd, rd) : rd / 3.0;
            }
            continue;
        }
        const R irho = R(1) / rho;
        const R u0z = sJz[lu] / rho, u0r = sJr[lu] / rho;
        const R duz = sFz[ti * TZ + tk] * irho, dur = sFr[ti * TZ + tk] * irho;
        R Hz = R(0), Hr = R(0), m0 = R(0);
        if (ax) {
            // H of Eq. (axihz) with the c_i factors taken outside H and the
            // viscous hoop term 2 mu d_r(u_r/r) (hr_sign = -1).
            const R duz_dr = fd_r<R, UW>(sUz + lu);
            const R dur_dz = fd_z<R, UW>(sUr + lu);
            const R dur_dr = fd_r<R, UW>(sUr + lu);
            const R ir = R(1) / (R(j) + R(0.5));
            const R mu = rho * p.nu;
            Hz = (mu * (duz_dr + dur_dz) - rho * ur * uz) * ir;
            Hr = (R(2) * mu * (dur_dr + R(p.hr_sign) * ur * ir) - rho * ur * ur) * ir;
            m0 = -rho * ur * ir;
        }
        const R u0sq = u0z * u0z + u0r * u0r;
        const R sz = R(2) * u0z + duz, sr = R(2) * u0r + dur;  // u0 + u1
        const R dusum = duz * sz + dur * sr;                   // u1^2 - u0^2
        // Guo forcing: f^eq at the fluid velocity u, and
        // S_i = w_i (1 - 1/(2 tau)) [3 (c_i - u).F + 9 (c_i.u)(c_i.F)]
        const R Fz = sFz[ti * TZ + tk], Fr = sFr[ti * TZ + tk];
        const R usq = uz * uz + ur * ur, uF = uz * Fz + ur * Fr;
        const R gpre = R(1) - R(0.5) * p.tau_inv;
        const long long o = (long long)j * p.pitch + k;
        // link-midpoint source: arrival half of the previous step's h at this
        // node, departure half of this step's; this step's S0, H kept for the next
        R a0 = R(0), az = R(0), ar = R(0), hs = R(1);
        if (lk.src) {
            a0 = lk.src[o];
            az = lk.src[p.plane + o];
            ar = lk.src[2 * p.plane + o];
            lk.dst[o] = m0;
            lk.dst[p.plane + o] = Hz;
            lk.dst[2 * p.plane + o] = Hr;
            hs = R(0.5);
        }
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const R w = w_of<R>(i);
            const R cx = R(cz_of(i)), cy = R(cr_of(i));
            R fi = f[pull_slot(p, k, j, i)];
            if (lk.src) fi += R(0.5) * w * (a0 + R(3) * (cx * az + cy * ar));
            R feq, force;
            if (GUO) {
                const R cu = cx * uz + cy * ur, cF = cx * Fz + cy * Fr;
                feq = w * (drho + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq));
                force = w * gpre * (R(3) * (cF - uF) + R(9) * cu * cF);
            } else {
                const R cu0 = cx * u0z + cy * u0r;
                const R cdu = cx * duz + cy * dur;
                const R csum = cx * sz + cy * sr;
                // f^eq(rho, u0) - w_i rho_ref (Sec. II.A) and the EDM shift
                // f^eq(rho, u0 + F/rho) - f^eq(rho, u0) written as a difference
                feq = w * (drho + rho * (R(3) * cu0 + R(4.5) * cu0 * cu0 - R(1.5) * u0sq));
                force = w * rho * (R(3) * cdu + R(4.5) * cdu * csum - R(1.5) * dusum);
            }
            const R h = hs * w * (m0 + R(3) * (cx * Hz + cy * Hr));  // h_i (Sec. II.B)
            fout[i * p.plane + o] = fi + (feq - fi) * p.tau_inv + force + h;
        }
    }
}

// --------------------------------------------------------------- init --
// f_i = f_i^eq(rho, u) - w_i rho_ref, written to the slot from which the
// next pull reads population i of node (k, j).
template <typename R>
__global__ void __launch_bounds__(256) k_init(Params<R> p, double rho_ref, const double* __restrict__ rho,
                                              const double* __restrict__ uz, const double* __restrict__ ur,
                                              R* __restrict__ f) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (k >= p.nz || j >= p.nr) return;
    const long long c = (long long)j * p.nz + k;
    const double d = rho[c];
    const double vz = uz ? uz[c] : 0.0, vr = ur ? ur[c] : 0.0;
    if constexpr (sizeof(R) == 4) {
        // FP32 deviations f_i - w_i rho_ref = w_i [(rho - rho_ref) + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)]:
        // rho - rho_ref in FP64, the velocity part in FP32 (FP64 arithmetic would set this kernel's time)
        const float dr = (float)(d - rho_ref), rf = (float)d, zf = (float)vz, rrf = (float)vr;
        const float usq = zf * zf + rrf * rrf;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const float cu = (float)cz_of(i) * zf + (float)cr_of(i) * rrf;
            f[pull_slot(p, k, j, i)] = w_of<float>(i) * (dr + rf * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
        }
    } else {
        const double usq = vz * vz + vr * vr;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const double cu = cz_of(i) * vz + cr_of(i) * vr;
            const double w = w_of<double>(i);
            const double feq = w * d * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
            f[pull_slot(p, k, j, i)] = (R)(feq - w * rho_ref);
        }
    }
}

// --------------------------------------------- kernel (c): reductions --
// Warp-shuffle sums in FP64; one partial per block, summed by k_reduce_final
// in a fixed order, so results are bitwise reproducible for a given grid.
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* out) {
    __shared__ double red[N][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < N; q++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
        if (lane == 0) red[q][warp] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < N; q++) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[q][w];
            out[q] = s;
        }
    }
}

// sum (j + 1/2) rho and sum rho over all nodes (blockDim.x = 256).
template <typename R>
__global__ void __launch_bounds__(256) k_mass(Params<R> p, double rho_ref, const R* __restrict__ aux,
                                              double* __restrict__ partial) {
    double v[2] = {0.0, 0.0};
    const long long n = (long long)p.nz * p.nr;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / p.nz), k = (int)(c - (long long)j * p.nz);
        const double rho = rho_ref + (double)aux[(long long)j * p.pitch + k];
        v[0] += (j + 0.5) * rho;
        v[1] += rho;
    }
    block_sum<2>(v, partial + 2 * blockIdx.x);
}

// Sums of P_k (in FP64) and node counts inside d < r_in and outside d > r_out.
template <typename R>
__global__ void __launch_bounds__(256) k_pjump(Params<R> p, Params<double> pd, const R* __restrict__ aux,
                                               double zc, double rc, double rin, double rout,
                                               double* __restrict__ partial) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const long long n = (long long)p.nz * p.nr;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / p.nz), k = (int)(c - (long long)j * p.nz);
        const double dz = k + 0.5 - zc, dr = j + 0.5 - rc;
        const double d = sqrt(dz * dz + dr * dr);
        if (d < rin || d > rout) {
            const double rho = pd.rho_ref + (double)aux[(long long)j * p.pitch + k];
            const double pk = p.multiphase ? eos_p(pd, rho) : rho / 3.0;
            if (d < rin) {
                v[0] += pk;
                v[1] += 1.0;
            } else {
                v[2] += pk;
                v[3] += 1.0;
            }
        }
    }
    block_sum<4>(v, partial + 4 * blockIdx.x);
}

// Final sum of the per-block partials by one warp (launch <<<1, 32>>>): lane l
// adds partials l, l + 32, l + 64, ... in that order, then a shuffle tree
// combines the lanes.  The order is fixed, so the result is bitwise
// reproducible for a given number of partials.
template <int N>
__global__ void k_reduce_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    double s[N];
#pragma unroll
    for (int q = 0; q < N; q++) s[q] = 0.0;
    for (int b = lane; b < nblocks; b += 32) {
#pragma unroll
        for (int q = 0; q < N; q++) s[q] += partial[N * b + q];
    }
#pragma unroll
    for (int q = 0; q < N; q++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_down_sync(0xffffffffu, s[q], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < N; q++) out[q] = s[q];
    }
}

}  // namespace lbm
