// Kernel (b'): one whole time step in a single pass -- gather, moments, psi,
// psi derivatives, F = F_K + F_axis (+ rho g), physical velocity, velocity
// gradients, H, EDM + BGK collision with the axisymmetric source.
//
// Each CTA owns a strip of TZ columns (z) and marches over a chunk of rows
// (r), RR rows per iteration.  Every intermediate lives in a shared-memory
// ring of rows (index row & (depth - 1)).  The stages run LAG = RR + 2 rows
// apart:
//
//   stage L  rows pb          pull 9 populations, rho, j, psi     width TZ+12
//   stage D  rows pb - LAG    psi_z, psi_r                        width TZ+8
//   stage U  rows pb - 2 LAG  F_K, psi_rr, psi_rz, F_axis, F -> u  width TZ+4
//   stage C  rows pb - 3 LAG  grad u, H, h_i, EDM + BGK, store     width TZ
//
// With that lag every stage reads only rows written in earlier iterations
// and writes ring slots no stage reads in the same iteration, so one barrier
// per iteration suffices and the global loads of stage L overlap the
// arithmetic of the other stages.  Global traffic is the populations only
// (9 reads + 9 writes per node; 72 B in FP32) plus the 12-wide column halo.
//
// Rows beyond the axis are evaluated in place from mirrored data (psi, rho,
// j_z even; j_r odd), which is the mirror image of the interior value; rows
// beyond a top wall are evaluated at their interior mirror row (already
// behind the marching front) and given the field's parity; with periodic r
// wrapped rows are evaluated in place.  Needs nr >= 16 (single reflections).
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

template <typename R>
__device__ __forceinline__ R rcp(R x) {
    return R(1) / x;
}
// FP32: the hardware approximate reciprocal (rcp.approx, ~1 ulp).
template <>
__device__ __forceinline__ float rcp<float>(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// sqrt of a non-negative argument (FP32: x * rsqrt.approx(x), ~2 ulp; 0 for x <= 0).
template <typename R>
__device__ __forceinline__ R sqrt_nonneg(R x) {
    return x > R(0) ? sqrt(x) : R(0);
}
template <>
__device__ __forceinline__ float sqrt_nonneg<float>(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return x > 0.0f ? x * y : 0.0f;
}

// P_k and c_k^2 = dP_k/drho with the reciprocal above.
template <typename R>
__device__ __forceinline__ R eos_p_fast(const Params<R>& p, R rho) {
    if (p.eos == EOS_VDW) {
        return p.lambda * (R(8) * rho * p.T * rcp(R(3) - rho) - R(3) * rho * rho);
    }
    const R e = p.b * rho * R(0.25);
    const R om = R(1) - e;
    const R num = R(1) + e * (R(1) + e * (R(1) - e));
    return rho * p.Rg * p.T * num * rcp(om * om * om) - p.a * rho * rho;
}
template <typename R>
__device__ __forceinline__ R eos_dp_fast(const Params<R>& p, R rho) {
    if (p.eos == EOS_VDW) {
        const R d = R(3) - rho;
        return p.lambda * (R(24) * p.T * rcp(d * d) - R(6) * rho);
    }
    const R e = p.b * rho * R(0.25);
    const R om = R(1) - e;
    const R om2 = om * om;
    const R num = R(1) + e * (R(4) + e * (R(4) + e * (R(-4) + e)));
    return p.Rg * p.T * num * rcp(om2 * om2) - R(2) * p.a * rho;
}
template <typename R>
__device__ __forceinline__ R kappa_fast(const Params<R>& p, R rho) {
    if (p.kappa == KAPPA_LATTICE) return R(1) / R(9);
    const R c2 = eos_dp_fast(p, rho);
    return p.kappa == KAPPA_MIXED ? c2 * (R(1) / R(3)) : c2 * c2;
}

// Both isotropic derivatives (Eq. fifthorderaccuratefinitedifference) from the
// 16 distinct stencil nodes; rows r-2..r+2 given as pointers, c the column.
template <typename R>
__device__ __forceinline__ void fd_both(const R* m2m, const R* mm, const R* m0, const R* mp, const R* m2p, int c,
                                        R& dz, R& dr) {
    const R a_e = m0[c + 1], a_w = m0[c - 1], a_n = mp[c], a_s = mm[c];
    const R a_ne = mp[c + 1], a_nw = mp[c - 1], a_se = mm[c + 1], a_sw = mm[c - 1];
    const R b_e = m0[c + 2], b_w = m0[c - 2], b_n = m2p[c], b_s = m2m[c];
    const R b_ne = m2p[c + 2], b_nw = m2p[c - 2], b_se = m2m[c + 2], b_sw = m2m[c - 2];
    const R n1z = (a_e + a_ne + a_se) - (a_w + a_nw + a_sw);
    const R n2z = (b_e + b_ne + b_se) - (b_w + b_nw + b_sw);
    const R n1r = (a_n + a_ne + a_nw) - (a_s + a_se + a_sw);
    const R n2r = (b_n + b_ne + b_nw) - (b_s + b_se + b_sw);
    dz = (R(8) * n1z - n2z) * (R(1) / R(36));
    dr = (R(8) * n1r - n2r) * (R(1) / R(36));
}
template <typename R>
__device__ __forceinline__ R fd_r_rows(const R* m2m, const R* mm, const R* mp, const R* m2p, int c) {
    const R n1 = (mp[c] + mp[c + 1] + mp[c - 1]) - (mm[c] + mm[c + 1] + mm[c - 1]);
    const R n2 = (m2p[c] + m2p[c + 2] + m2p[c - 2]) - (m2m[c] + m2m[c + 2] + m2m[c - 2]);
    return (R(8) * n1 - n2) * (R(1) / R(36));
}

template <int TZ, int RR>
struct StepShape {
    static constexpr int LAG = RR + 2;
    static constexpr int WL = TZ + 12, WD = TZ + 8, WU = TZ + 4;
    // one item per thread in every stage (the widest, stage L, sets the count)
    static constexpr int NT = (RR * WL + 31) / 32 * 32;
    static constexpr int DP = 16, DD = 16, DJ = 16, DU = 8;  // ring depths (rows)
    static constexpr int elems = DP * WL + 2 * DD * WD + 3 * DJ * WU + 2 * DU * WU;
    // schedule constraints (checked exhaustively on the CPU for RR = 2)
    static_assert(11 + 2 * RR <= DP && 7 + 2 * RR <= DD && 6 + 4 * RR <= DJ && 4 + 2 * RR <= DU, "ring depth");
};

// Pulled populations of node (k, j); kc = wrapped columns k-1, k, k+1.
template <typename R>
__device__ __forceinline__ void gather32(const Params<R>& p, const R* __restrict__ f, int j, const int (&kc)[3],
                                         R (&fi)[Q]) {
    const int plane = (int)p.plane;
    if (j >= 1 && j + 1 < p.nr) {
        const int r0 = j * p.pitch;
#pragma unroll
        for (int i = 0; i < Q; i++) fi[i] = f[i * plane + r0 - cr_of(i) * p.pitch + kc[1 - cz_of(i)]];
    } else {
#pragma unroll
        for (int i = 0; i < Q; i++) fi[i] = f[pull_slot(p, kc[1], j, i)];
    }
}

// Gather issued one iteration ahead (software pipelining): valid = the node
// will be used; otherwise the registers are left untouched.
template <typename R>
__device__ __forceinline__ void prefetch(const Params<R>& p, const R* __restrict__ f, bool valid, int j,
                                         const int (&kc)[3], R (&fi)[Q]) {
    if (valid) gather32(p, f, j, kc, fi);
}

// One CTA marches z-strip `strip` over rows [j0, jend).  MP / AX: pseudopotential
// force and axisymmetric terms compiled in or out.
template <typename R, int TZ, int RR, bool MP, bool AX>
__device__ __forceinline__ void march(const Params<R>& p, const R* __restrict__ f, R* __restrict__ fout, int strip,
                                      int j0, int jend, unsigned char* smem_raw, int& bad) {
    using S = StepShape<TZ, RR>;
    constexpr int WL = S::WL, WD = S::WD, WU = S::WU, LAG = S::LAG;
    constexpr int DP = S::DP, DD = S::DD, DJ = S::DJ, DU = S::DU;
    R* sPsi = reinterpret_cast<R*>(smem_raw);  // [DP][WL]
    R* sPz = sPsi + DP * WL;                   // [DD][WD]
    R* sPr = sPz + DD * WD;
    R* sRho = sPr + DD * WD;  // [DJ][WU]  rho - rho_ref
    R* sJz = sRho + DJ * WU;
    R* sJr = sJz + DJ * WU;
    R* sUz = sJr + DJ * WU;  // [DU][WU]  physical velocity
    R* sUr = sUz + DU * WU;

    const int tid = threadIdx.x;
    const int k0 = strip * TZ;
    const int kn = min(TZ, p.nz - k0);
    constexpr bool mp = MP, ax = AX;
    const bool periodic = p.top == TOP_PERIODIC;
    const int plane = (int)p.plane;

    // Every thread owns one item (row offset, column) in each stage, the same
    // in every iteration; inactive items get a row offset far out of range.
    constexpr int OFF = -100000;
    const int lr = tid / WL, lc = tid - (tid / WL) * WL;
    const int l_rr = (tid < RR * WL && lc < kn + 12) ? lr : OFF;
    const int dr_ = tid / WD, dc = tid - (tid / WD) * WD;
    const int d_rr = (tid < RR * WD && dc < kn + 8) ? dr_ : OFF;
    const int ur_ = tid / WU, uc = tid - (tid / WU) * WU;
    const int u_rr = (tid < RR * WU && uc < kn + 4) ? ur_ : OFF;
    const int cr_ = tid / TZ, cc = tid - (tid / TZ) * TZ;
    const int c_rr = (tid < RR * TZ && cc < kn) ? cr_ : OFF;

    int lkc[3], ckc[3];
    {
        const int kg = wrap_any(k0 - 6 + lc, p.nz);
        lkc[0] = wrap_small(kg - 1, p.nz);
        lkc[1] = kg;
        lkc[2] = wrap_small(kg + 1, p.nz);
        const int k = min(k0 + cc, p.nz - 1);
        ckc[0] = wrap_small(k - 1, p.nz);
        ckc[1] = k;
        ckc[2] = wrap_small(k + 1, p.nz);
    }
    const R omega = p.tau_inv, om1 = R(1) - p.tau_inv;
    const R c9 = R(1) / R(9), c36 = R(1) / R(36);
    const R kA = p.A, kB = R(1) - R(2) * p.A;
    const int uz_top = p.top == TOP_NOSLIP ? -1 : 1;

    // Source row of a stage-L node (mirror or wrap for ghost rows).
    auto lsrc = [&](int row, int& sgn_r) {
        int jm = row;
        sgn_r = 1;
        if (row < 0 || row >= p.nr) jm = map_row(p, row, -1, -1, sgn_r);
        return jm;
    };
    auto l_valid = [&](int row) { return row >= j0 - 6 && row < jend + 6; };
    auto c_valid = [&](int row) { return row >= j0 && row < jend; };

    R lpf[Q], cpf[Q];  // populations gathered one iteration ahead (stage L, stage C)
    {
        int sg;
        const int row = j0 - 6 + l_rr;
        const bool v = l_valid(row);
        prefetch(p, f, v, v ? lsrc(row, sg) : 0, lkc, lpf);
        const int crw = j0 - 6 - 3 * LAG + c_rr;
        prefetch(p, f, c_valid(crw), crw, ckc, cpf);
    }

    for (int pb = j0 - 6; pb - 3 * LAG < jend; pb += RR) {
        // ---- stage L: rows pb .. pb+RR-1: rho, j, psi from the prefetched populations.
        {
            const int row = pb + l_rr;
            if (l_valid(row)) {
                int sgn_r;
                lsrc(row, sgn_r);
                const R d1 = lpf[1] + lpf[5] + lpf[7], d2 = lpf[2] + lpf[6] + lpf[8];
                const R drho = lpf[0] + lpf[3] + lpf[4] + d1 + d2;
                const R jz = d1 - d2;
                const R jr = (lpf[3] + lpf[5] + lpf[8]) - (lpf[4] + lpf[6] + lpf[7]);
                const R rho = p.rho_ref + drho;
                if (mp) {
                    const R arg = rho * (R(1) / R(3)) - eos_p_fast(p, rho);
                    if (!(arg >= R(0))) bad |= ERRBIT_PSI;
                    sPsi[(row & (DP - 1)) * WL + lc] = sqrt_nonneg(arg);
                }
                if (!(rho > R(0))) bad |= ERRBIT_RHO;
                const int cu = lc - 4;
                if (cu >= 0 && cu < WU) {
                    const int sj = (row & (DJ - 1)) * WU + cu;
                    sRho[sj] = drho;
                    sJz[sj] = jz;
                    sJr[sj] = periodic ? jr : R(sgn_r) * jr;
                }
            }
            // issue the next iteration's gather now; it lands behind this iteration's arithmetic
            int sg;
            const int nrow = row + RR;
            const bool nv = l_valid(nrow);  // (inactive items sit far out of range: no map_row for them)
            prefetch(p, f, nv, nv ? lsrc(nrow, sg) : 0, lkc, lpf);
        }

        // ---- stage D: rows pb-LAG ..: psi_z, psi_r (only with F_axis).
        if (mp && ax) {
            const int row = pb - LAG + d_rr;
            if (row >= j0 - 4 && row < jend + 4) {
                int er = row, s = 1;
                if (!periodic && row >= p.nr) er = map_row(p, row, -1, -1, s);
                R dz, dr;
                fd_both(sPsi + ((er - 2) & (DP - 1)) * WL, sPsi + ((er - 1) & (DP - 1)) * WL,
                        sPsi + (er & (DP - 1)) * WL, sPsi + ((er + 1) & (DP - 1)) * WL,
                        sPsi + ((er + 2) & (DP - 1)) * WL, dc + 2, dz, dr);
                const int o = (row & (DD - 1)) * WD + dc;
                sPz[o] = dz;
                sPr[o] = R(s) * dr;
            }
        }

        // ---- stage U: rows pb-2 LAG ..: total force and physical velocity.
        {
            const int row = pb - 2 * LAG + u_rr;
            if (row >= j0 - 2 && row < jend + 2) {
                const int c = uc;
                int er = row, s_ur = 1, s_uz = 1;
                if (!periodic && row >= p.nr) {
                    er = map_row(p, row, -1, -1, s_ur);
                    s_uz = uz_top;
                }
                const int sj = (er & (DJ - 1)) * WU + c;
                const R drho = sRho[sj];
                const R rho = p.rho_ref + drho;
                R fz = rho * p.gz, fr = R(0);
                if (mp) {
                    const R* m0 = sPsi + (er & (DP - 1)) * WL + c + 4;
                    const R* mm = sPsi + ((er - 1) & (DP - 1)) * WL + c + 4;
                    const R* mq = sPsi + ((er + 1) & (DP - 1)) * WL + c + 4;
                    // Kupershtokh force, Eq. (kupershtokhforcing)
                    const R e = m0[1], w = m0[-1], n = mq[0], so = mm[0];
                    const R ne = mq[1], nw = mq[-1], se = mm[1], sw = mm[-1];
                    const R s1z = c9 * (e - w) + c36 * ((ne + se) - (nw + sw));
                    const R s1r = c9 * (n - so) + c36 * ((ne + nw) - (se + sw));
                    const R s2z = c9 * (e * e - w * w) + c36 * ((ne * ne + se * se) - (nw * nw + sw * sw));
                    const R s2r = c9 * (n * n - so * so) + c36 * ((ne * ne + nw * nw) - (se * se + sw * sw));
                    const R bk = kB * m0[0];
                    fz += R(6) * (kA * s2z + bk * s1z);
                    fr += R(6) * (kA * s2r + bk * s1r);
                    if (ax) {
                        // F_axis, Eq. (multiphasecorrections); psi_rr = D_r(psi_r), psi_rz = D_r(psi_z)
                        const int cd = c + 2;
                        const int o2m = ((er - 2) & (DD - 1)) * WD, o1m = ((er - 1) & (DD - 1)) * WD;
                        const int o1p = ((er + 1) & (DD - 1)) * WD, o2p = ((er + 2) & (DD - 1)) * WD;
                        const int o0 = (er & (DD - 1)) * WD;
                        const R prr = fd_r_rows(sPr + o2m, sPr + o1m, sPr + o1p, sPr + o2p, cd);
                        const R prz = fd_r_rows(sPz + o2m, sPz + o1m, sPz + o1p, sPz + o2p, cd);
                        const R psz = sPz[o0 + cd], psr = sPr[o0 + cd];
                        int rrow = er;
                        if (periodic) rrow = row < 0 ? row + p.nr : (row >= p.nr ? row - p.nr : row);
                        const R ir = rcp(R(rrow) + R(0.5));
                        const R k3 = R(3) * kappa_fast(p, rho);
                        const R a6 = R(6) * kA * ir * psr;
                        const R psi = m0[0];
                        fz += k3 * (psi * prz * ir + a6 * psz);
                        fr += k3 * (psi * (prr - psr * ir) * ir + a6 * psr);
                    }
                }
                const R irho = rcp(rho);
                const int ou = (row & (DU - 1)) * WU + c;
                sUz[ou] = R(s_uz) * ((sJz[sj] + R(0.5) * fz) * irho);
                sUr[ou] = R(s_ur) * ((sJr[sj] + R(0.5) * fr) * irho);
            }
        }

        // ---- stage C: rows pb-3 LAG ..: collide and store.
        {
            const int row = pb - 3 * LAG + c_rr;
            R fi[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) fi[i] = cpf[i];
            prefetch(p, f, c_valid(row + RR), row + RR, ckc, cpf);  // next iteration's gather
            if (c_valid(row)) {
                const int c = cc + 2;
                const int sj = (row & (DJ - 1)) * WU + c;
                const R drho = sRho[sj];
                const R rho = p.rho_ref + drho;
                const R irho = rcp(rho);
                const R u0z = sJz[sj] * irho, u0r = sJr[sj] * irho;
                const int ou = (row & (DU - 1)) * WU + c;
                const R uz = sUz[ou], ur = sUr[ou];
                // EDM velocity shift F / rho from u = u0 + F / (2 rho)
                const R duz = R(2) * (uz - u0z), dur = R(2) * (ur - u0r);
                const R u1z = u0z + duz, u1r = u0r + dur;
                R Hz = R(0), Hr = R(0), m0 = R(0);
                if (ax) {
                    const int o2m = ((row - 2) & (DU - 1)) * WU, o1m = ((row - 1) & (DU - 1)) * WU;
                    const int o1p = ((row + 1) & (DU - 1)) * WU, o2p = ((row + 2) & (DU - 1)) * WU;
                    const R duz_dr = fd_r_rows(sUz + o2m, sUz + o1m, sUz + o1p, sUz + o2p, c);
                    R dur_dz, dur_dr;
                    fd_both(sUr + o2m, sUr + o1m, sUr + (row & (DU - 1)) * WU, sUr + o1p, sUr + o2p, c, dur_dz,
                            dur_dr);
                    const R ir = rcp(R(row) + R(0.5));
                    const R mu = rho * p.nu;
                    Hz = (mu * (duz_dr + dur_dz) - rho * ur * uz) * ir;
                    Hr = (R(2) * mu * (dur_dr + R(p.hr_sign) * ur * ir) - rho * ur * ur) * ir;
                    m0 = -rho * ur * ir;
                }
                // f*_i = f_i + omega (f^eq_i(u0) - f_i) + [f^eq_i(u1) - f^eq_i(u0)] + h_i
                //      = (1 - omega) f_i + f^eq_i(u1) - (1 - omega) f^eq_i(u0) + h_i,
                // split for opposite pairs +-c into an even and an odd part:
                //   even = w [omega drho + rho (q(u1) - (1 - omega) q(u0)) + m0],
                //          q(u) = 4.5 (c.u)^2 - 1.5 u.u
                //   odd  = 3 w [rho ((c.u1) - (1 - omega)(c.u0)) + c.H]
                const R u0sq = u0z * u0z + u0r * u0r, u1sq = u1z * u1z + u1r * u1r;
                const R base = omega * drho + rho * (om1 * R(1.5) * u0sq - R(1.5) * u1sq);
                const int o = row * p.pitch + k0 + cc;
                fout[o] = om1 * fi[0] + w_of<R>(0) * (base + m0);
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    const int i = 2 * m + 1;  // i and i+1 are opposite
                    const R w = w_of<R>(i);
                    const R cx = R(cz_of(i)), cy = R(cr_of(i));
                    const R cu0 = cx * u0z + cy * u0r, cu1 = cx * u1z + cy * u1r;
                    const R even = w * (base + rho * R(4.5) * (cu1 * cu1 - om1 * cu0 * cu0) + m0);
                    const R odd = R(3) * w * (rho * (cu1 - om1 * cu0) + cx * Hz + cy * Hr);
                    fout[i * plane + o] = om1 * fi[i] + even + odd;
                    fout[(i + 1) * plane + o] = om1 * fi[i + 1] + even - odd;
                }
            }
        }
        __syncthreads();
    }
}

// Grid: one CTA per resident slot.  The flattened strip-row space
// (strip * nr + row) is cut into gridDim.x equal contiguous ranges; a CTA
// marches each strip segment of its range (usually one or two).  rows_per_cta
// > 0 instead gives fixed chunks: CTA (x, y) = strip x, rows [y R, y R + R).
template <typename R, int TZ, int RR, int MINB, bool MP, bool AX>
__global__ void __launch_bounds__(StepShape<TZ, RR>::NT, MINB) k_step(Params<R> p, const R* __restrict__ f,
                                                                      R* __restrict__ fout, int rows_per_cta,
                                                                      int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int bad = 0;
    if (rows_per_cta > 0) {
        const int j0 = blockIdx.y * rows_per_cta;
        march<R, TZ, RR, MP, AX>(p, f, fout, blockIdx.x, j0, min(j0 + rows_per_cta, p.nr), smem_raw, bad);
    } else {
        const int nstrips = (p.nz + TZ - 1) / TZ;
        const long long total = (long long)nstrips * p.nr;
        const long long per = (total + gridDim.x - 1) / gridDim.x;
        long long a = (long long)blockIdx.x * per;
        const long long b = min(a + per, total);
        while (a < b) {
            const int strip = (int)(a / p.nr), j0 = (int)(a - (long long)strip * p.nr);
            const int jend = (int)min((long long)p.nr, j0 + (b - a));
            march<R, TZ, RR, MP, AX>(p, f, fout, strip, j0, jend, smem_raw, bad);
            a += jend - j0;
        }
    }
    if (bad) atomicOr(err, bad);
}

// ------------------------------------------------------------ batched step --
// Many independent solves advanced by one launch.  The strip-row spaces of the
// solves are concatenated (solve s occupies [start[s], start[s+1])); a
// one-wave grid cuts the concatenation into equal contiguous shares, and each
// CTA marches the (solve, strip, rows) segments of its share.  Even batch
// steps read f_a and write f_b, odd steps the reverse.
template <typename R, int TZ, int RR, int MINB, bool MP, bool AX>
__global__ void __launch_bounds__(StepShape<TZ, RR>::NT, MINB)
    k_step_batch(const BatchSolve<R>* __restrict__ solves, const long long* __restrict__ start, int nsolves,
                 int parity, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Params<R> sp;
    const long long total = start[nsolves];
    const long long per = (total + gridDim.x - 1) / gridDim.x;
    long long a = (long long)blockIdx.x * per;
    const long long b = min(a + per, total);
    while (a < b) {
        int lo = 0, hi = nsolves - 1;  // last solve with start <= a
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (start[mid] <= a) lo = mid;
            else hi = mid - 1;
        }
        const int s = lo;
        __syncthreads();  // everyone is done with the previous segment's parameters
        if (threadIdx.x == 0) sp = solves[s].p;
        __syncthreads();
        const long long off = a - start[s];
        const int strip = (int)(off / sp.nr), j0 = (int)(off - (long long)strip * sp.nr);
        const int jend = (int)min((long long)sp.nr, j0 + (b - a));
        const R* fin = parity ? solves[s].f_b : solves[s].f_a;
        R* fo = parity ? const_cast<R*>(solves[s].f_a) : solves[s].f_b;
        int bad = 0;
        march<R, TZ, RR, MP, AX>(sp, fin, fo, strip, j0, jend, smem_raw, bad);
        if (bad) atomicOr(&err[s], bad);
        a += jend - j0;
    }
}

}  // namespace lbm
