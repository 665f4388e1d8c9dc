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
#include "lbm_tiles.h"

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

// CP = columns per thread (1: march, 2: march2).
template <int TZ, int RR, int CP = 1>
struct StepShape {
    static constexpr int LAG = RR + 2;
    static constexpr int WL = TZ + 12, WD = TZ + 8, WU = TZ + 4;
    // one item per thread in every stage (the widest, stage L, sets the count)
    static constexpr int NT = (RR * WL / CP + 31) / 32 * 32;
    // ring depths (rows), powers of two; schedule checked on the CPU for RR = 2 and 4
    static constexpr int DP = RR <= 2 ? 16 : 32, DD = RR <= 2 ? 8 : 16, DJ = RR <= 2 ? 16 : 32, DU = RR <= 2 ? 8 : 16;
    static constexpr int elems = DP * WL + 2 * DD * WD + 3 * DJ * WU + 2 * DU * WU;
    // schedule constraints
    static_assert(11 + 2 * RR <= DP && 4 + 2 * RR <= DD && 6 + 4 * RR <= DJ && 4 + 2 * RR <= DU, "ring depth");
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

// The three source planes (S0, H_z, H_r) of the link-midpoint source at node (k, j).
template <typename R>
__device__ __forceinline__ void link3(const Params<R>& p, const R* __restrict__ h, int j, int k, R (&a)[3]) {
    const int o = j * p.pitch + k, plane = (int)p.plane;
    a[0] = h[o];
    a[1] = h[plane + o];
    a[2] = h[2 * plane + o];
}

// One CTA marches z-strip `strip` over rows [j0, jend).  MP / AX: pseudopotential
// force and axisymmetric terms compiled in or out.  FV: collision form (FV_GUO:
// Guo forcing; FV_LINK: h_i as the link average, reading the previous step's
// source planes from hsrc and writing this step's to hdst).
template <typename R, int TZ, int RR, bool MP, bool AX, int FV = 0>
__device__ __forceinline__ void march(const Params<R>& p, const R* __restrict__ f, R* __restrict__ fout, int strip,
                                      int j0, int jend, unsigned char* smem_raw, int& bad,
                                      const R* __restrict__ hsrc = nullptr, R* __restrict__ hdst = nullptr) {
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
    R lpa[3] = {R(0), R(0), R(0)}, cpa[3] = {R(0), R(0), R(0)};  // link source planes, likewise
    constexpr bool link = (FV & FV_LINK) != 0, guo = (FV & FV_GUO) != 0;
    {
        int sg;
        const int row = j0 - 6 + l_rr;
        const bool v = l_valid(row);
        const int jm = v ? lsrc(row, sg) : 0;
        prefetch(p, f, v, jm, lkc, lpf);
        if (link && v) link3(p, hsrc, jm, lkc[1], lpa);
        const int crw = j0 - 6 - 3 * LAG + c_rr;
        prefetch(p, f, c_valid(crw), crw, ckc, cpf);
        if (link && c_valid(crw)) link3(p, hsrc, crw, ckc[1], cpa);
    }

    for (int pb = j0 - 6; pb - 3 * LAG < jend; pb += RR) {
        // ---- stage L: rows pb .. pb+RR-1: rho, j, psi from the prefetched populations.
        {
            const int row = pb + l_rr;
            if (l_valid(row)) {
                int sgn_r;
                lsrc(row, sgn_r);
                const R d1 = lpf[1] + lpf[5] + lpf[7], d2 = lpf[2] + lpf[6] + lpf[8];
                R drho = lpf[0] + lpf[3] + lpf[4] + d1 + d2;
                R jz = d1 - d2;
                R jr = (lpf[3] + lpf[5] + lpf[8]) - (lpf[4] + lpf[6] + lpf[7]);
                if (link) {
                    // arrival halves h_i(y)/2: zeroth moment S0/2, first moment H/2
                    drho += R(0.5) * lpa[0];
                    jz += R(0.5) * lpa[1];
                    jr += R(0.5) * lpa[2];
                }
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
            const int njm = nv ? lsrc(nrow, sg) : 0;
            prefetch(p, f, nv, njm, lkc, lpf);
            if (link && nv) link3(p, hsrc, njm, lkc[1], lpa);
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
                        const R a6 = p.axis_a * kA * ir * psr;
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
            const R a0 = cpa[0], az = cpa[1], ar = cpa[2];
            prefetch(p, f, c_valid(row + RR), row + RR, ckc, cpf);  // next iteration's gather
            if (link && c_valid(row + RR)) link3(p, hsrc, row + RR, ckc[1], cpa);
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
                const int o = row * p.pitch + k0 + cc;
                // link-midpoint source: this node's arrival half of the previous step's
                // h_i and the departure half of this step's; S0, H kept for the next step
                const R hs = link ? R(0.5) : R(1);
                const R hm0 = hs * m0, hHz = hs * Hz, hHr = hs * Hr;
                if (link) {
#pragma unroll
                    for (int i = 0; i < Q; i++)
                        fi[i] += R(0.5) * w_of<R>(i) * (a0 + R(3) * (R(cz_of(i)) * az + R(cr_of(i)) * ar));
                    hdst[o] = m0;
                    hdst[plane + o] = Hz;
                    hdst[2 * plane + o] = Hr;
                }
                if (guo) {
                    // Guo forcing: f*_i = f_i + omega (f^eq_i(u) - f_i) + S_i + h_i with
                    // S_i = w_i (1 - omega/2) [3 (c_i - u).F + 9 (c_i.u)(c_i.F)], F = 2 rho (u - u0)
                    const R Fz = R(2) * rho * (uz - u0z), Fr = R(2) * rho * (ur - u0r);
                    const R usq = uz * uz + ur * ur, uF = uz * Fz + ur * Fr;
                    const R gpre = R(1) - R(0.5) * omega;
                    const R base = omega * (drho - R(1.5) * rho * usq) - gpre * R(3) * uF + hm0;
                    fout[o] = om1 * fi[0] + w_of<R>(0) * base;
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const int i = 2 * m + 1;
                        const R w = w_of<R>(i);
                        const R cx = R(cz_of(i)), cy = R(cr_of(i));
                        const R cu = cx * uz + cy * ur, cF = cx * Fz + cy * Fr;
                        const R even = w * (base + R(4.5) * omega * rho * cu * cu + gpre * R(9) * cu * cF);
                        const R odd = R(3) * w * (omega * rho * cu + gpre * cF + cx * hHz + cy * hHr);
                        fout[i * plane + o] = om1 * fi[i] + even + odd;
                        fout[(i + 1) * plane + o] = om1 * fi[i + 1] + even - odd;
                    }
                } else {
                    const R u0sq = u0z * u0z + u0r * u0r, u1sq = u1z * u1z + u1r * u1r;
                    const R base = omega * drho + rho * (om1 * R(1.5) * u0sq - R(1.5) * u1sq);
                    fout[o] = om1 * fi[0] + w_of<R>(0) * (base + hm0);
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const int i = 2 * m + 1;  // i and i+1 are opposite
                        const R w = w_of<R>(i);
                        const R cx = R(cz_of(i)), cy = R(cr_of(i));
                        const R cu0 = cx * u0z + cy * u0r, cu1 = cx * u1z + cy * u1r;
                        const R even = w * (base + rho * R(4.5) * (cu1 * cu1 - om1 * cu0 * cu0) + hm0);
                        const R odd = R(3) * w * (rho * (cu1 - om1 * cu0) + cx * hHz + cy * hHr);
                        fout[i * plane + o] = om1 * fi[i] + even + odd;
                        fout[(i + 1) * plane + o] = om1 * fi[i + 1] + even - odd;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------- two columns each --
// march2 runs the same stages, lags and rings as march, but every thread owns
// two adjacent columns (c, c+1), c even, in every stage.  The index arithmetic,
// bounds checks and ring addressing of an item serve two nodes; a quantity's
// values at the two nodes travel as a pair that is loaded and stored as one
// 2-wide access (ring widths and strip origins are even, so pairs are aligned)
// and combined with the packed f32x2 instructions in FP32 (one issue for both
// lanes).  A stencil over columns c-2 .. c+3 of a row is three aligned pairs.

template <typename R>
struct PairOf;
template <>
struct PairOf<float> {
    using T = float2;
};
template <>
struct PairOf<double> {
    using T = double2;
};

__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 pk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as one packed subtract (sub.rn.f32x2), without a (-1, -1) operand pair
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
    unsigned long long x, y, d;
    memcpy(&x, &a, 8);
    memcpy(&y, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
    float2 r;
    memcpy(&r, &d, 8);
    return r;
}
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

template <typename T, typename R>
__device__ __forceinline__ T ld2(const R* a, int c) {
    return *reinterpret_cast<const T*>(a + c);
}
template <typename T, typename R>
__device__ __forceinline__ void st2(R* a, int c, T v) {
    *reinterpret_cast<T*>(a + c) = v;
}
template <typename T>
struct Tri {
    T a, b, c;  // columns (c-2, c-1), (c, c+1), (c+2, c+3)
};
template <typename T, typename R>
__device__ __forceinline__ Tri<T> ld3(const R* row, int c) {
    return {ld2<T>(row, c - 2), ld2<T>(row, c), ld2<T>(row, c + 2)};
}

// fd_both for the nodes at columns c and c+1 (15 pair loads instead of 32).
// Distance 1: n1z(k) = S(k+1) - S(k-1) with S the column sum of rows r-1..r+1,
// n1r(k) = D(k-1) + D(k) + D(k+1) with D = row r+1 - row r-1.  Distance 2:
// n2z = T(k+2) - T(k-2) with T the column sum of rows r-2, r, r+2, and
// n2r = E(k-2) + E(k) + E(k+2) with E = row r+2 - row r-2: aligned pairs.
template <typename R, typename T>
__device__ __forceinline__ void fd_both2(const R* m2m, const R* mm, const R* m0, const R* mp, const R* m2p, int c,
                                         T& dz, T& dr) {
    const Tri<T> z0 = ld3<T>(m0, c), zm = ld3<T>(mm, c), zp = ld3<T>(mp, c);
    const Tri<T> z2m = ld3<T>(m2m, c), z2p = ld3<T>(m2p, c);
    const T Sa = padd(padd(z0.a, zp.a), zm.a), Sb = padd(padd(z0.b, zp.b), zm.b);
    const T Sc = padd(padd(z0.c, zp.c), zm.c);
    const T Da = psub(zp.a, zm.a), Db = psub(zp.b, zm.b), Dc = psub(zp.c, zm.c);
    const R t = Db.x + Db.y;
    const T n1z = pk(Sb.y - Sa.y, Sc.x - Sb.x);
    const T n1r = pk(Da.y + t, Dc.x + t);
    const T n2z = psub(padd(padd(z0.c, z2p.c), z2m.c), padd(padd(z0.a, z2p.a), z2m.a));
    const T n2r = padd(padd(psub(z2p.a, z2m.a), psub(z2p.b, z2m.b)), psub(z2p.c, z2m.c));
    const T k8 = pk(R(8) / R(36), R(8) / R(36)), k1 = pk(R(-1) / R(36), R(-1) / R(36));
    dz = pfma(n1z, k8, pmul(n2z, k1));
    dr = pfma(n1r, k8, pmul(n2r, k1));
}
// fd_r_rows for columns c and c+1 (12 pair loads instead of 24).
template <typename R, typename T>
__device__ __forceinline__ T fd_r2(const R* m2m, const R* mm, const R* mp, const R* m2p, int c) {
    const Tri<T> zm = ld3<T>(mm, c), zp = ld3<T>(mp, c), z2m = ld3<T>(m2m, c), z2p = ld3<T>(m2p, c);
    const T Da = psub(zp.a, zm.a), Db = psub(zp.b, zm.b), Dc = psub(zp.c, zm.c);
    const R t = Db.x + Db.y;
    const T n1 = pk(Da.y + t, Dc.x + t);
    const T n2 = padd(padd(psub(z2p.a, z2m.a), psub(z2p.b, z2m.b)), psub(z2p.c, z2m.c));
    const T k8 = pk(R(8) / R(36), R(8) / R(36)), k1 = pk(R(-1) / R(36), R(-1) / R(36));
    return pfma(n1, k8, pmul(n2, k1));
}
// First moments of the Kupershtokh force for columns c and c+1 from psi (s1)
// or psi^2 (s2) on rows r-1 (zm), r (z0), r+1 (zq):
// sz(k) = V(k+1) - V(k-1), V = c9 row r + c36 (row r+1 + row r-1);
// sr(k) = c9 D(k) + c36 (D(k-1) + D(k+1)), D = row r+1 - row r-1.
template <typename R, typename T>
__device__ __forceinline__ void kup_moments2(const Tri<T>& zm, const Tri<T>& z0, const Tri<T>& zq, T& sz, T& sr) {
    const T c9 = pk(R(1) / R(9), R(1) / R(9)), c36 = pk(R(1) / R(36), R(1) / R(36));
    const T Va = pfma(z0.a, c9, pmul(padd(zq.a, zm.a), c36));
    const T Vb = pfma(z0.b, c9, pmul(padd(zq.b, zm.b), c36));
    const T Vc = pfma(z0.c, c9, pmul(padd(zq.c, zm.c), c36));
    sz = pk(Vb.y - Va.y, Vc.x - Vb.x);
    const T Da = psub(zq.a, zm.a), Db = psub(zq.b, zm.b), Dc = psub(zq.c, zm.c);
    sr = pfma(Db, c9, pmul(pk(Da.y + Db.y, Db.x + Dc.x), c36));
}
template <typename T>
__device__ __forceinline__ Tri<T> sq3(const Tri<T>& z) {
    return {pmul(z.a, z.a), pmul(z.b, z.b), pmul(z.c, z.c)};
}

template <typename R, typename T>
__device__ __forceinline__ T prcp(T x) {
    return pk(rcp<R>(x.x), rcp<R>(x.y));
}
// P_k and c_k^2 of a pair of densities (the formulas of eos_p_fast, eos_dp_fast).
template <typename R, typename T>
__device__ __forceinline__ T eos_p2(const Params<R>& p, T rho) {
    const T one = pk(R(1), R(1));
    if (p.eos == EOS_VDW) {
        const T l8T = pk(R(8) * p.T * p.lambda, R(8) * p.T * p.lambda), l3 = pk(R(-3) * p.lambda, R(-3) * p.lambda);
        const T d = psub(pk(R(3), R(3)), rho);
        return pfma(pmul(rho, l8T), prcp<R>(d), pmul(pmul(rho, rho), l3));
    }
    const T e = pmul(rho, pk(p.b * R(0.25), p.b * R(0.25)));
    const T om = psub(one, e);
    const T num = pfma(e, pfma(e, om, one), one);
    const T RT = pk(p.Rg * p.T, p.Rg * p.T), ma = pk(-p.a, -p.a);
    return pfma(pmul(pmul(rho, RT), num), prcp<R>(pmul(pmul(om, om), om)), pmul(pmul(rho, rho), ma));
}
template <typename R, typename T>
__device__ __forceinline__ T eos_dp2(const Params<R>& p, T rho) {
    const T one = pk(R(1), R(1));
    if (p.eos == EOS_VDW) {
        const T d = psub(pk(R(3), R(3)), rho);
        const T l24T = pk(R(24) * p.T * p.lambda, R(24) * p.T * p.lambda), l6 = pk(R(-6) * p.lambda, R(-6) * p.lambda);
        return pfma(l24T, prcp<R>(pmul(d, d)), pmul(rho, l6));
    }
    const T e = pmul(rho, pk(p.b * R(0.25), p.b * R(0.25)));
    const T om = psub(one, e);
    const T om2 = pmul(om, om);
    const T four = pk(R(4), R(4));
    const T num = pfma(e, pfma(e, pfma(e, psub(e, four), four), four), one);
    const T RT = pk(p.Rg * p.T, p.Rg * p.T), m2a = pk(R(-2) * p.a, R(-2) * p.a);
    return pfma(pmul(RT, num), prcp<R>(pmul(om2, om2)), pmul(rho, m2a));
}
template <typename R, typename T>
__device__ __forceinline__ T kappa2(const Params<R>& p, T rho) {
    if (p.kappa == KAPPA_LATTICE) return pk(R(1) / R(9), R(1) / R(9));
    const T c2 = eos_dp2<R>(p, rho);
    return p.kappa == KAPPA_MIXED ? pmul(c2, pk(R(1) / R(3), R(1) / R(3))) : pmul(c2, c2);
}

// Pulled populations of nodes (k, j) and (k+1, j) (k, k+1 wrapped in z).
// contig: columns k-1 .. k+2 need no wrap and k is even, so the second node's
// slots follow the first's and the c_z = 0 directions load as aligned pairs.
// LAST: the last read of these values in the step (stage C), loaded with the
// evict-first streaming hint so that they do not displace lines still to be read.
template <bool LAST, typename R, typename T>
__device__ __forceinline__ void gather2(const Params<R>& p, const R* __restrict__ f, int j, int k, bool contig,
                                        T (&fi)[Q]) {
    if (contig && j >= 1 && j + 1 < p.nr) {
        const int plane = (int)p.plane;
        const R* b = f + j * p.pitch + k;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const R* q = b + i * plane - cr_of(i) * p.pitch - cz_of(i);
            if (LAST) {
                if (cz_of(i) == 0)
                    fi[i] = __ldcs(reinterpret_cast<const T*>(q));
                else
                    fi[i] = pk(__ldcs(q), __ldcs(q + 1));
            } else {
                if (cz_of(i) == 0)
                    fi[i] = ld2<T>(q, 0);
                else
                    fi[i] = pk(q[0], q[1]);
            }
        }
    } else {
        const int k1 = wrap_small(k + 1, p.nz);
        const int kc0[3] = {wrap_small(k - 1, p.nz), k, k1};
        const int kc1[3] = {k, k1, wrap_small(k1 + 1, p.nz)};
        R a[Q], c[Q];
        gather32(p, f, j, kc0, a);
        gather32(p, f, j, kc1, c);
#pragma unroll
        for (int i = 0; i < Q; i++) fi[i] = pk(a[i], c[i]);
    }
}

// The link source planes at nodes (k, j) and (k+1, j) (k+1 wrapped in z).
template <typename R, typename T>
__device__ __forceinline__ void link2(const Params<R>& p, const R* __restrict__ h, int j, int k, bool contig,
                                      T (&a)[3]) {
    const int plane = (int)p.plane;
    const R* b = h + j * p.pitch;
    if (contig) {
#pragma unroll
        for (int q = 0; q < 3; q++) a[q] = ld2<T>(b + q * plane, k);
    } else {
        const int k1 = wrap_small(k + 1, p.nz);
#pragma unroll
        for (int q = 0; q < 3; q++) a[q] = pk(b[q * plane + k], b[q * plane + k1]);
    }
}

template <typename R, int TZ, int RR, bool MP, bool AX, int FV = 0>
__device__ __forceinline__ void march2(const Params<R>& p, const R* __restrict__ f, R* __restrict__ fout, int strip,
                                       int j0, int jend, unsigned char* smem_raw, int& bad,
                                       const R* __restrict__ hsrc = nullptr, R* __restrict__ hdst = nullptr) {
    using S = StepShape<TZ, RR, 2>;
    using T = typename PairOf<R>::T;
    constexpr int WL = S::WL, WD = S::WD, WU = S::WU, LAG = S::LAG;
    constexpr int DP = S::DP, DD = S::DD, DJ = S::DJ, DU = S::DU;
    constexpr int HL = WL / 2, HD = WD / 2, HU = WU / 2, HC = TZ / 2;  // pairs per row
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
    // evict-first hints on stage C's loads (the last read of those populations
    // in the step) and on the stores (read only in the next step, after the
    // whole lattice has streamed through L2): measured ~1 % faster together
    constexpr bool kStreamC = true, kStreamStore = true;
    const bool periodic = p.top == TOP_PERIODIC;
    const int nz = p.nz, nr = p.nr, pitch = p.pitch, plane = (int)p.plane;
    const R rho_ref = p.rho_ref;

    // Items: (row offset, first column of the pair); inactive items get a row
    // offset far out of range.  Lane 1 of a pair may lie past the strip's
    // last used column: it is computed (from in-range data) but never stored
    // to global memory and raises no error bits.  With 128 threads and rows of
    // at most 64 pairs (112-column strips) each row's items sit on two whole
    // warps: no warp straddles two ring rows, whose loads would replay as bank
    // conflicts (a reader stage's row is narrower than the ring's stride);
    // measured 2 % faster.  Otherwise the items of a stage are packed row after row.
    constexpr int OFF = -100000;
    constexpr bool kWarpRows = S::NT == 128 && RR == 2 && HL <= 64;
    int lr, lc, dr_, dc, ur_, uc, cr_, cc;
    bool la, da, ua, ca;
    if (kWarpRows) {
        const int wrow = tid >> 6, wcol = tid & 63;
        lr = dr_ = ur_ = cr_ = wrow;
        lc = dc = uc = cc = 2 * wcol;
        la = wcol < HL;
        da = wcol < HD;
        ua = wcol < HU;
        ca = wcol < HC;
    } else {
        lr = tid / HL, lc = 2 * (tid - (tid / HL) * HL), la = tid < RR * HL;
        dr_ = tid / HD, dc = 2 * (tid - (tid / HD) * HD), da = tid < RR * HD;
        ur_ = tid / HU, uc = 2 * (tid - (tid / HU) * HU), ua = tid < RR * HU;
        cr_ = tid / HC, cc = 2 * (tid - (tid / HC) * HC), ca = tid < RR * HC;
    }
    const int l_rr = (la && lc < kn + 12) ? lr : OFF;
    const bool l_v1 = lc + 1 < kn + 12;
    const int d_rr = (da && dc < kn + 8) ? dr_ : OFF;
    const int u_rr = (ua && uc < kn + 4) ? ur_ : OFF;
    const int c_rr = (ca && cc < kn) ? cr_ : OFF;
    const bool c_v1 = cc + 1 < kn;

    const int lk = wrap_any(k0 - 6 + lc, nz);
    const bool l_contig = lk >= 1 && lk + 2 < nz && (lk & 1) == 0;
    const int ck = min(k0 + cc, nz - 1);
    const bool c_contig = ck >= 1 && ck + 2 < nz && (ck & 1) == 0;

    const R omega = p.tau_inv, om1 = R(1) - p.tau_inv;
    const R kA = p.A, kB = R(1) - R(2) * p.A;
    const R nu = p.nu, gz = p.gz, hrs = R(p.hr_sign);
    const int uz_top = p.top == TOP_NOSLIP ? -1 : 1;

    auto lsrc = [&](int row, int& sgn_r) {
        int jm = row;
        sgn_r = 1;
        if (row < 0 || row >= nr) jm = map_row(p, row, -1, -1, sgn_r);
        return jm;
    };
    auto l_valid = [&](int row) { return row >= j0 - 6 && row < jend + 6; };
    auto c_valid = [&](int row) { return row >= j0 && row < jend; };

    T lpf[Q], cpf[Q];  // populations gathered one iteration ahead (stage L, stage C)
    T lpa[3], cpa[3];  // link source planes, likewise (FV_LINK)
    constexpr bool link = (FV & FV_LINK) != 0, guo = (FV & FV_GUO) != 0;
    if (link) {
#pragma unroll
        for (int q = 0; q < 3; q++) lpa[q] = cpa[q] = pk(R(0), R(0));
    }
    {
        int sg;
        const int row = j0 - 6 + l_rr;
        if (l_valid(row)) {
            const int jm = lsrc(row, sg);
            gather2<false>(p, f, jm, lk, l_contig, lpf);
            if (link) link2<R>(p, hsrc, jm, lk, l_contig, lpa);
        }
        const int crw = j0 - 6 - 3 * LAG + c_rr;
        if (c_valid(crw)) {
            gather2<kStreamC>(p, f, crw, ck, c_contig, cpf);
            if (link) link2<R>(p, hsrc, crw, ck, c_contig, cpa);
        }
    }

    for (int pb = j0 - 6; pb - 3 * LAG < jend; pb += RR) {
        // ---- stage L: rho, j, psi of the prefetched populations.
        {
            const int row = pb + l_rr;
            if (l_valid(row)) {
                int sgn_r;
                lsrc(row, sgn_r);
                const T d1 = padd(padd(lpf[1], lpf[5]), lpf[7]), d2 = padd(padd(lpf[2], lpf[6]), lpf[8]);
                T drho = padd(padd(padd(lpf[0], lpf[3]), padd(lpf[4], d1)), d2);
                T jz = psub(d1, d2);
                T jr = psub(padd(padd(lpf[3], lpf[5]), lpf[8]), padd(padd(lpf[4], lpf[6]), lpf[7]));
                if (link) {
                    // arrival halves h_i(y)/2: zeroth moment S0/2, first moment H/2
                    const T half = pk(R(0.5), R(0.5));
                    drho = pfma(half, lpa[0], drho);
                    jz = pfma(half, lpa[1], jz);
                    jr = pfma(half, lpa[2], jr);
                }
                const T rho = padd(drho, pk(rho_ref, rho_ref));
                if (mp) {
                    const T arg = psub(pmul(rho, pk(R(1) / R(3), R(1) / R(3))), eos_p2<R>(p, rho));
                    if (!(arg.x >= R(0)) || (l_v1 && !(arg.y >= R(0)))) bad |= ERRBIT_PSI;
                    st2(sPsi + (row & (DP - 1)) * WL, lc, pk(sqrt_nonneg(arg.x), sqrt_nonneg(arg.y)));
                }
                if (!(rho.x > R(0)) || (l_v1 && !(rho.y > R(0)))) bad |= ERRBIT_RHO;
                const int cu = lc - 4;
                if (cu >= 0 && cu < WU) {
                    const int sj = (row & (DJ - 1)) * WU;
                    st2(sRho + sj, cu, drho);
                    st2(sJz + sj, cu, jz);
                    st2(sJr + sj, cu, (periodic || sgn_r > 0) ? jr : psub(pk(R(0), R(0)), jr));
                }
            }
            // issue the next iteration's gather now; it lands behind this iteration's arithmetic
            int sg;
            const int nrow = row + RR;
            if (l_valid(nrow)) {
                const int jm = lsrc(nrow, sg);
                gather2<false>(p, f, jm, lk, l_contig, lpf);
                if (link) link2<R>(p, hsrc, jm, lk, l_contig, lpa);
            }
        }

        // ---- stage D: psi_z, psi_r (only with F_axis).
        if (mp && ax) {
            const int row = pb - LAG + d_rr;
            if (row >= j0 - 4 && row < jend + 4) {
                int er = row, s = 1;
                if (!periodic && row >= nr) er = map_row(p, row, -1, -1, s);
                T dz, dr;
                fd_both2<R>(sPsi + ((er - 2) & (DP - 1)) * WL, sPsi + ((er - 1) & (DP - 1)) * WL,
                            sPsi + (er & (DP - 1)) * WL, sPsi + ((er + 1) & (DP - 1)) * WL,
                            sPsi + ((er + 2) & (DP - 1)) * WL, dc + 2, dz, dr);
                const int o = (row & (DD - 1)) * WD;
                st2(sPz + o, dc, dz);
                st2(sPr + o, dc, s > 0 ? dr : psub(pk(R(0), R(0)), dr));
            }
        }

        // ---- stage U: total force and physical velocity.
        {
            const int row = pb - 2 * LAG + u_rr;
            if (row >= j0 - 2 && row < jend + 2) {
                int er = row, s_ur = 1, s_uz = 1;
                if (!periodic && row >= nr) {
                    er = map_row(p, row, -1, -1, s_ur);
                    s_uz = uz_top;
                }
                const int sj = (er & (DJ - 1)) * WU;
                const T drho = ld2<T>(sRho + sj, uc);
                const T rho = padd(drho, pk(rho_ref, rho_ref));
                T fz = pmul(rho, pk(gz, gz)), fr = pk(R(0), R(0));
                if (mp) {
                    const int c = uc + 4;
                    const Tri<T> z0 = ld3<T>(sPsi + (er & (DP - 1)) * WL, c);
                    const Tri<T> zm = ld3<T>(sPsi + ((er - 1) & (DP - 1)) * WL, c);
                    const Tri<T> zq = ld3<T>(sPsi + ((er + 1) & (DP - 1)) * WL, c);
                    // Kupershtokh force, Eq. (kupershtokhforcing)
                    T s1z, s1r, s2z, s2r;
                    kup_moments2<R>(zm, z0, zq, s1z, s1r);
                    kup_moments2<R>(sq3(zm), sq3(z0), sq3(zq), s2z, s2r);
                    const T psi = z0.b;
                    const T bk = pmul(pk(R(6) * kB, R(6) * kB), psi), a6k = pk(R(6) * kA, R(6) * kA);
                    fz = pfma(a6k, s2z, pfma(bk, s1z, fz));
                    fr = pfma(a6k, s2r, pfma(bk, s1r, fr));
                    if (ax) {
                        // F_axis, Eq. (multiphasecorrections); psi_rr = D_r(psi_r), psi_rz = D_r(psi_z)
                        const int cd = uc + 2;
                        const int o2m = ((er - 2) & (DD - 1)) * WD, o1m = ((er - 1) & (DD - 1)) * WD;
                        const int o1p = ((er + 1) & (DD - 1)) * WD, o2p = ((er + 2) & (DD - 1)) * WD;
                        const int o0 = (er & (DD - 1)) * WD;
                        const T prr = fd_r2<R, T>(sPr + o2m, sPr + o1m, sPr + o1p, sPr + o2p, cd);
                        const T prz = fd_r2<R, T>(sPz + o2m, sPz + o1m, sPz + o1p, sPz + o2p, cd);
                        const T psz = ld2<T>(sPz + o0, cd), psr = ld2<T>(sPr + o0, cd);
                        int rrow = er;
                        if (periodic) rrow = row < 0 ? row + nr : (row >= nr ? row - nr : row);
                        const R ir = rcp(R(rrow) + R(0.5));
                        const T irr = pk(ir, ir);
                        const T k3 = pmul(pk(R(3), R(3)), kappa2<R>(p, rho));
                        const R ca = p.axis_a * kA * ir;
                        const T a6 = pmul(pk(ca, ca), psr);
                        const T pir = pmul(psi, irr);
                        fz = pfma(k3, pfma(pir, prz, pmul(a6, psz)), fz);
                        fr = pfma(k3, pfma(pir, psub(prr, pmul(psr, irr)), pmul(a6, psr)), fr);
                    }
                }
                const T irho = prcp<R>(rho);
                const T half = pk(R(0.5), R(0.5));
                const int ou = (row & (DU - 1)) * WU;
                const T vz = pmul(pfma(half, fz, ld2<T>(sJz + sj, uc)), irho);
                const T vr = pmul(pfma(half, fr, ld2<T>(sJr + sj, uc)), irho);
                st2(sUz + ou, uc, s_uz > 0 ? vz : psub(pk(R(0), R(0)), vz));
                st2(sUr + ou, uc, s_ur > 0 ? vr : psub(pk(R(0), R(0)), vr));
            }
        }

        // ---- stage C: collide and store.
        {
            const int row = pb - 3 * LAG + c_rr;
            T fi[Q], ca[3];
#pragma unroll
            for (int i = 0; i < Q; i++) fi[i] = cpf[i];
            if (link) {
#pragma unroll
                for (int q = 0; q < 3; q++) ca[q] = cpa[q];
            }
            if (c_valid(row + RR)) {  // next iteration's gather
                gather2<kStreamC>(p, f, row + RR, ck, c_contig, cpf);
                if (link) link2<R>(p, hsrc, row + RR, ck, c_contig, cpa);
            }
            if (c_valid(row)) {
                const int c = cc + 2;
                const int sj = (row & (DJ - 1)) * WU;
                const T drho = ld2<T>(sRho + sj, c);
                const T rho = padd(drho, pk(rho_ref, rho_ref));
                const T irho = prcp<R>(rho);
                const T u0z = pmul(ld2<T>(sJz + sj, c), irho), u0r = pmul(ld2<T>(sJr + sj, c), irho);
                const int ou = (row & (DU - 1)) * WU;
                const T uz = ld2<T>(sUz + ou, c), ur = ld2<T>(sUr + ou, c);
                // EDM velocity shift F / rho from u = u0 + F / (2 rho)
                const T two = pk(R(2), R(2));
                const T u1z = pfma(two, psub(uz, u0z), u0z), u1r = pfma(two, psub(ur, u0r), u0r);
                T Hz = pk(R(0), R(0)), Hr = Hz, m0 = Hz;
                if (ax) {
                    const int o2m = ((row - 2) & (DU - 1)) * WU, o1m = ((row - 1) & (DU - 1)) * WU;
                    const int o1p = ((row + 1) & (DU - 1)) * WU, o2p = ((row + 2) & (DU - 1)) * WU;
                    const T duz_dr = fd_r2<R, T>(sUz + o2m, sUz + o1m, sUz + o1p, sUz + o2p, c);
                    T dur_dz, dur_dr;
                    fd_both2<R>(sUr + o2m, sUr + o1m, sUr + ou, sUr + o1p, sUr + o2p, c, dur_dz, dur_dr);
                    const R ir = rcp(R(row) + R(0.5));
                    const T irr = pk(ir, ir);
                    const T mu = pmul(rho, pk(nu, nu));
                    const T rur = pmul(rho, ur);
                    Hz = pmul(psub(pmul(mu, padd(duz_dr, dur_dz)), pmul(rur, uz)), irr);
                    Hr = pmul(psub(pmul(pmul(pk(R(2), R(2)), mu), pfma(pk(hrs * ir, hrs * ir), ur, dur_dr)),
                                   pmul(rur, ur)),
                              irr);
                    m0 = pmul(pk(-ir, -ir), rur);
                }
                // f*_i = (1 - omega) f_i + f^eq_i(u1) - (1 - omega) f^eq_i(u0) + h_i, opposite
                // directions sharing the even part (see march)
                const T om1p = pk(om1, om1), c15 = pk(R(1.5), R(1.5)), c45 = pk(R(4.5), R(4.5));
                R* o = fout + row * pitch + k0 + cc;
                auto store_to = [&](R* q, int i, T v) {
                    if (kStreamStore) {
                        if (c_v1)
                            __stcs(reinterpret_cast<T*>(q + i * plane), v);
                        else
                            __stcs(q + i * plane, v.x);
                    } else {
                        if (c_v1)
                            st2(q + i * plane, 0, v);
                        else
                            q[i * plane] = v.x;
                    }
                };
                auto store = [&](int i, T v) { store_to(o, i, v); };
                // c_i . v for the first direction of opposite pair i, i+1 (i odd)
                auto cdot = [&](int i, T vz, T vr) {
                    const int cx = cz_of(i), cy = cr_of(i);
                    T r = cy == 0 ? vz : (cx == 0 ? vr : (cx == cy ? padd(vz, vr) : psub(vz, vr)));
                    if (cx + cy < 0) r = psub(pk(R(0), R(0)), r);  // the first direction points to -z or -r
                    return r;
                };
                // link-midpoint source: this node's arrival half of the previous step's h_i and
                // the departure half of this step's; this step's S0, H kept for the next step
                const T half = pk(R(0.5), R(0.5));
                const T hm0 = link ? pmul(half, m0) : m0, hHz = link ? pmul(half, Hz) : Hz;
                const T hHr = link ? pmul(half, Hr) : Hr;
                if (link) {
                    fi[0] = pfma(pk(R(0.5) * w_of<R>(0), R(0.5) * w_of<R>(0)), ca[0], fi[0]);
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const int i = 2 * m + 1;
                        const R w = w_of<R>(i);
                        const T ea = pmul(pk(R(0.5) * w, R(0.5) * w), ca[0]);
                        const T oa = pmul(pk(R(1.5) * w, R(1.5) * w), cdot(i, ca[1], ca[2]));
                        fi[i] = padd(fi[i], padd(ea, oa));
                        fi[i + 1] = padd(fi[i + 1], psub(ea, oa));
                    }
                    R* hq = hdst + row * pitch + k0 + cc;
                    store_to(hq, 0, m0);
                    store_to(hq, 1, Hz);
                    store_to(hq, 2, Hr);
                }
                if (guo) {
                    // Guo forcing: f*_i = f_i + omega (f^eq_i(u) - f_i) + S_i + h_i with
                    // S_i = w_i (1 - omega/2) [3 (c_i - u).F + 9 (c_i.u)(c_i.F)], F = 2 rho (u - u0)
                    const T r2 = pmul(pk(R(2), R(2)), rho);
                    const T Fz = pmul(r2, psub(uz, u0z)), Fr = pmul(r2, psub(ur, u0r));
                    const T usq = pfma(uz, uz, pmul(ur, ur)), uF = pfma(uz, Fz, pmul(ur, Fr));
                    const R gpre = R(1) - R(0.5) * omega;
                    const T om = pk(omega, omega), gp = pk(gpre, gpre);
                    const T base = padd(pfma(om, psub(drho, pmul(c15, pmul(rho, usq))),
                                             pmul(pk(R(-3) * gpre, R(-3) * gpre), uF)),
                                        hm0);
                    store(0, pfma(om1p, fi[0], pmul(pk(w_of<R>(0), w_of<R>(0)), base)));
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const int i = 2 * m + 1;
                        const R w = w_of<R>(i);
                        const T cu = cdot(i, uz, ur), cF = cdot(i, Fz, Fr), cH = cdot(i, hHz, hHr);
                        const T even = pmul(pk(w, w), padd(base, padd(pmul(pk(R(4.5) * omega, R(4.5) * omega),
                                                                           pmul(rho, pmul(cu, cu))),
                                                                      pmul(pk(R(9) * gpre, R(9) * gpre), pmul(cu, cF)))));
                        const T odd = pmul(pk(R(3) * w, R(3) * w), padd(padd(pmul(om, pmul(rho, cu)), pmul(gp, cF)), cH));
                        store(i, padd(pfma(om1p, fi[i], even), odd));
                        store(i + 1, psub(pfma(om1p, fi[i + 1], even), odd));
                    }
                } else {
                    const T u0sq = pfma(u0z, u0z, pmul(u0r, u0r)), u1sq = pfma(u1z, u1z, pmul(u1r, u1r));
                    const T base =
                        pfma(pk(omega, omega), drho, pmul(rho, pmul(c15, psub(pmul(om1p, u0sq), u1sq))));
                    store(0, pfma(om1p, fi[0], pmul(pk(w_of<R>(0), w_of<R>(0)), padd(base, hm0))));
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const int i = 2 * m + 1;  // i and i+1 are opposite
                        const R w = w_of<R>(i);
                        const T cu0 = cdot(i, u0z, u0r), cu1 = cdot(i, u1z, u1r), cH = cdot(i, hHz, hHr);
                        const T even = pmul(pk(w, w), padd(padd(base, hm0),
                                                           pmul(rho, pmul(c45, psub(pmul(cu1, cu1),
                                                                                    pmul(om1p, pmul(cu0, cu0)))))));
                        const T odd = pmul(pk(R(3) * w, R(3) * w), pfma(rho, psub(cu1, pmul(om1p, cu0)), cH));
                        store(i, padd(pfma(om1p, fi[i], even), odd));
                        store(i + 1, psub(pfma(om1p, fi[i + 1], even), odd));
                    }
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
template <typename R, int TZ, int RR, int CP, bool MP, bool AX, int FV = 0>
__device__ __forceinline__ void march_cp(const Params<R>& p, const R* __restrict__ f, R* __restrict__ fout, int strip,
                                         int j0, int jend, unsigned char* smem_raw, int& bad,
                                         const R* __restrict__ hsrc = nullptr, R* __restrict__ hdst = nullptr) {
    if constexpr (CP == 2)
        march2<R, TZ, RR, MP, AX, FV>(p, f, fout, strip, j0, jend, smem_raw, bad, hsrc, hdst);
    else
        march<R, TZ, RR, MP, AX, FV>(p, f, fout, strip, j0, jend, smem_raw, bad, hsrc, hdst);
}

template <typename R, int TZ, int RR, int CP, int MINB, bool MP, bool AX>
__global__ void __launch_bounds__(StepShape<TZ, RR, CP>::NT, MINB) k_step(Params<R> p, const R* __restrict__ f,
                                                                          R* __restrict__ fout, int rows_per_cta,
                                                                          int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int bad = 0;
    if (rows_per_cta > 0) {
        const int j0 = blockIdx.y * rows_per_cta;
        march_cp<R, TZ, RR, CP, MP, AX>(p, f, fout, blockIdx.x, j0, min(j0 + rows_per_cta, p.nr), smem_raw, bad);
    } else {
        const int nstrips = (p.nz + TZ - 1) / TZ;
        const long long total = (long long)nstrips * p.nr;
        const long long per = (total + gridDim.x - 1) / gridDim.x;
        long long a = (long long)blockIdx.x * per;
        const long long b = min(a + per, total);
        while (a < b) {
            const int strip = (int)(a / p.nr), j0 = (int)(a - (long long)strip * p.nr);
            const int jend = (int)min((long long)p.nr, j0 + (b - a));
            march_cp<R, TZ, RR, CP, MP, AX>(p, f, fout, strip, j0, jend, smem_raw, bad);
            a += jend - j0;
        }
    }
    if (bad) atomicOr(err, bad);
}

// ------------------------------------------------------------ batched step --
// Many independent solves advanced by one launch.  The host cuts every
// solve's (z-strip, row) space into tiles and deals them to the CTAs
// (lbm_tiles.cu): CTA c marches tiles first[c] .. first[c + 1] - 1, each a row
// range of one strip of one solve.  Even batch steps read f_a and write f_b,
// odd steps the reverse (and the link source planes h_a / h_b likewise).  A
// single solve runs as a batch of one.
template <typename R, int TZ, int RR, int CP, int MINB, bool MP, bool AX, int FV = 0>
__global__ void __launch_bounds__(StepShape<TZ, RR, CP>::NT, MINB)
    k_step_batch(const BatchSolve<R>* __restrict__ solves, const Tile* __restrict__ tiles,
                 const int* __restrict__ first, int parity, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Params<R> sp;
    __shared__ int skip;  // the solve already went unphysical: its populations are void, leave them
    const int t1 = first[blockIdx.x + 1];
    for (int t = first[blockIdx.x]; t < t1; t++) {
        const Tile tl = tiles[t];
        __syncthreads();  // everyone is done with the previous tile's parameters
        if (threadIdx.x == 0) {
            sp = solves[tl.solve].p;
            skip = *static_cast<volatile const int*>(err + tl.solve);
        }
        __syncthreads();  // parameters and the skip decision are the same for the whole CTA
        const R* fin = parity ? solves[tl.solve].f_b : solves[tl.solve].f_a;
        R* fo = parity ? const_cast<R*>(solves[tl.solve].f_a) : solves[tl.solve].f_b;
        const R* hin = nullptr;
        R* ho = nullptr;
        if (FV & FV_LINK) {
            hin = parity ? solves[tl.solve].h_b : solves[tl.solve].h_a;
            ho = parity ? const_cast<R*>(solves[tl.solve].h_a) : solves[tl.solve].h_b;
        }
        if (!skip) {
            int bad = 0;
            march_cp<R, TZ, RR, CP, MP, AX, FV>(sp, fin, fo, tl.strip, tl.j0, tl.jend, smem_raw, bad, hin, ho);
            if (bad) atomicOr(&err[tl.solve], bad);
        }
    }
}

// The batched step with the solves' descriptors as one kernel argument
// (batches of at most BatchTable<R>::N solves): a tile's parameters are read
// through the constant bank by the tile's solve index instead of being staged
// in shared memory (the same arithmetic, so the same results).
template <typename R, int TZ, int RR, int CP, int MINB, bool MP, bool AX>
__global__ void __launch_bounds__(StepShape<TZ, RR, CP>::NT, MINB)
    k_step_table(const __grid_constant__ BatchTable<R> tab, const Tile* __restrict__ tiles,
                 const int* __restrict__ first, int parity, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int skip;  // the solve already went unphysical: its populations are void, leave them
    const int t1 = first[blockIdx.x + 1];
    for (int t = first[blockIdx.x]; t < t1; t++) {
        const Tile tl = tiles[t];
        __syncthreads();  // everyone is done with the previous tile
        if (threadIdx.x == 0) skip = *static_cast<volatile const int*>(err + tl.solve);
        __syncthreads();
        const BatchSolve<R>& s = tab.s[tl.solve];
        const R* fin = parity ? s.f_b : s.f_a;
        R* fo = parity ? const_cast<R*>(s.f_a) : s.f_b;
        if (!skip) {
            int bad = 0;
            march_cp<R, TZ, RR, CP, MP, AX>(s.p, fin, fo, tl.strip, tl.j0, tl.jend, smem_raw, bad);
            if (bad) atomicOr(&err[tl.solve], bad);
        }
    }
}

// The same step for a single solve, its descriptor passed by value: the
// parameters are read from the kernel's constant bank instead of a shared-memory
// copy per tile (fewer shared-memory loads on the bound pipe; the arithmetic,
// and so every result, is that of k_step_batch for a batch of one).
template <typename R, int TZ, int RR, int CP, int MINB, bool MP, bool AX, int FV = 0>
__global__ void __launch_bounds__(StepShape<TZ, RR, CP>::NT, MINB)
    k_step_single(const BatchSolve<R> s, const Tile* __restrict__ tiles, const int* __restrict__ first, int parity,
                  int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int skip;  // the solve already went unphysical: its populations are void, leave them
    const R* fin = parity ? s.f_b : s.f_a;
    R* fo = parity ? const_cast<R*>(s.f_a) : s.f_b;
    const R* hin = nullptr;
    R* ho = nullptr;
    if (FV & FV_LINK) {
        hin = parity ? s.h_b : s.h_a;
        ho = parity ? const_cast<R*>(s.h_a) : s.h_b;
    }
    const int t1 = first[blockIdx.x + 1];
    for (int t = first[blockIdx.x]; t < t1; t++) {
        const Tile tl = tiles[t];
        __syncthreads();  // everyone is done with the previous tile
        if (threadIdx.x == 0) skip = *static_cast<volatile const int*>(err);
        __syncthreads();
        if (!skip) {
            int bad = 0;
            march_cp<R, TZ, RR, CP, MP, AX, FV>(s.p, fin, fo, tl.strip, tl.j0, tl.jend, smem_raw, bad, hin, ho);
            if (bad) atomicOr(err, bad);
        }
    }
}

}  // namespace lbm
