/*
 * FP64 CPU oracle for the axisymmetric pseudopotential D2Q9 update of
 * Reijers, Gelderblom & Toschi, "Axisymmetric multiphase lattice Boltzmann
 * method for generic equations of state" (arXiv:1512.01977).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library: the lattice tables and every formula below are written out here
 * on their own.
 *
 * It is deliberately plain: whole-field passes over arrays that carry ghost
 * layers, one pass per quantity, in the order in which the paper introduces
 * the quantities.  No blocking, no fusion.  The passes carry OpenMP pragmas
 * over rows (every row of a pass is independent) for the timing build that
 * runs on all host cores; the parity build compiles without OpenMP, and the
 * two give bitwise the same results.  Populations are stored
 * pre-collision, f[i][j][k] with k (z) contiguous, and streamed by pushing.
 *
 * Grid: nz x nr nodes (k, j); r_j = j + 1/2 (the axis lies midway between
 * row 0 and its mirror ghost, Sec. III.A); dt = dx = 1; c_s^2 = 1/3.
 *
 * Parity status: every function here is pinned by a test in tests/ against a
 * closed form, an exact identity or a law printed in the paper.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q 9
#define ORC_G 6 /* ghost width: psi is needed 6 nodes out (force ring 2 + psi_rr radius 4) */

/* D2Q9 velocities c_i = (c_iz, c_ir) and weights w_i, Sec. II.A. */
static const int orc_cz[ORC_Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int orc_cr[ORC_Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double orc_w[ORC_Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                                    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

enum { ORC_TOP_FREESLIP = 0, ORC_TOP_NOSLIP = 1, ORC_TOP_PERIODIC = 2 };
enum { ORC_EOS_VDW = 0, ORC_EOS_CS = 1 };
enum { ORC_KAPPA_THERMO = 0, ORC_KAPPA_LATTICE = 1, ORC_KAPPA_MIXED = 2 };
enum { ORC_H_LOCAL = 0, ORC_H_LINK_AVG = 1 };
enum { ORC_FORCING_EDM = 0, ORC_FORCING_GUO = 1 };
enum { ORC_OK = 0, ORC_ERR_UNPHYSICAL = -4 };

typedef struct {
    int nz, nr;
    double tau;     /* BGK relaxation time, Eq. (lbm) */
    double A;       /* Kupershtokh mixing parameter, Eq. (kupershtokhforcing) */
    int eos;        /* ORC_EOS_VDW (Eq. kupershtokvdwpressure) or ORC_EOS_CS */
    double T;       /* EOS temperature: reduced T for vdW, absolute T for CS */
    double a, b, R; /* Carnahan-Starling constants */
    double lambda;  /* vdW scaling parameter lambda */
    int top;        /* boundary at r = nr: ORC_TOP_* */
    int axis;       /* 1: axisymmetric source h_i and F_axis on; 0: plain 2D (z, r) */
    int multiphase; /* 1: pseudopotential force on */
    int kappa;      /* which c^4 multiplies F_axis: ORC_KAPPA_THERMO (c_k^4) or _LATTICE (c_s^4) */
    int hr_sign;    /* sign in front of u_r/r inside H_r */
    double gz;      /* constant body acceleration along z (0 for the paper's runs) */
    double r0;      /* row j sits at r = r0 + j + 1/2; 0 for a lattice that starts at the
                       axis.  r0 > 0 describes a window cut out of a larger lattice (tests). */
    int h_eval;     /* where h_i of Eq. (lbm) is evaluated: ORC_H_LOCAL or ORC_H_LINK_AVG */
    int forcing;    /* how F enters the collision: ORC_FORCING_EDM (Sec. II.C) or ORC_FORCING_GUO (Sec. II.A) */
    double axis_a;  /* c of the c A psi_r grad psi / r term of F_axis: 6 as printed in Eq.
                       (multiphasecorrections), 2 from the exact expansion of Eq. (kupershtokhforcing) */
} orc_params;

/* ------------------------------------------------------------------ EOS -- */

/* Non-ideal pressure P_k(rho).  vdW: Eq. (kupershtokvdwpressure).
 * CS: p = rho R T (1 + e + e^2 - e^3)/(1 - e)^3 - a rho^2 with e = b rho / 4. */
double orc_eos_p(const orc_params* P, double rho) {
    if (P->eos == ORC_EOS_VDW) {
        return P->lambda * (8.0 * rho * P->T / (3.0 - rho) - 3.0 * rho * rho);
    }
    double e = P->b * rho / 4.0;
    double num = 1.0 + e + e * e - e * e * e;
    double den = (1.0 - e) * (1.0 - e) * (1.0 - e);
    return rho * P->R * P->T * num / den - P->a * rho * rho;
}

/* dP_k/drho, i.e. c_k^2.  vdW: Eq. (kupershtokhspeedofsound) squared.
 * CS: derivative of the expression above, written out by the product rule. */
double orc_eos_dpdrho(const orc_params* P, double rho) {
    if (P->eos == ORC_EOS_VDW) {
        return P->lambda * (24.0 * P->T / ((rho - 3.0) * (rho - 3.0)) - 6.0 * rho);
    }
    double e = P->b * rho / 4.0;
    double num = 1.0 + e + e * e - e * e * e;
    double den = (1.0 - e) * (1.0 - e) * (1.0 - e);
    double dnum_de = 1.0 + 2.0 * e - 3.0 * e * e;
    double dden_de = -3.0 * (1.0 - e) * (1.0 - e);
    double z = num / den;
    double dz_de = (dnum_de * den - num * dden_de) / (den * den);
    /* d/drho [rho R T z(e)] = R T (z + rho z'(e) b/4) */
    return P->R * P->T * (z + rho * dz_de * P->b / 4.0) - 2.0 * P->a * rho;
}

/* ----------------------------------------------------------- equilibrium -- */

/* f_i^eq = w_i rho [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u], Sec. II.A with c_s^2 = 1/3. */
void orc_feq(double rho, double uz, double ur, double* feq) {
    double uu = uz * uz + ur * ur;
    for (int i = 0; i < ORC_Q; i++) {
        double cu = orc_cz[i] * uz + orc_cr[i] * ur;
        feq[i] = orc_w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* ------------------------------------------------------ ghosted fields -- */

static int orc_ext_nz(const orc_params* P) { return P->nz + 2 * ORC_G; }
static int orc_ext_len(const orc_params* P) { return (P->nz + 2 * ORC_G) * (P->nr + 2 * ORC_G); }
static long orc_ext(const orc_params* P, int k, int j) {
    return (long)(j + ORC_G) * orc_ext_nz(P) + (k + ORC_G);
}

/* Map a row index outside [0, nr) onto the interior row it mirrors, and the
 * sign the field picks up on the way.  Axis: mid-grid mirror -1-m <-> m
 * (Sec. III.A, specular reflection about r = 0).  Top: mirror nr+m <->
 * nr-1-m for free-slip and no-slip walls, wrap for periodic r.  The signs for
 * the two mirrors are given per field by the caller. */
static int orc_map_row(const orc_params* P, int j, int sign_axis, int sign_top, int* sign) {
    int s = 1;
    for (;;) {
        if (j < 0) {
            if (P->top == ORC_TOP_PERIODIC) {
                j += P->nr;
            } else {
                j = -1 - j;
                s *= sign_axis;
            }
        } else if (j >= P->nr) {
            if (P->top == ORC_TOP_PERIODIC) {
                j -= P->nr;
            } else {
                j = 2 * P->nr - 1 - j;
                s *= sign_top;
            }
        } else {
            break;
        }
    }
    *sign = s;
    return j;
}

/* Fill all ghost nodes of an extended field from its interior: periodic in
 * z, mirrored (with the given parities) or periodic in r. */
void orc_fill_ghosts(const orc_params* P, double* a, int sign_axis, int sign_top) {
    int nz = P->nz;
    #pragma omp parallel for
    for (int j = -ORC_G; j < P->nr + ORC_G; j++) {
        int s = 1;
        int js = orc_map_row(P, j, sign_axis, sign_top, &s);
        for (int k = -ORC_G; k < nz + ORC_G; k++) {
            int ks = ((k % nz) + nz) % nz;
            if (js == j && ks == k) continue;
            a[orc_ext(P, k, j)] = s * a[orc_ext(P, ks, js)];
        }
    }
}

/* --------------------------------------------- finite differences (FD) -- */

/* Isotropic derivative stencil, Eq. (fifthorderaccuratefinitedifference):
 * d_alpha phi(x) = 1/36 sum_{i=1..8} (8 phi(x + c_i) - phi(x + 2 c_i)) c_{i,alpha}.
 * Evaluated at every interior node of an extended field. */
void orc_grad(const orc_params* P, const double* a, double* dz, double* dr) {
    #pragma omp parallel for
    for (int j = 0; j < P->nr; j++) {
        for (int k = 0; k < P->nz; k++) {
            double sz = 0.0, sr = 0.0;
            for (int i = 1; i < ORC_Q; i++) {
                double near = a[orc_ext(P, k + orc_cz[i], j + orc_cr[i])];
                double far = a[orc_ext(P, k + 2 * orc_cz[i], j + 2 * orc_cr[i])];
                double t = 8.0 * near - far;
                sz += t * orc_cz[i];
                sr += t * orc_cr[i];
            }
            dz[orc_ext(P, k, j)] = sz / 36.0;
            dr[orc_ext(P, k, j)] = sr / 36.0;
        }
    }
}

/* --------------------------------------------------------- force terms -- */

/* Kupershtokh single-neighbour force, Eq. (kupershtokhforcing) with dt = 1:
 * F = 18/3 [A sum_i w_i psi^2(x+c_i) c_i + (1-2A) psi(x) sum_i w_i psi(x+c_i) c_i]. */
void orc_force_kupershtokh(const orc_params* P, const double* psi, double* fz, double* fr) {
    #pragma omp parallel for
    for (int j = 0; j < P->nr; j++) {
        for (int k = 0; k < P->nz; k++) {
            double s2z = 0.0, s2r = 0.0, s1z = 0.0, s1r = 0.0;
            for (int i = 1; i < ORC_Q; i++) {
                double pn = psi[orc_ext(P, k + orc_cz[i], j + orc_cr[i])];
                s2z += orc_w[i] * pn * pn * orc_cz[i];
                s2r += orc_w[i] * pn * pn * orc_cr[i];
                s1z += orc_w[i] * pn * orc_cz[i];
                s1r += orc_w[i] * pn * orc_cr[i];
            }
            double p0 = psi[orc_ext(P, k, j)];
            fz[orc_ext(P, k, j)] = 18.0 / 3.0 * (P->A * s2z + (1.0 - 2.0 * P->A) * p0 * s1z);
            fr[orc_ext(P, k, j)] = 18.0 / 3.0 * (P->A * s2r + (1.0 - 2.0 * P->A) * p0 * s1r);
        }
    }
}

/* The c^4 factor of F_axis (Sec. II.C).  ORC_KAPPA_LATTICE: c_s^4 = 1/9, the
 * lattice moment the Taylor expansion produces.  ORC_KAPPA_THERMO: c_k^4 =
 * (dP_k/drho)^2 at the local density, every c_s of F_axis replaced by the
 * thermodynamic speed of sound.  ORC_KAPPA_MIXED: c_s^2 c_k^2, only the c_s^2
 * of the bracketed correction replaced. */
double orc_kappa(const orc_params* P, double rho) {
    if (P->kappa == ORC_KAPPA_LATTICE) return 1.0 / 9.0;
    double ck2 = orc_eos_dpdrho(P, rho);
    if (P->kappa == ORC_KAPPA_MIXED) return ck2 / 3.0;
    return ck2 * ck2;
}

/* Cylindrical contribution to the multiphase force, Eq. (multiphasecorrections):
 * F_axis = 3 kappa [psi grad_c(psi_r / r) + (c A / r) psi_r grad_c psi], with
 * grad_c(psi_r/r) = (psi_rz / r, psi_rr / r - psi_r / r^2).  The paper prints
 * c = 6, from its Taylor form Eq. (taylorexpanssion); the exact expansion of the
 * discrete force Eq. (kupershtokhforcing) gives c = 2 (P->axis_a selects). */
void orc_force_axis(double kappa, double A, double c, double r, double psi, double psi_z, double psi_r,
                    double psi_rr, double psi_rz, double* fz, double* fr) {
    *fz = 3.0 * kappa * (psi * psi_rz / r + c * A / r * psi_r * psi_z);
    *fr = 3.0 * kappa * (psi * (psi_rr / r - psi_r / (r * r)) + c * A / r * psi_r * psi_r);
}

/* --------------------------------------------------- axisymmetric source -- */

/* H_z, H_r of Eq. (axihz), read with the c_i factors outside H (inside, the
 * first moment of h_i would vanish):
 * H_z = (1/r) (mu (d_r u_z + d_z u_r) - rho u_r u_z)
 * H_r = (1/r) (2 mu (d_r u_r + s u_r / r) - rho u_r^2), s = hr_sign. */
void orc_source_H(double r, double rho, double mu, double uz, double ur, double duz_dr,
                  double dur_dz, double dur_dr, int hr_sign, double* Hz, double* Hr) {
    *Hz = (mu * (duz_dr + dur_dz) - rho * ur * uz) / r;
    *Hr = (2.0 * mu * (dur_dr + hr_sign * ur / r) - rho * ur * ur) / r;
}

/* h_i = w_i (-rho u_r / r + (c_iz H_z + c_ir H_r) / c_s^2), Sec. II.B. */
void orc_source_h(double r, double rho, double ur, double Hz, double Hr, double* h) {
    for (int i = 0; i < ORC_Q; i++) {
        h[i] = orc_w[i] * (-rho * ur / r + 3.0 * (orc_cz[i] * Hz + orc_cr[i] * Hr));
    }
}

/* ----------------------------------------------------------- streaming -- */

/* Destination of population i leaving interior node (k, j): periodic in z;
 * specular reflection at the axis (mid-grid, the r-component of c_i flips);
 * at the top either specular reflection (free-slip), mid-grid bounce-back
 * (no-slip: both components flip, node unchanged) or wrap (periodic). */
void orc_stream_dest(const orc_params* P, int k, int j, int i, int* kd, int* jd, int* id) {
    int cz = orc_cz[i], cr = orc_cr[i];
    int kk = k + cz, jj = j + cr;
    int ncz = cz, ncr = cr;
    if (jj < 0) {
        if (P->top == ORC_TOP_PERIODIC) {
            jj += P->nr;
        } else {
            jj = 0;
            ncr = -cr;
        }
    } else if (jj >= P->nr) {
        if (P->top == ORC_TOP_PERIODIC) {
            jj -= P->nr;
        } else if (P->top == ORC_TOP_FREESLIP) {
            jj = P->nr - 1;
            ncr = -cr;
        } else {
            kk = k;
            jj = j;
            ncz = -cz;
            ncr = -cr;
        }
    }
    kk = ((kk % P->nz) + P->nz) % P->nz;
    int d = 0;
    for (int q = 0; q < ORC_Q; q++) {
        if (orc_cz[q] == ncz && orc_cr[q] == ncr) d = q;
    }
    *kd = kk;
    *jd = jj;
    *id = d;
}

/* f_next = S(fpost): every post-collision population moves to its destination. */
void orc_stream(const orc_params* P, const double* fpost, double* fnext) {
    long n = (long)P->nz * P->nr;
    for (int i = 0; i < ORC_Q; i++) {
        #pragma omp parallel for
        for (int j = 0; j < P->nr; j++) {
            for (int k = 0; k < P->nz; k++) {
                int kd, jd, id;
                orc_stream_dest(P, k, j, i, &kd, &jd, &id);
                fnext[id * n + (long)jd * P->nz + kd] = fpost[i * n + (long)j * P->nz + k];
            }
        }
    }
}

/* ------------------------------------------------------------ the step -- */

/* Work arrays of one step; the extended ones carry ORC_G ghost layers. */
typedef struct {
    double *rho, *jz, *jr, *psi, *psiz, *psir, *psirr, *psirz, *fkz, *fkr;
    double *Fz, *Fr, *u0z, *u0r, *uz, *ur, *duzdr, *durdz, *durdr, *Hz, *Hr, *fpost;
} orc_work;

static void orc_work_free(orc_work* w) {
    double** p = (double**)w;
    for (size_t q = 0; q < sizeof(orc_work) / sizeof(double*); q++) free(p[q]);
}

static int orc_work_alloc(const orc_params* P, orc_work* w) {
    memset(w, 0, sizeof(*w));
    size_t m = (size_t)orc_ext_len(P);
    double** p = (double**)w;
    size_t nfields = sizeof(orc_work) / sizeof(double*) - 1;
    for (size_t q = 0; q < nfields; q++) {
        p[q] = (double*)calloc(m, sizeof(double));
        if (!p[q]) return -2;
    }
    w->fpost = (double*)calloc((size_t)ORC_Q * P->nz * P->nr, sizeof(double));
    return w->fpost ? 0 : -2;
}

/* Everything a step computes before collision: density, momentum, psi, the
 * forces, the physical velocity and the axisymmetric source ingredients.
 * Returns ORC_ERR_UNPHYSICAL when rho <= 0, psi^2 < 0 or a value is not finite. */
static int orc_fields(const orc_params* P, const double* f, orc_work* w) {
    long n = (long)P->nz * P->nr;
    int bad = 0;
    /* Moments, Sec. II.A: rho = sum_i f_i, j = sum_i c_i f_i. */
    #pragma omp parallel for reduction(|:bad)
    for (int j = 0; j < P->nr; j++) {
        for (int k = 0; k < P->nz; k++) {
            double rho = 0.0, jz = 0.0, jr = 0.0;
            for (int i = 0; i < ORC_Q; i++) {
                double fi = f[i * n + (long)j * P->nz + k];
                rho += fi;
                jz += orc_cz[i] * fi;
                jr += orc_cr[i] * fi;
            }
            if (!(rho > 0.0) || !isfinite(rho) || !isfinite(jz) || !isfinite(jr)) {
                bad = 1;
                continue;
            }
            long e = orc_ext(P, k, j);
            w->rho[e] = rho;
            w->jz[e] = jz;
            w->jr[e] = jr;
        }
    }
    if (bad) return ORC_ERR_UNPHYSICAL;
    /* Pseudopotential psi = sqrt(rho/3 - P_k(rho)) = sqrt(-U), Sec. II.C. */
    #pragma omp parallel for reduction(|:bad)
    for (int j = 0; j < P->nr; j++) {
        for (int k = 0; k < P->nz; k++) {
            long e = orc_ext(P, k, j);
            double psi = 0.0;
            if (P->multiphase) {
                double arg = w->rho[e] / 3.0 - orc_eos_p(P, w->rho[e]);
                if (!(arg >= 0.0) || !isfinite(arg)) {
                    bad = 1;
                    continue;
                }
                psi = sqrt(arg);
            }
            w->psi[e] = psi;
        }
    }
    if (bad) return ORC_ERR_UNPHYSICAL;
    orc_fill_ghosts(P, w->psi, +1, +1);

    /* F = F_K + F_axis + rho g. */
    for (int q = 0; q < orc_ext_len(P); q++) {
        w->fkz[q] = 0.0;
        w->fkr[q] = 0.0;
    }
    if (P->multiphase) {
        orc_force_kupershtokh(P, w->psi, w->fkz, w->fkr);
        /* psi_z, psi_r, then psi_rr = D_r(psi_r), psi_rz = D_r(psi_z). */
        orc_grad(P, w->psi, w->psiz, w->psir);
        orc_fill_ghosts(P, w->psiz, +1, +1);
        orc_fill_ghosts(P, w->psir, -1, -1);
        double* scratch = w->Hz; /* D_z of psi_r and psi_z is not needed; borrow Hz, Hr */
        orc_grad(P, w->psir, scratch, w->psirr);
        orc_grad(P, w->psiz, w->Hr, w->psirz);
    }
    #pragma omp parallel for reduction(|:bad)
    for (int j = 0; j < P->nr; j++) {
        double r = P->r0 + j + 0.5;
        for (int k = 0; k < P->nz; k++) {
            long e = orc_ext(P, k, j);
            double rho = w->rho[e];
            double fz = w->fkz[e] + rho * P->gz;
            double fr = w->fkr[e];
            if (P->multiphase && P->axis) {
                double az, ar;
                orc_force_axis(orc_kappa(P, rho), P->A, P->axis_a, r, w->psi[e], w->psiz[e], w->psir[e],
                               w->psirr[e], w->psirz[e], &az, &ar);
                fz += az;
                fr += ar;
            }
            w->Fz[e] = fz;
            w->Fr[e] = fr;
            /* u0 = j / rho (bare), physical u = u0 + F / (2 rho), Sec. II.A. */
            w->u0z[e] = w->jz[e] / rho;
            w->u0r[e] = w->jr[e] / rho;
            w->uz[e] = w->u0z[e] + fz / (2.0 * rho);
            w->ur[e] = w->u0r[e] + fr / (2.0 * rho);
            if (!isfinite(w->uz[e]) || !isfinite(w->ur[e])) bad = 1;
        }
    }
    if (bad) return ORC_ERR_UNPHYSICAL;
    /* Velocity derivatives for H (same stencil, physical u; u_z even, u_r odd
     * across the axis; at a no-slip top both odd). */
    if (P->axis) {
        orc_fill_ghosts(P, w->uz, +1, P->top == ORC_TOP_NOSLIP ? -1 : +1);
        orc_fill_ghosts(P, w->ur, -1, -1);
        orc_grad(P, w->uz, w->Hz, w->duzdr);
        orc_grad(P, w->ur, w->durdz, w->durdr);
        double nu = (P->tau - 0.5) / 3.0;
        #pragma omp parallel for
        for (int j = 0; j < P->nr; j++) {
            double r = P->r0 + j + 0.5;
            for (int k = 0; k < P->nz; k++) {
                long e = orc_ext(P, k, j);
                double rho = w->rho[e];
                orc_source_H(r, rho, rho * nu, w->uz[e], w->ur[e], w->duzdr[e], w->durdz[e],
                             w->durdr[e], P->hr_sign, &w->Hz[e], &w->Hr[e]);
            }
        }
    }
    return ORC_OK;
}

/* Guo forcing term of Sec. II.A with dt = 1 and c_s^2 = 1/3:
 * S_i = w_i (1 - 1/(2 tau)) [(c_i - u).F / c_s^2 + (c_i.u)(c_i.F) / c_s^4],
 * u the fluid velocity u0 + F/(2 rho).  The second term is printed as
 * (c_i - u).(c_i - F)/c_s^4, which is not a vector identity of Guo's scheme
 * (it is neither linear in F nor of zero mass); it is read as the second-order
 * Hermite term (c_i.u)(c_i.F)/c_s^4 of Guo et al., whose moments are
 * sum S_i = 0 and sum c_i S_i = (1 - 1/(2 tau)) F. */
void orc_guo_source(double tau, double uz, double ur, double Fz, double Fr, double* S) {
    double pre = 1.0 - 1.0 / (2.0 * tau);
    for (int i = 0; i < ORC_Q; i++) {
        double cmu_F = (orc_cz[i] - uz) * Fz + (orc_cr[i] - ur) * Fr;
        double cu = orc_cz[i] * uz + orc_cr[i] * ur;
        double cF = orc_cz[i] * Fz + orc_cr[i] * Fr;
        S[i] = orc_w[i] * pre * (3.0 * cmu_F + 9.0 * cu * cF);
    }
}

/* Collision with the axisymmetric source, Eq. (lbm) with h_i, and either
 * EDM forcing (Sec. II.C; the default):
 *   f*_i = f_i + (f_i^eq(rho,u0) - f_i)/tau + [f_i^eq(rho,u0+F/rho) - f_i^eq(rho,u0)] + h_i,
 * or Guo forcing (Sec. II.A), whose equilibrium takes the fluid velocity u:
 *   f*_i = f_i + (f_i^eq(rho,u) - f_i)/tau + S_i + h_i. */
static void orc_collide(const orc_params* P, const double* f, orc_work* w) {
    long n = (long)P->nz * P->nr;
    #pragma omp parallel for
    for (int j = 0; j < P->nr; j++) {
        double r = P->r0 + j + 0.5;
        for (int k = 0; k < P->nz; k++) {
            long e = orc_ext(P, k, j);
            double rho = w->rho[e];
            double feq[ORC_Q], S[ORC_Q], h[ORC_Q];
            if (P->forcing == ORC_FORCING_GUO) {
                orc_feq(rho, w->uz[e], w->ur[e], feq);
                orc_guo_source(P->tau, w->uz[e], w->ur[e], w->Fz[e], w->Fr[e], S);
            } else {
                double feq1[ORC_Q];
                orc_feq(rho, w->u0z[e], w->u0r[e], feq);
                orc_feq(rho, w->u0z[e] + w->Fz[e] / rho, w->u0r[e] + w->Fr[e] / rho, feq1);
                for (int i = 0; i < ORC_Q; i++) S[i] = feq1[i] - feq[i];
            }
            if (P->axis) {
                orc_source_h(r, rho, w->ur[e], w->Hz[e], w->Hr[e], h);
                if (P->h_eval == ORC_H_LINK_AVG)
                    for (int i = 0; i < ORC_Q; i++) h[i] *= 0.5; /* departure half, see orc_arrival_half */
            } else {
                for (int i = 0; i < ORC_Q; i++) h[i] = 0.0;
            }
            for (int i = 0; i < ORC_Q; i++) {
                long c = i * n + (long)j * P->nz + k;
                w->fpost[c] = f[c] + (feq[i] - f[c]) / P->tau + S[i] + h[i];
            }
        }
    }
}

/* h_i at the midpoint x + c_i/2 of the link, Eq. (lbm), read as the mean of
 * its two end nodes at time t (ORC_H_LINK_AVG): the population leaving x
 * carries h_i(x)/2 from the collision and receives h_i(y)/2 on arrival at y.
 * After a boundary rule the arrival term is that of the direction and node
 * the population arrives with; at the axis and at a free-slip top this is
 * the h_i of the mirror ghost node for the original direction, because
 * -rho u_r/r and H_z are even and H_r odd under r -> -r, u_r -> -u_r; at a
 * no-slip top (bounce-back) it is the reversed direction's h_i at the same node.
 * Called after streaming, with the fields of the step that just collided. */
static void orc_arrival_half(const orc_params* P, const orc_work* w, double* f) {
    long n = (long)P->nz * P->nr;
    #pragma omp parallel for
    for (int j = 0; j < P->nr; j++) {
        double r = P->r0 + j + 0.5;
        for (int k = 0; k < P->nz; k++) {
            long e = orc_ext(P, k, j);
            double h[ORC_Q];
            orc_source_h(r, w->rho[e], w->ur[e], w->Hz[e], w->Hr[e], h);
            for (int i = 0; i < ORC_Q; i++) f[i * n + (long)j * P->nz + k] += 0.5 * h[i];
        }
    }
}

/* Advance f (pre-collision populations, 9 x nr x nz) by nsteps in place. */
int orc_run(const orc_params* P, double* f, long nsteps) {
    orc_work w;
    if (orc_work_alloc(P, &w)) {
        orc_work_free(&w);
        return -2;
    }
    int rc = ORC_OK;
    for (long s = 0; s < nsteps && rc == ORC_OK; s++) {
        rc = orc_fields(P, f, &w);
        if (rc != ORC_OK) break;
        orc_collide(P, f, &w);
        orc_stream(P, w.fpost, f);
        if (P->axis && P->h_eval == ORC_H_LINK_AVG) orc_arrival_half(P, &w, f);
    }
    orc_work_free(&w);
    return rc;
}

/* f = f^eq(rho, u) at every node; the given u is taken as the bare velocity. */
void orc_init(const orc_params* P, const double* rho, const double* uz, const double* ur, double* f) {
    long n = (long)P->nz * P->nr;
    for (long c = 0; c < n; c++) {
        double feq[ORC_Q];
        orc_feq(rho[c], uz[c], ur[c], feq);
        for (int i = 0; i < ORC_Q; i++) f[i * n + c] = feq[i];
    }
}

/* Start with the given u as the PHYSICAL velocity (a fluid at rest when u = 0).
 * Sec. II.A defines the fluid velocity as u = u0 + F/(2 rho), u0 = sum_i c_i f_i / rho;
 * Sec. III starts its droplets from the equilibrium densities with the fluid at
 * rest.  So f = f^eq(rho, u - F/(2 rho)), with F = F_K + F_axis + rho g the force
 * of the density field itself (first evaluated on f^eq(rho, u), whose density is
 * rho up to rounding).  Returns ORC_ERR_UNPHYSICAL like a step. */
int orc_init_physical(const orc_params* P, const double* rho, const double* uz, const double* ur, double* f) {
    orc_init(P, rho, uz, ur, f);
    orc_work w;
    if (orc_work_alloc(P, &w)) {
        orc_work_free(&w);
        return -2;
    }
    int rc = orc_fields(P, f, &w);
    if (rc == ORC_OK) {
        long n = (long)P->nz * P->nr;
        for (int j = 0; j < P->nr; j++) {
            for (int k = 0; k < P->nz; k++) {
                long c = (long)j * P->nz + k, e = orc_ext(P, k, j);
                double feq[ORC_Q];
                orc_feq(rho[c], uz[c] - w.Fz[e] / (2.0 * w.rho[e]), ur[c] - w.Fr[e] / (2.0 * w.rho[e]), feq);
                for (int i = 0; i < ORC_Q; i++) f[i * n + c] = feq[i];
            }
        }
    }
    orc_work_free(&w);
    return rc;
}

/* Macroscopic output of the current state: rho, physical u = u0 + F/(2 rho),
 * P_k(rho) (or rho/3 for a single-phase run).  Optional diagnostics (may be
 * NULL): the total force and H fields of the step that would follow. */
int orc_moments(const orc_params* P, const double* f, double* rho, double* uz, double* ur, double* p,
                double* Fz, double* Fr, double* Hz, double* Hr) {
    orc_work w;
    if (orc_work_alloc(P, &w)) {
        orc_work_free(&w);
        return -2;
    }
    int rc = orc_fields(P, f, &w);
    if (rc == ORC_OK) {
        for (int j = 0; j < P->nr; j++) {
            for (int k = 0; k < P->nz; k++) {
                long e = orc_ext(P, k, j);
                long c = (long)j * P->nz + k;
                double d = w.rho[e];
                if (rho) rho[c] = d;
                if (uz) uz[c] = w.uz[e];
                if (ur) ur[c] = w.ur[e];
                if (p) p[c] = P->multiphase ? orc_eos_p(P, d) : d / 3.0;
                if (Fz) Fz[c] = w.Fz[e];
                if (Fr) Fr[c] = w.Fr[e];
                if (Hz) Hz[c] = P->axis ? w.Hz[e] : 0.0;
                if (Hr) Hr[c] = P->axis ? w.Hr[e] : 0.0;
            }
        }
    }
    orc_work_free(&w);
    return rc;
}

/* One collision without streaming (post-collision populations), for tests of
 * the collision operator's moments. */
int orc_collide_only(const orc_params* P, const double* f, double* fpost) {
    orc_work w;
    if (orc_work_alloc(P, &w)) {
        orc_work_free(&w);
        return -2;
    }
    int rc = orc_fields(P, f, &w);
    if (rc == ORC_OK) {
        orc_collide(P, f, &w);
        memcpy(fpost, w.fpost, sizeof(double) * ORC_Q * P->nz * P->nr);
    }
    orc_work_free(&w);
    return rc;
}

/* r-weighted mass sum_{k,j} (j + 1/2) sum_i f_i (the 2 pi factor omitted). */
double orc_mass_rweighted(const orc_params* P, const double* f) {
    long n = (long)P->nz * P->nr;
    double m = 0.0;
    for (int j = 0; j < P->nr; j++) {
        for (int k = 0; k < P->nz; k++) {
            double rho = 0.0;
            for (int i = 0; i < ORC_Q; i++) rho += f[i * n + (long)j * P->nz + k];
            m += (j + 0.5) * rho;
        }
    }
    return m;
}

/* Threads the whole-field passes use: n > 0 sets the count of an OpenMP build
 * (the plain build ignores it and runs on one thread); returns the count in use. */
#ifdef _OPENMP
#include <omp.h>
#endif
int orc_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Test hooks for extended (ghosted) fields: size and index of node (k, j). */
int orc_ghost_width(void) { return ORC_G; }
long orc_ext_index(const orc_params* P, int k, int j) { return orc_ext(P, k, j); }
