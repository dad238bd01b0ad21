/*
 * lfe_oracle.c -- plain FP64 CPU oracle for the alchemical nonbonded energy.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA path against a slow,
 * obviously correct restatement of the paper's definitions.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * What it computes (paper: Correa, Abreu, Nair, Tuckerman, "Integrated
 * Alchemical and Conformational Enhanced Sampling for Solvation Free Energy
 * Calculations"):
 *   U(lambda) = U_vv + U_uu + h_A(lambda) U_uv + h_B(lambda) U_soft      (Eq. 4)
 * where the classes vv (solvent-solvent), uu (solute-solute) and uv
 * (solute-solvent) split every nonbonded term, U_soft is the capped soft
 * Lennard-Jones basis of Eq. 5-6, and h_A, h_B are the switching functions of
 * Eq. 7-10.  Coulomb is Ewald-summed (Section 2.6 names PME; Darden 1993,
 * Essmann 1995):
 *   level 1: real-space erfc pairs + direct reciprocal k-sum (the definition)
 *   level 2: real-space erfc pairs + smooth PME on a K1 x K2 x K3 grid with
 *            order-n cardinal B-splines, transformed by a naive separable DFT
 *            (the defined PME approximation, Essmann 1995, Eq. 4.1-4.9).
 *
 * Readings where the paper is silent:
 *   - Lorentz-Berthelot mixing: sigma_ij = (sigma_i+sigma_j)/2,
 *     eps_ij = sqrt(eps_i eps_j).
 *   - LJ and soft-LJ are multiplied by the quintic switch
 *     S(t) = 1 - 10 t^3 + 15 t^4 - 6 t^5, t = (r - r_sw)/(r_c - r_sw),
 *     Coulomb is not switched; r_sw < 0 means plain truncation at r_c.
 *   - h_A scales the whole solute-solvent Coulomb interaction, including its
 *     reciprocal-space cross term and its share of the neutralising
 *     background (U_solu-solv is "the full" interaction, Section 2.2).
 *   - Neutralising background -k_e pi Q^2 / (2 V alpha^2), split into
 *     Q_v^2, Q_u^2 and 2 Q_u Q_v.
 *   - Excluded pairs (any distance, minimum image) contribute
 *     -k_e q_i q_j erf(alpha r)/r; 1-4 pairs (also listed as excluded) add
 *     s_C k_e q_i q_j / r + s_LJ LJ(r), unswitched and uncut.
 *   - Pairs with eps_ij = 0 carry no LJ or soft-LJ term.
 *
 * Optional soft-core coupling (the conventional alternative the paper sets
 * its linear-basis method against; the paper gives no formula): with
 * sc_alpha > 0 the solute-solvent Lennard-Jones term is replaced, at the
 * given sc_lambda, by the soft-core form of Beutler et al. (1994)
 *   U_sc(r, l) = 4 eps_ij l^p [1/D^2 - 1/D] S(r),  D = sc_alpha (1 - l) + (r/sigma_ij)^6,
 * p = sc_power; the solute-solvent Coulomb terms stay in U_uv (weighted by
 * h_A), U_soft holds U_sc at sc_lambda (weighted by 1), and E[24] holds
 *   dU_sc/dl = 4 eps_ij S [p l^(p-1) (1/D^2 - 1/D) + sc_alpha l^p (2/D^3 - 1/D^2)],
 * so that U = U_vv + U_uu + h_A U_uv + U_soft and
 * dU/dl = h_A' U_uv + E[24], F = F0 + h_A Fuv + Fsoft.
 *
 * Units: nm, kJ/mol, e.  k_e = 138.935458 kJ mol^-1 nm e^-2.
 *
 * Energy array E[ORC_NE] layout (all kJ/mol):
 *   0 U_vv   1 U_uu   2 U_uv   3 U_soft
 *   4 coul_real_vv   5 coul_real_uu   6 coul_real_uv
 *   7 rec_vv         8 rec_uu         9 rec_uv
 *  10 self_vv       11 self_uu
 *  12 bg_vv         13 bg_uu         14 bg_uv
 *  15 lj_vv         16 lj_uu         17 lj_uv
 *  18 excl_vv       19 excl_uu       20 excl_uv
 *  21 pair14_vv     22 pair14_uu
 *  23 number of non-excluded pairs with r < r_c (as a double)
 *  24 dU_sc/dlambda (soft-core coupling only; 0 otherwise)
 * Force arrays (each [3N], any may be NULL) hold -grad of one basis:
 *   F0    = -grad (U_vv + U_uu)
 *   Fuv   = -grad U_uv
 *   Fsoft = -grad U_soft
 * so that F(lambda) = F0 + h_A Fuv + h_B Fsoft.
 *
 * orc_param_grad gives the class-resolved derivatives of the same energies
 * with respect to every atom's charge, sigma and epsilon (the gradients that
 * force-field fitting to solvation free energies needs); the reciprocal part
 * is the potential of each class at the atom's site.  Reading: where
 * eps_i = 0 the derivative of eps_ij = sqrt(eps_i eps_j) is singular and is
 * reported as 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_KE 138.935458
#define ORC_NE 25
#define ORC_PI 3.14159265358979323846

typedef struct {
    double box[3];
    double r_cut;
    double r_switch;   /* < 0: no LJ switch */
    double alpha;      /* Ewald splitting parameter, nm^-1 */
    int level;         /* 1: direct k-sum, 2: smooth PME, 0: no reciprocal */
    int kmax[3];       /* level 1: |m_d| <= kmax[d] */
    int grid[3];       /* level 2: K1, K2, K3 */
    int order;         /* level 2: B-spline order n */
    double sc_alpha;   /* > 0: soft-core solute-solvent LJ at sc_lambda (see above) */
    double sc_power;
    double sc_lambda;
} orc_params;

/* ---------------------------------------------------------------- helpers */

/* Capped soft-LJ reduced potential u_cap(x) and its derivative (Eq. 6). */
double orc_ucap(double x, double* du)
{
    if (x < 1.0) {
        double x2 = x * x, x3 = x2 * x, x4 = x3 * x, x5 = x4 * x, x6 = x5 * x;
        if (du) *du = -6.0 * 868.0 * x5 + 5.0 * 2188.8 * x4 - 4.0 * 1440.0 * x3;
        return -868.0 * x6 + 2188.8 * x5 - 1440.0 * x4 + 119.2;
    } else {
        double i6 = 1.0 / (x * x * x * x * x * x);
        if (du) *du = (-48.0 * i6 * i6 + 24.0 * i6) / x;
        return 4.0 * i6 * i6 - 4.0 * i6;
    }
}

/* Smoothstep S22 (Eq. 9) and S32 (Eq. 10) with derivatives. */
double orc_S22(double x, double* d)
{
    if (x <= 0.0) { if (d) *d = 0.0; return 0.0; }
    if (x >= 1.0) { if (d) *d = 0.0; return 1.0; }
    if (d) *d = 30.0 * x * x * x * x - 60.0 * x * x * x + 30.0 * x * x;
    return 6.0 * pow(x, 5) - 15.0 * pow(x, 4) + 10.0 * pow(x, 3);
}

double orc_S32(double x, double* d)
{
    if (x <= 0.0) { if (d) *d = 0.0; return 0.0; }
    if (x >= 1.0) { if (d) *d = 0.0; return 1.0; }
    if (d) *d = 60.0 * pow(x, 5) - 120.0 * pow(x, 4) + 60.0 * pow(x, 3);
    return 10.0 * pow(x, 6) - 24.0 * pow(x, 5) + 15.0 * pow(x, 4);
}

/* h_A and h_B of Eq. 7-8 and their lambda-derivatives. */
void orc_switching(double lam, double* hA, double* hB, double* dhA, double* dhB)
{
    double d32, d22;
    double a = orc_S32((lam - 0.35) / 0.65, &d32);
    double s22 = orc_S22(lam, &d22);
    *hA = a;
    *hB = s22 - a;
    *dhA = d32 / 0.65;
    *dhB = d22 - d32 / 0.65;
}

/* Quintic LJ switch (reading: smoothstep from r_sw to r_c). */
double orc_switch(double r, double rc, double rs, double* dS)
{
    if (rs < 0.0 || r <= rs) { *dS = 0.0; return 1.0; }
    if (r >= rc) { *dS = 0.0; return 0.0; }
    double w = rc - rs, t = (r - rs) / w;
    double t2 = t * t, t3 = t2 * t;
    *dS = (-30.0 * t2 + 60.0 * t3 - 30.0 * t2 * t2) / w;
    return 1.0 - 10.0 * t3 + 15.0 * t3 * t - 6.0 * t3 * t2;
}

static void min_image(double d[3], const double box[3])
{
    for (int k = 0; k < 3; ++k) d[k] -= box[k] * nearbyint(d[k] / box[k]);
}

/* Class of a pair: 0 vv, 1 uu, 2 uv. */
static int pair_class(unsigned char a, unsigned char b)
{
    if (a && b) return 1;
    if (!a && !b) return 0;
    return 2;
}

/* ------------------------------------------------- real-space pair terms */

/* Full double loop over ordered pairs i != j; every energy gets a factor 1/2,
 * every force goes to atom i only.  No Newton-third-law bookkeeping. */
static void real_space(const orc_params* p, int n, const double* pos, const double* q,
                       const double* sig, const double* eps, const unsigned char* solute,
                       const int* ex_start, const int* ex_list,
                       double* E, double* F0, double* Fuv, double* Fsoft)
{
    const double rc = p->r_cut, rs = p->r_switch, a = p->alpha;
    const double rc2 = rc * rc;
    double e_c[3] = {0, 0, 0}, e_lj[3] = {0, 0, 0}, e_soft = 0.0, npairs = 0.0, e_dsc = 0.0;
    const int sc = p->sc_alpha > 0.0;
    const double lam = p->sc_lambda, sa = p->sc_alpha, sp = p->sc_power;

#pragma omp parallel
    {
        char* mark = (char*)calloc((size_t)n, 1);
        double tc[3] = {0, 0, 0}, tlj[3] = {0, 0, 0}, tsoft = 0.0, tnp = 0.0, tdsc = 0.0;
#pragma omp for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            for (int e = ex_start[i]; e < ex_start[i + 1]; ++e) mark[ex_list[e]] = 1;
            double f0[3] = {0, 0, 0}, fuv[3] = {0, 0, 0}, fs[3] = {0, 0, 0};
            for (int j = 0; j < n; ++j) {
                if (j == i || mark[j]) continue;
                double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1],
                               pos[3 * j + 2] - pos[3 * i + 2]};
                min_image(d, p->box);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 >= rc2) continue;
                double r = sqrt(r2);
                int c = pair_class(solute[i], solute[j]);
                tnp += 0.5;
                /* Coulomb, real space: k_e q_i q_j erfc(alpha r)/r */
                double qq = ORC_KE * q[i] * q[j];
                double ec = qq * erfc(a * r) / r;
                double dec = -ec / r - qq * 2.0 * a / sqrt(ORC_PI) * exp(-a * a * r2) / r;
                tc[c] += 0.5 * ec;
                /* LJ (Lorentz-Berthelot, switched) */
                double s = 0.5 * (sig[i] + sig[j]);
                double ep = sqrt(eps[i] * eps[j]);
                double dS, S = orc_switch(r, rc, rs, &dS);
                double elj = 0.0, delj = 0.0;
                if (sc && c == 2) {
                    /* soft-core solute-solvent LJ at lambda (the soft slot) */
                    if (ep > 0.0 && s > 0.0) {
                        double x6 = pow(r / s, 6), D = sa * (1.0 - lam) + x6;
                        double lp = pow(lam, sp), u = 1.0 / (D * D) - 1.0 / D;
                        double du_dD = -2.0 / (D * D * D) + 1.0 / (D * D);
                        double es = 4.0 * ep * lp * u * S;
                        double des = 4.0 * ep * lp * (du_dD * 6.0 * x6 / r * S + u * dS);
                        double dl = 4.0 * ep * S * (sp * pow(lam, sp - 1.0) * u + sa * lp * (2.0 / (D * D * D) - 1.0 / (D * D)));
                        tsoft += 0.5 * es;
                        tdsc += 0.5 * dl;
                        double gs = des / r;
                        fs[0] += gs * d[0]; fs[1] += gs * d[1]; fs[2] += gs * d[2];
                    }
                    double g = dec / r;
                    fuv[0] += g * d[0]; fuv[1] += g * d[1]; fuv[2] += g * d[2];
                    continue;
                }
                if (ep > 0.0) {
                    double sr6 = pow(s / r, 6);
                    double v = 4.0 * ep * (sr6 * sr6 - sr6);
                    double dv = 4.0 * ep * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r;
                    elj = v * S;
                    delj = dv * S + v * dS;
                }
                tlj[c] += 0.5 * elj;
                /* dU/dr along d = r_j - r_i: force on i is +dU/dr * d/r */
                double g = (dec + delj) / r;
                if (c == 2) {
                    fuv[0] += g * d[0]; fuv[1] += g * d[1]; fuv[2] += g * d[2];
                    /* soft basis, Eq. 5-6 */
                    if (ep > 0.0 && s > 0.0) {
                        double du, u = orc_ucap(r / s, &du);
                        double es = ep * u * S;
                        double des = ep * (du / s * S + u * dS);
                        tsoft += 0.5 * es;
                        double gs = des / r;
                        fs[0] += gs * d[0]; fs[1] += gs * d[1]; fs[2] += gs * d[2];
                    }
                } else {
                    f0[0] += g * d[0]; f0[1] += g * d[1]; f0[2] += g * d[2];
                }
            }
            for (int e = ex_start[i]; e < ex_start[i + 1]; ++e) mark[ex_list[e]] = 0;
            for (int k = 0; k < 3; ++k) {
                if (F0) F0[3 * i + k] += f0[k];
                if (Fuv) Fuv[3 * i + k] += fuv[k];
                if (Fsoft) Fsoft[3 * i + k] += fs[k];
            }
        }
#pragma omp critical
        {
            for (int c = 0; c < 3; ++c) { e_c[c] += tc[c]; e_lj[c] += tlj[c]; }
            e_soft += tsoft;
            e_dsc += tdsc;
            npairs += tnp;
        }
        free(mark);
    }
    E[4] += e_c[0]; E[5] += e_c[1]; E[6] += e_c[2];
    E[15] += e_lj[0]; E[16] += e_lj[1]; E[17] += e_lj[2];
    E[3] += e_soft;
    E[23] += npairs;
    E[24] += e_dsc;
}

static double* basis_for_class(int c, double* F0, double* Fuv)
{
    return c == 2 ? Fuv : F0;
}

static void add_pair_force(double* F, int i, int j, double g, const double d[3])
{
    /* d = r_j - r_i, g = (dU/dr)/r: force on i = +g d, on j = -g d */
    if (!F) return;
    for (int k = 0; k < 3; ++k) { F[3 * i + k] += g * d[k]; F[3 * j + k] -= g * d[k]; }
}

/* Excluded pairs: -k_e q_i q_j erf(alpha r)/r at the minimum image. */
static void exclusion_terms(const orc_params* p, const double* pos, const double* q,
                            const unsigned char* solute, int n_excl, const int* excl,
                            double* E, double* F0, double* Fuv)
{
    const double a = p->alpha;
    for (int e = 0; e < n_excl; ++e) {
        int i = excl[2 * e], j = excl[2 * e + 1];
        double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1],
                       pos[3 * j + 2] - pos[3 * i + 2]};
        min_image(d, p->box);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double r = sqrt(r2);
        double qq = ORC_KE * q[i] * q[j];
        double u, du;
        if (r < 1e-12) {
            /* limit r -> 0 of erf(a r)/r is 2a/sqrt(pi); force 0 */
            u = -qq * 2.0 * a / sqrt(ORC_PI);
            du = 0.0;
        } else {
            u = -qq * erf(a * r) / r;
            du = qq * erf(a * r) / r2 - qq * 2.0 * a / sqrt(ORC_PI) * exp(-a * a * r2) / r;
        }
        int c = pair_class(solute[i], solute[j]);
        E[18 + c] += u;
        add_pair_force(basis_for_class(c, F0, Fuv), i, j, du / (r > 1e-12 ? r : 1.0), d);
    }
}

/* 1-4 pairs: s_C k_e q_i q_j / r + s_LJ 4 eps_ij [(s/r)^12 - (s/r)^6]. */
static void pair14_terms(const orc_params* p, const double* pos, const double* q,
                         const double* sig, const double* eps, const unsigned char* solute,
                         int n14, const int* p14, const double* s14,
                         double* E, double* F0, double* Fuv)
{
    for (int e = 0; e < n14; ++e) {
        int i = p14[2 * e], j = p14[2 * e + 1];
        double sLJ = s14[2 * e], sC = s14[2 * e + 1];
        double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1],
                       pos[3 * j + 2] - pos[3 * i + 2]};
        min_image(d, p->box);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double r = sqrt(r2);
        double qq = ORC_KE * q[i] * q[j];
        double u = sC * qq / r, du = -sC * qq / r2;
        double s = 0.5 * (sig[i] + sig[j]), ep = sqrt(eps[i] * eps[j]);
        if (ep > 0.0) {
            double sr6 = pow(s / r, 6);
            u += sLJ * 4.0 * ep * (sr6 * sr6 - sr6);
            du += sLJ * 4.0 * ep * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r;
        }
        int c = pair_class(solute[i], solute[j]);
        if (c == 2) E[20] += u; /* a uv 1-4 pair is not expected; keep it in uv */
        else E[21 + c] += u;
        add_pair_force(basis_for_class(c, F0, Fuv), i, j, du / r, d);
    }
}

/* Self and neutralising-background terms. */
static void self_background(const orc_params* p, int n, const double* q,
                            const unsigned char* solute, double* E)
{
    double a = p->alpha, V = p->box[0] * p->box[1] * p->box[2];
    double s2[2] = {0, 0}, Q[2] = {0, 0};
    for (int i = 0; i < n; ++i) {
        int c = solute[i] ? 1 : 0;
        s2[c] += q[i] * q[i];
        Q[c] += q[i];
    }
    E[10] = -ORC_KE * a / sqrt(ORC_PI) * s2[0];
    E[11] = -ORC_KE * a / sqrt(ORC_PI) * s2[1];
    double pre = -ORC_KE * ORC_PI / (2.0 * V * a * a);
    E[12] = pre * Q[0] * Q[0];
    E[13] = pre * Q[1] * Q[1];
    E[14] = pre * 2.0 * Q[0] * Q[1];
}

/* ------------------------------------------- level 1: direct Ewald k-sum */

static void ewald_ksum(const orc_params* p, int n, const double* pos, const double* q,
                       const unsigned char* solute, double* E, double* F0, double* Fuv, double* phi2)
{
    const double a = p->alpha;
    const double V = p->box[0] * p->box[1] * p->box[2];
    const int K0 = p->kmax[0], K1 = p->kmax[1], K2 = p->kmax[2];
    const int W0 = 2 * K0 + 1, W1 = 2 * K1 + 1, W2 = 2 * K2 + 1;
    /* per-atom tables e^{i 2 pi m x / L} for m = -kmax..kmax (separable exponent) */
    double* tc[3]; double* ts[3];
    int W[3] = {W0, W1, W2}, Km[3] = {K0, K1, K2};
    for (int d = 0; d < 3; ++d) {
        tc[d] = (double*)malloc(sizeof(double) * (size_t)n * W[d]);
        ts[d] = (double*)malloc(sizeof(double) * (size_t)n * W[d]);
        for (int i = 0; i < n; ++i)
            for (int m = -Km[d]; m <= Km[d]; ++m) {
                double ph = 2.0 * ORC_PI * m * pos[3 * i + d] / p->box[d];
                tc[d][(size_t)i * W[d] + m + Km[d]] = cos(ph);
                ts[d][(size_t)i * W[d] + m + Km[d]] = sin(ph);
            }
    }
    /* half space of m: mx > 0, or mx = 0 and my > 0, or mx = my = 0 and mz > 0 */
    int nk = 0;
    int* ml = (int*)malloc(sizeof(int) * 3 * (size_t)W0 * W1 * W2);
    for (int mx = 0; mx <= K0; ++mx)
        for (int my = -K1; my <= K1; ++my)
            for (int mz = -K2; mz <= K2; ++mz) {
                if (mx == 0 && (my < 0 || (my == 0 && mz <= 0))) continue;
                ml[3 * nk] = mx; ml[3 * nk + 1] = my; ml[3 * nk + 2] = mz; ++nk;
            }
    double* S = (double*)malloc(sizeof(double) * 4 * (size_t)nk); /* Re Sv, Im Sv, Re Su, Im Su */
    double* gk = (double*)malloc(sizeof(double) * (size_t)nk);
    double* kv = (double*)malloc(sizeof(double) * 3 * (size_t)nk);
    double evv = 0, euu = 0, euv = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : evv, euu, euv)
    for (int t = 0; t < nk; ++t) {
        int mx = ml[3 * t], my = ml[3 * t + 1], mz = ml[3 * t + 2];
        double k[3] = {2.0 * ORC_PI * mx / p->box[0], 2.0 * ORC_PI * my / p->box[1],
                       2.0 * ORC_PI * mz / p->box[2]};
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double g = exp(-k2 / (4.0 * a * a)) / k2;
        double s[4] = {0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            size_t ix = (size_t)i * W0 + mx + K0, iy = (size_t)i * W1 + my + K1,
                   iz = (size_t)i * W2 + mz + K2;
            double cxy = tc[0][ix] * tc[1][iy] - ts[0][ix] * ts[1][iy];
            double sxy = tc[0][ix] * ts[1][iy] + ts[0][ix] * tc[1][iy];
            double c = cxy * tc[2][iz] - sxy * ts[2][iz];
            double sn = cxy * ts[2][iz] + sxy * tc[2][iz];
            int u = solute[i] ? 2 : 0;
            s[u] += q[i] * c;
            s[u + 1] += q[i] * sn;
        }
        S[4 * t] = s[0]; S[4 * t + 1] = s[1]; S[4 * t + 2] = s[2]; S[4 * t + 3] = s[3];
        gk[t] = g;
        kv[3 * t] = k[0]; kv[3 * t + 1] = k[1]; kv[3 * t + 2] = k[2];
        /* factor 2 for the half space */
        evv += 2.0 * g * (s[0] * s[0] + s[1] * s[1]);
        euu += 2.0 * g * (s[2] * s[2] + s[3] * s[3]);
        euv += 2.0 * g * 2.0 * (s[2] * s[0] + s[3] * s[1]);
    }
    double pre = 2.0 * ORC_PI * ORC_KE / V;
    E[7] += pre * evv; E[8] += pre * euu; E[9] += pre * euv;
    /* forces: F_i = (4 pi k_e / V) q_i sum_k g k Im(S_c*(k) e^{i k r_i}), x2 for half space */
    double fpre = 2.0 * 4.0 * ORC_PI * ORC_KE / V;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double f0[3] = {0, 0, 0}, fuv[3] = {0, 0, 0};
        double pv = 0.0, pu = 0.0;
        int own = solute[i] ? 2 : 0, oth = solute[i] ? 0 : 2;
        for (int t = 0; t < nk; ++t) {
            int mx = ml[3 * t], my = ml[3 * t + 1], mz = ml[3 * t + 2];
            size_t ix = (size_t)i * W0 + mx + K0, iy = (size_t)i * W1 + my + K1,
                   iz = (size_t)i * W2 + mz + K2;
            double cxy = tc[0][ix] * tc[1][iy] - ts[0][ix] * ts[1][iy];
            double sxy = tc[0][ix] * ts[1][iy] + ts[0][ix] * tc[1][iy];
            double c = cxy * tc[2][iz] - sxy * ts[2][iz];
            double sn = cxy * ts[2][iz] + sxy * tc[2][iz];
            /* Im(conj(S) e^{i phi}) = Re S * sin - Im S * cos */
            double im_own = S[4 * t + own] * sn - S[4 * t + own + 1] * c;
            double im_oth = S[4 * t + oth] * sn - S[4 * t + oth + 1] * c;
            for (int d = 0; d < 3; ++d) {
                f0[d] += gk[t] * kv[3 * t + d] * im_own;
                fuv[d] += gk[t] * kv[3 * t + d] * im_oth;
            }
            /* potential of class c at r_i: (4 pi k_e / V) sum_full g Re(S_c* e^{i k r_i}) */
            pv += gk[t] * (S[4 * t] * c + S[4 * t + 1] * sn);
            pu += gk[t] * (S[4 * t + 2] * c + S[4 * t + 3] * sn);
        }
        if (phi2) {
            phi2[2 * i] = fpre * pv;
            phi2[2 * i + 1] = fpre * pu;
        }
        for (int d = 0; d < 3; ++d) {
            if (F0) F0[3 * i + d] += fpre * q[i] * f0[d];
            if (Fuv) Fuv[3 * i + d] += fpre * q[i] * fuv[d];
        }
    }
    for (int d = 0; d < 3; ++d) { free(tc[d]); free(ts[d]); }
    free(ml); free(S); free(gk); free(kv);
}

/* --------------------------------------------- level 2: smooth PME (SPME) */

/* Cardinal B-spline M_n(u) by its recursion (Essmann 1995, Eq. 4.1). */
double orc_bspline(int n, double u)
{
    if (n == 2) return (u < 0.0 || u > 2.0) ? 0.0 : 1.0 - fabs(u - 1.0);
    return u / (n - 1) * orc_bspline(n - 1, u) + (n - u) / (n - 1) * orc_bspline(n - 1, u - 1.0);
}

/* dM_n/du = M_{n-1}(u) - M_{n-1}(u - 1) (Essmann 1995, Eq. 4.2). */
static double bspline_d(int n, double u)
{
    return orc_bspline(n - 1, u) - orc_bspline(n - 1, u - 1.0);
}

/* |b(m)|^2 (Essmann 1995, Eq. 4.4). */
double orc_bmod2(int n, int K, int m)
{
    double re = 0.0, im = 0.0;
    for (int k = 0; k <= n - 2; ++k) {
        double w = orc_bspline(n, k + 1.0);
        re += w * cos(2.0 * ORC_PI * m * k / K);
        im += w * sin(2.0 * ORC_PI * m * k / K);
    }
    return 1.0 / (re * re + im * im);
}

/* naive 1-D DFT of every line along axis `ax` of a complex K0*K1*K2 array
 * (layout index = (i0*K1 + i1)*K2 + i2), sign = +1 or -1 in the exponent. */
static void dft_axis(double* re, double* im, const int K[3], int ax, int sign)
{
    int Ka = K[ax];
    int stride = (ax == 0) ? K[1] * K[2] : (ax == 1) ? K[2] : 1;
    int nlines = K[0] * K[1] * K[2] / Ka;
    double* cw = (double*)malloc(sizeof(double) * Ka);
    double* sw = (double*)malloc(sizeof(double) * Ka);
    for (int t = 0; t < Ka; ++t) {
        cw[t] = cos(2.0 * ORC_PI * t / Ka);
        sw[t] = sign * sin(2.0 * ORC_PI * t / Ka);
    }
#pragma omp parallel
    {
        double* br = (double*)malloc(sizeof(double) * Ka);
        double* bi = (double*)malloc(sizeof(double) * Ka);
#pragma omp for
        for (int l = 0; l < nlines; ++l) {
            /* base offset of line l */
            int base;
            if (ax == 0) base = l;                                   /* (i1,i2) */
            else if (ax == 1) base = (l / K[2]) * K[1] * K[2] + l % K[2]; /* (i0,i2) */
            else base = l * K[2];                                    /* (i0,i1) */
            for (int m = 0; m < Ka; ++m) {
                double sr = 0.0, si = 0.0;
                for (int k = 0; k < Ka; ++k) {
                    int t = (int)(((long)m * k) % Ka);
                    double xr = re[base + k * stride], xi = im[base + k * stride];
                    sr += xr * cw[t] - xi * sw[t];
                    si += xr * sw[t] + xi * cw[t];
                }
                br[m] = sr; bi[m] = si;
            }
            for (int m = 0; m < Ka; ++m) { re[base + m * stride] = br[m]; im[base + m * stride] = bi[m]; }
        }
        free(br); free(bi);
    }
    free(cw); free(sw);
}

static void spme(const orc_params* p, int n, const double* pos, const double* q,
                 const unsigned char* solute, double* E, double* F0, double* Fuv, double* phi2)
{
    const int K[3] = {p->grid[0], p->grid[1], p->grid[2]};
    const int no = p->order;
    const size_t G = (size_t)K[0] * K[1] * K[2];
    const double V = p->box[0] * p->box[1] * p->box[2];
    const double a = p->alpha;
    /* grids: class 0 solvent, class 1 solute */
    double* Qr[2]; double* Qi[2];
    for (int c = 0; c < 2; ++c) {
        Qr[c] = (double*)calloc(G, sizeof(double));
        Qi[c] = (double*)calloc(G, sizeof(double));
    }
    /* spread: Q_c(k) = sum_{i in c} q_i prod_d M_n(u_id - k_d) over periodic images */
    double* u = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            double s = pos[3 * i + d] / p->box[d];
            s -= floor(s);
            u[3 * i + d] = K[d] * s;
        }
    for (int i = 0; i < n; ++i) {
        int c = solute[i] ? 1 : 0;
        int f[3];
        for (int d = 0; d < 3; ++d) f[d] = (int)floor(u[3 * i + d]);
        /* grid points k with 0 < u - k < n: k = f - j, j = 0..n-1 */
        for (int j0 = 0; j0 < no; ++j0)
            for (int j1 = 0; j1 < no; ++j1)
                for (int j2 = 0; j2 < no; ++j2) {
                    int k0 = f[0] - j0, k1 = f[1] - j1, k2 = f[2] - j2;
                    double w = orc_bspline(no, u[3 * i] - k0) * orc_bspline(no, u[3 * i + 1] - k1) *
                               orc_bspline(no, u[3 * i + 2] - k2);
                    k0 = ((k0 % K[0]) + K[0]) % K[0];
                    k1 = ((k1 % K[1]) + K[1]) % K[1];
                    k2 = ((k2 % K[2]) + K[2]) % K[2];
                    Qr[c][((size_t)k0 * K[1] + k1) * K[2] + k2] += q[i] * w;
                }
    }
    /* F(Q)(m) = sum_k Q(k) exp(+2 pi i m.k/K) */
    for (int c = 0; c < 2; ++c)
        for (int ax = 0; ax < 3; ++ax) dft_axis(Qr[c], Qi[c], K, ax, +1);
    /* influence function G(m) = k_e/(pi V) exp(-pi^2 m^2/alpha^2)/m^2 B(m) */
    double* Gm = (double*)malloc(sizeof(double) * G);
    double* b2[3];
    for (int d = 0; d < 3; ++d) {
        b2[d] = (double*)malloc(sizeof(double) * K[d]);
        for (int m = 0; m < K[d]; ++m) b2[d][m] = orc_bmod2(no, K[d], m);
    }
    double evv = 0, euu = 0, euv = 0;
    for (int m0 = 0; m0 < K[0]; ++m0)
        for (int m1 = 0; m1 < K[1]; ++m1)
            for (int m2 = 0; m2 < K[2]; ++m2) {
                size_t idx = ((size_t)m0 * K[1] + m1) * K[2] + m2;
                int mm[3] = {m0, m1, m2};
                double msq = 0.0;
                for (int d = 0; d < 3; ++d) {
                    int md = (mm[d] <= K[d] / 2) ? mm[d] : mm[d] - K[d];
                    double mr = md / p->box[d];
                    msq += mr * mr;
                }
                double g = 0.0;
                if (idx != 0)
                    g = ORC_KE / (ORC_PI * V) * exp(-ORC_PI * ORC_PI * msq / (a * a)) / msq *
                        b2[0][m0] * b2[1][m1] * b2[2][m2];
                Gm[idx] = g;
                evv += 0.5 * g * (Qr[0][idx] * Qr[0][idx] + Qi[0][idx] * Qi[0][idx]);
                euu += 0.5 * g * (Qr[1][idx] * Qr[1][idx] + Qi[1][idx] * Qi[1][idx]);
                euv += g * (Qr[1][idx] * Qr[0][idx] + Qi[1][idx] * Qi[0][idx]);
            }
    E[7] += evv; E[8] += euu; E[9] += euv;
    /* potentials phi_c(k) = sum_m G(m) F(Q_c)(m) exp(-2 pi i m.k/K) */
    for (int c = 0; c < 2; ++c) {
        for (size_t idx = 0; idx < G; ++idx) { Qr[c][idx] *= Gm[idx]; Qi[c][idx] *= Gm[idx]; }
        for (int ax = 0; ax < 3; ++ax) dft_axis(Qr[c], Qi[c], K, ax, -1);
    }
    /* forces: F_i = -q_i sum_k grad theta_i(k) phi(k) */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        int own = solute[i] ? 1 : 0, oth = 1 - own;
        int f[3];
        for (int d = 0; d < 3; ++d) f[d] = (int)floor(u[3 * i + d]);
        double g0[3] = {0, 0, 0}, g1[3] = {0, 0, 0};
        double pot[2] = {0.0, 0.0};
        for (int j0 = 0; j0 < no; ++j0)
            for (int j1 = 0; j1 < no; ++j1)
                for (int j2 = 0; j2 < no; ++j2) {
                    int k[3] = {f[0] - j0, f[1] - j1, f[2] - j2};
                    double w[3], dw[3];
                    for (int d = 0; d < 3; ++d) {
                        w[d] = orc_bspline(no, u[3 * i + d] - k[d]);
                        dw[d] = bspline_d(no, u[3 * i + d] - k[d]) * K[d] / p->box[d];
                    }
                    for (int d = 0; d < 3; ++d) k[d] = ((k[d] % K[d]) + K[d]) % K[d];
                    size_t idx = ((size_t)k[0] * K[1] + k[1]) * K[2] + k[2];
                    double grad[3] = {dw[0] * w[1] * w[2], w[0] * dw[1] * w[2], w[0] * w[1] * dw[2]};
                    for (int d = 0; d < 3; ++d) {
                        g0[d] += grad[d] * Qr[own][idx];
                        g1[d] += grad[d] * Qr[oth][idx];
                    }
                    pot[0] += w[0] * w[1] * w[2] * Qr[0][idx];
                    pot[1] += w[0] * w[1] * w[2] * Qr[1][idx];
                }
        if (phi2) {
            phi2[2 * i] = pot[0];
            phi2[2 * i + 1] = pot[1];
        }
        for (int d = 0; d < 3; ++d) {
            if (F0) F0[3 * i + d] -= q[i] * g0[d];
            if (Fuv) Fuv[3 * i + d] -= q[i] * g1[d];
        }
    }
    for (int c = 0; c < 2; ++c) { free(Qr[c]); free(Qi[c]); }
    for (int d = 0; d < 3; ++d) free(b2[d]);
    free(Gm); free(u);
}

/* ------------------------------------------------------------- entry */

static void build_exclusion_csr(int n, int n_excl, const int* excl, int** start, int** list)
{
    int* cnt = (int*)calloc((size_t)n + 1, sizeof(int));
    for (int e = 0; e < n_excl; ++e) { cnt[excl[2 * e] + 1]++; cnt[excl[2 * e + 1] + 1]++; }
    for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int* l = (int*)malloc(sizeof(int) * (size_t)(2 * n_excl + 1));
    int* fill = (int*)calloc((size_t)n, sizeof(int));
    for (int e = 0; e < n_excl; ++e) {
        int i = excl[2 * e], j = excl[2 * e + 1];
        l[cnt[i] + fill[i]++] = j;
        l[cnt[j] + fill[j]++] = i;
    }
    free(fill);
    *start = cnt;
    *list = l;
}

int orc_nonbonded(const orc_params* p, int n, const double* pos, const double* q,
                  const double* sig, const double* eps, const unsigned char* solute,
                  int n_excl, const int* excl, int n14, const int* p14, const double* s14,
                  double* E, double* F0, double* Fuv, double* Fsoft)
{
    if (n <= 0 || !p || !pos || !q || !sig || !eps || !solute || !E) return -1;
    for (int d = 0; d < 3; ++d)
        if (!(p->r_cut <= 0.5 * p->box[d])) return -2;
    memset(E, 0, sizeof(double) * ORC_NE);
    if (F0) memset(F0, 0, sizeof(double) * 3 * (size_t)n);
    if (Fuv) memset(Fuv, 0, sizeof(double) * 3 * (size_t)n);
    if (Fsoft) memset(Fsoft, 0, sizeof(double) * 3 * (size_t)n);
    int *st, *li;
    build_exclusion_csr(n, n_excl, excl, &st, &li);
    real_space(p, n, pos, q, sig, eps, solute, st, li, E, F0, Fuv, Fsoft);
    free(st); free(li);
    exclusion_terms(p, pos, q, solute, n_excl, excl, E, F0, Fuv);
    pair14_terms(p, pos, q, sig, eps, solute, n14, p14, s14, E, F0, Fuv);
    if (p->level != 0) {
        self_background(p, n, q, solute, E);
        if (p->level == 1) ewald_ksum(p, n, pos, q, solute, E, F0, Fuv, NULL);
        else spme(p, n, pos, q, solute, E, F0, Fuv, NULL);
    }
    E[0] = E[4] + E[7] + E[10] + E[12] + E[15] + E[18] + E[21];
    E[1] = E[5] + E[8] + E[11] + E[13] + E[16] + E[19] + E[22];
    E[2] = E[6] + E[9] + E[14] + E[17] + E[20];
    return 0;
}

/* ---------------------------------------------------------- bonded terms */

/* Harmonic bonds 1/2 k (r - r0)^2, harmonic angles 1/2 k (theta - theta0)^2,
 * periodic torsions k (1 + cos(n phi - phi0)).  Packed arrays:
 *   bonds   [nb]: idx (i,j)      par (k, r0)
 *   angles  [na]: idx (i,j,k)    par (k, theta0)     j is the vertex
 *   torsions[nt]: idx (i,j,k,l)  par (k, n, phi0)
 * These are the intramolecular U_solv / U_solu terms of Eq. 4 (unchanged
 * along lambda).  Returns the bonded energy; F (may be NULL) gets -grad. */
static double dihedral(const double* a, const double* b, const double* c, const double* d,
                       const double box[3], double g[4][3])
{
    double b1[3], b2[3], b3[3];
    for (int k = 0; k < 3; ++k) { b1[k] = b[k] - a[k]; b2[k] = c[k] - b[k]; b3[k] = d[k] - c[k]; }
    min_image(b1, box); min_image(b2, box); min_image(b3, box);
    double n1[3] = {b1[1] * b2[2] - b1[2] * b2[1], b1[2] * b2[0] - b1[0] * b2[2], b1[0] * b2[1] - b1[1] * b2[0]};
    double n2[3] = {b2[1] * b3[2] - b2[2] * b3[1], b2[2] * b3[0] - b2[0] * b3[2], b2[0] * b3[1] - b2[1] * b3[0]};
    double lb2 = sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]);
    double m1[3] = {n1[1] * b2[2] - n1[2] * b2[1], n1[2] * b2[0] - n1[0] * b2[2], n1[0] * b2[1] - n1[1] * b2[0]};
    double x = n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2];
    double y = (m1[0] * n2[0] + m1[1] * n2[1] + m1[2] * n2[2]) / lb2;
    double phi = atan2(-y, x);
    /* gradient of phi (Blondel & Karplus 1996 form) */
    double n1sq = n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2];
    double n2sq = n2[0] * n2[0] + n2[1] * n2[1] + n2[2] * n2[2];
    double b1b2 = b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2];
    double b3b2 = b3[0] * b2[0] + b3[1] * b2[1] + b3[2] * b2[2];
    for (int k = 0; k < 3; ++k) {
        double ga = -lb2 / n1sq * n1[k];
        double gd = lb2 / n2sq * n2[k];
        g[0][k] = ga;
        g[3][k] = gd;
        g[1][k] = -ga - (b1b2 / (lb2 * lb2)) * ga + (b3b2 / (lb2 * lb2)) * gd;
        g[2][k] = -gd + (b1b2 / (lb2 * lb2)) * ga - (b3b2 / (lb2 * lb2)) * gd;
    }
    return phi;
}

double orc_dihedral(const double* a, const double* b, const double* c, const double* d, const double* box)
{
    double g[4][3];
    return dihedral(a, b, c, d, box, g);
}

/* The dihedral and its gradient with respect to the four positions
 * (grad[3 j + k]: atom j, component k), as used by the torsion forces. */
double orc_dihedral_grad(const double* a, const double* b, const double* c, const double* d, const double* box,
                         double* grad)
{
    double g[4][3];
    const double phi = dihedral(a, b, c, d, box, g);
    for (int j = 0; j < 4; ++j)
        for (int k = 0; k < 3; ++k) grad[3 * j + k] = g[j][k];
    return phi;
}

double orc_bonded(const double* box, int n, const double* pos,
                  int nb, const int* bi, const double* bp,
                  int na, const int* ai, const double* ap,
                  int nt, const int* ti, const double* tp, double* F)
{
    double U = 0.0;
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)n);
    for (int e = 0; e < nb; ++e) {
        int i = bi[2 * e], j = bi[2 * e + 1];
        double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1], pos[3 * j + 2] - pos[3 * i + 2]};
        min_image(d, box);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dr = r - bp[2 * e + 1];
        U += 0.5 * bp[2 * e] * dr * dr;
        if (F) add_pair_force(F, i, j, bp[2 * e] * dr / r, d);
    }
    for (int e = 0; e < na; ++e) {
        int i = ai[3 * e], j = ai[3 * e + 1], k = ai[3 * e + 2];
        double u[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1], pos[3 * i + 2] - pos[3 * j + 2]};
        double v[3] = {pos[3 * k] - pos[3 * j], pos[3 * k + 1] - pos[3 * j + 1], pos[3 * k + 2] - pos[3 * j + 2]};
        min_image(u, box); min_image(v, box);
        double lu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double lv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double c = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) / (lu * lv);
        if (c > 1.0) c = 1.0;
        if (c < -1.0) c = -1.0;
        double th = acos(c);
        double dth = th - ap[2 * e + 1];
        U += 0.5 * ap[2 * e] * dth * dth;
        if (F) {
            double sn = sqrt(1.0 - c * c);
            if (sn < 1e-12) sn = 1e-12;
            double dU = ap[2 * e] * dth;        /* dU/dtheta */
            double pre = dU / sn;               /* dtheta/dcos = -1/sin */
            for (int t = 0; t < 3; ++t) {
                double dci = (v[t] / (lu * lv) - c * u[t] / (lu * lu));
                double dck = (u[t] / (lu * lv) - c * v[t] / (lv * lv));
                /* F = -dU/dx = -dU/dth * dth/dc * dc/dx = pre * dc/dx */
                F[3 * i + t] += pre * dci;
                F[3 * k + t] += pre * dck;
                F[3 * j + t] -= pre * (dci + dck);
            }
        }
    }
    for (int e = 0; e < nt; ++e) {
        int idx[4] = {ti[4 * e], ti[4 * e + 1], ti[4 * e + 2], ti[4 * e + 3]};
        double g[4][3];
        double phi = dihedral(pos + 3 * idx[0], pos + 3 * idx[1], pos + 3 * idx[2], pos + 3 * idx[3], box, g);
        double k = tp[3 * e], mult = tp[3 * e + 1], ph0 = tp[3 * e + 2];
        U += k * (1.0 + cos(mult * phi - ph0));
        if (F) {
            double dU = -k * mult * sin(mult * phi - ph0);
            for (int a = 0; a < 4; ++a)
                for (int t = 0; t < 3; ++t) F[3 * idx[a] + t] -= dU * g[a][t];
        }
    }
    return U;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}


/* ------------------------------------------------- parameter gradients
 *
 * Derivatives of the class energies with respect to each atom's charge,
 * sigma and epsilon (the differentiation configuration: gradients of U and
 * dU/dlambda with respect to solute parameters).  Output G[9 n]:
 *   G[9 i + 3 p + c],  p = 0 charge, 1 sigma, 2 epsilon,
 *                      c = 0 the atom's own class (U_vv for a solvent atom,
 *                            U_uu for a solute atom), 1 U_uv, 2 U_soft.
 * Then dU/dp_i = G_own + h_A G_uv + h_B G_soft and
 * d2U/dlambda dp_i = h_A' G_uv + h_B' G_soft (Eq. 4 is linear in the bases).
 * Coulomb: d/dq_i of k_e q_i q_j f(r) is k_e q_j f(r) for every pair term
 * (erfc real space, -erf exclusion correction, scaled 1-4), -2 k_e alpha/sqrt(pi) q_i
 * for the self term, the derivative of the background, and the reciprocal
 * potential of each class at r_i (level 1: k-sum; level 2: SPME grid
 * interpolation).  LJ: sigma_ij = (sigma_i + sigma_j)/2 and eps_ij = sqrt(eps_i
 * eps_j), so d sigma_ij / d sigma_i = 1/2 and dE/d eps_i = E / (2 eps_i)
 * (eps_i > 0; 0 otherwise).  Returns 0 on success. */
int orc_param_grad(const orc_params* p, int n, const double* pos, const double* q,
                   const double* sig, const double* eps, const unsigned char* solute,
                   int n_excl, const int* excl, int n14, const int* p14, const double* s14,
                   double* G)
{
    if (n <= 0 || !G) return -1;
    memset(G, 0, sizeof(double) * 9 * (size_t)n);
    const double rc = p->r_cut, rs = p->r_switch, a = p->alpha, rc2 = rc * rc;
    const double V = p->box[0] * p->box[1] * p->box[2];
    int *st, *li;
    build_exclusion_csr(n, n_excl, excl, &st, &li);
    /* real-space pairs: loop over i, derivatives with respect to atom i's parameters */
#pragma omp parallel
    {
        char* mark = (char*)calloc((size_t)n, 1);
#pragma omp for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            for (int e = st[i]; e < st[i + 1]; ++e) mark[li[e]] = 1;
            double* g = G + 9 * (size_t)i;
            for (int j = 0; j < n; ++j) {
                if (j == i || mark[j]) continue;
                double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1],
                               pos[3 * j + 2] - pos[3 * i + 2]};
                min_image(d, p->box);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 >= rc2) continue;
                double r = sqrt(r2);
                int c = pair_class(solute[i], solute[j]) == 2 ? 1 : 0;
                g[0 + c] += ORC_KE * q[j] * erfc(a * r) / r;
                double sg = 0.5 * (sig[i] + sig[j]), ep = sqrt(eps[i] * eps[j]);
                if (ep > 0.0) {
                    double dS, S = orc_switch(r, rc, rs, &dS);
                    double s6 = pow(sg / r, 6);
                    double elj = 4.0 * ep * (s6 * s6 - s6) * S;
                    g[3 + c] += 12.0 * ep / sg * (2.0 * s6 * s6 - s6) * S;
                    if (eps[i] > 0.0) g[6 + c] += elj / (2.0 * eps[i]);
                    if (c == 1 && sg > 0.0) {
                        double du, u = orc_ucap(r / sg, &du);
                        double es = ep * u * S;
                        g[3 + 2] += -ep * du * (r / sg) / (2.0 * sg) * S;
                        if (eps[i] > 0.0) g[6 + 2] += es / (2.0 * eps[i]);
                    }
                }
            }
            for (int e = st[i]; e < st[i + 1]; ++e) mark[li[e]] = 0;
        }
        free(mark);
    }
    free(st); free(li);
    /* exclusion corrections and 1-4 terms: both atoms of the pair */
    for (int e = 0; e < n_excl; ++e) {
        int i = excl[2 * e], j = excl[2 * e + 1];
        double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1], pos[3 * j + 2] - pos[3 * i + 2]};
        min_image(d, p->box);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double f = r < 1e-12 ? 2.0 * a / sqrt(ORC_PI) : erf(a * r) / r;
        int c = pair_class(solute[i], solute[j]) == 2 ? 1 : 0;
        G[9 * (size_t)i + c] += -ORC_KE * q[j] * f;
        G[9 * (size_t)j + c] += -ORC_KE * q[i] * f;
    }
    for (int e = 0; e < n14; ++e) {
        int i = p14[2 * e], j = p14[2 * e + 1];
        double sLJ = s14[2 * e], sC = s14[2 * e + 1];
        double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1], pos[3 * j + 2] - pos[3 * i + 2]};
        min_image(d, p->box);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        int c = pair_class(solute[i], solute[j]) == 2 ? 1 : 0;
        G[9 * (size_t)i + c] += sC * ORC_KE * q[j] / r;
        G[9 * (size_t)j + c] += sC * ORC_KE * q[i] / r;
        double sg = 0.5 * (sig[i] + sig[j]), ep = sqrt(eps[i] * eps[j]);
        if (ep > 0.0) {
            double s6 = pow(sg / r, 6);
            double elj = 4.0 * ep * (s6 * s6 - s6);
            double ds = sLJ * 12.0 * ep / sg * (2.0 * s6 * s6 - s6);
            G[9 * (size_t)i + 3 + c] += ds;
            G[9 * (size_t)j + 3 + c] += ds;
            if (eps[i] > 0.0) G[9 * (size_t)i + 6 + c] += sLJ * elj / (2.0 * eps[i]);
            if (eps[j] > 0.0) G[9 * (size_t)j + 6 + c] += sLJ * elj / (2.0 * eps[j]);
        }
    }
    if (p->level != 0) {
        /* self and background */
        double Q[2] = {0, 0};
        for (int i = 0; i < n; ++i) Q[solute[i] ? 1 : 0] += q[i];
        double pre = -ORC_KE * ORC_PI / (2.0 * V * a * a);
        double* phi2 = (double*)malloc(sizeof(double) * 2 * (size_t)n);
        double E[ORC_NE];
        memset(E, 0, sizeof(E));
        if (p->level == 1) ewald_ksum(p, n, pos, q, solute, E, NULL, NULL, phi2);
        else spme(p, n, pos, q, solute, E, NULL, NULL, phi2);
        for (int i = 0; i < n; ++i) {
            int u = solute[i] ? 1 : 0;
            double* g = G + 9 * (size_t)i;
            g[0] += -2.0 * ORC_KE * a / sqrt(ORC_PI) * q[i] + 2.0 * pre * Q[u];
            g[1] += 2.0 * pre * Q[1 - u];
            g[0] += phi2[2 * i + u];        /* own class potential */
            g[1] += phi2[2 * i + 1 - u];    /* other class potential: the uv cross term */
        }
        free(phi2);
    }
    return 0;
}
