/*
 * pf_oracle.c -- FP64 single-threaded oracle of the phase-field energy F_eps
 * (Song, arXiv 2103.04856, eq. Feps) and of its exact discrete gradient.
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA path is checked against.
 * Deliberately plain: every voxel is evaluated by itself, in the order the
 * paper builds the quantities (Sec. 2.3 eq. Meps -> Sec. 3.1 eqs. Beps..kepsb
 * -> Sec. 3.2 eq. Feps), and the gradient is formed in two explicit passes
 * (local reverse mode per voxel, then the transposed finite-difference
 * stencils).  No tiling, no fusion, no reordering.
 *
 * Readings taken where the paper is silent (each one is a test pin or is
 * listed as a reading in the design notes):
 *  - finite differences (Sec. 4.1 says only "classical, periodic"): central
 *    first derivatives, 3-point second derivatives, 4-point mixed derivatives;
 *    the integral is h^3 times the sum over voxels;
 *  - n_u (x) n_u is (grad u)(grad u)^T / (|grad u|^2 + xi^2): the xi offset of
 *    Sec. 4.1 applied to the normal as well;
 *  - x^+ is replaced by xi*log(1+exp(x/xi)) (Sec. 4.1), evaluated in the
 *    overflow-free form max(x,0) + xi*log1p(exp(-|x|/xi));
 *  - the derivative of sqrt(P) is taken as 0 where P underflows to exactly 0
 *    (its limit there);
 *  - the a00 term uses the plain |grad u|^2, the a10/a01 terms the regularised
 *    norm sqrt(|grad u|^2 + xi^2).
 */
#include "pf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- helpers */

typedef struct { double s, c; } nsum;   /* Neumaier compensated sum */

static void nsum_add(nsum* a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else                       a->c += (v - t) + a->s;
    a->s = t;
}
static double nsum_get(const nsum* a) { return a->s + a->c; }

static int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

static long vid(const pfo_problem* p, int x, int y, int z)
{
    x = wrap(x, p->nx); y = wrap(y, p->ny); z = wrap(z, p->nz);
    return ((long)z * p->ny + y) * p->nx + x;
}

static int check(const pfo_problem* p)
{
    if (!p) return -1;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
    if (!(p->h > 0) || !(p->eps > 0) || !(p->xi > 0)) return -1;
    if (p->well != 0 && p->well != 1) return -1;
    return 0;
}

/* Double well and its first two derivatives (Sec. 2.3, "Notations"):
 * well 1 is the paper's W(s) = (1-s^2)^2/4; well 0 is W(u) = u^2 (1-u)^2,
 * the same shape moved to the wells 0 and 1. */
static double Wp(int well, double u)
{
    if (well == 1) return u * u * u - u;
    return 2.0 * u * (1.0 - u) * (1.0 - 2.0 * u);
}
static double Wpp(int well, double u)
{
    if (well == 1) return 3.0 * u * u - 1.0;
    return 2.0 * (1.0 - 6.0 * u + 6.0 * u * u);
}

/* smooth positive part of Sec. 4.1 and its derivative (the logistic) */
static double softplus_xi(double x, double xi)
{
    double m = x > 0.0 ? x : 0.0;
    return m + xi * log1p(exp(-fabs(x) / xi));
}
static double softplus_xi_prime(double x, double xi)
{
    if (x >= 0.0) return 1.0 / (1.0 + exp(-x / xi));
    double t = exp(x / xi);
    return t / (1.0 + t);
}

/* coefficients of eq. Feps */
typedef struct { double c1, c2, c3, c4, c5, c6; } coefs;

/* Per-voxel state of the forward evaluation. */
typedef struct {
    coefs cf;        /* eq. Feps coefficients at this voxel (a, or a(x)) */
    double u;        /* centre value                                   */
    double G[3];     /* grad u                                          */
    double Hs[3][3]; /* Hess u (symmetric, all nine entries stored)     */
    double rho, q;   /* |grad u|^2 + xi^2 and its square root          */
    double w;        /* W'(u)/eps                                       */
    double M[3][3];  /* eq. Meps with the regularised normal            */
    double T, S, D;  /* Tr M, ||M||^2, 2||M||^2 - (Tr M)^2             */
    double P, r;     /* smooth positive part of D and its square root   */
    double tg;       /* theta . grad u (orientation term, Sec. 5.2)     */
    double e;        /* integrand of eq. Feps (plus the orientation term) */
} voxel;

static coefs make_coefs(const pfo_problem* p, const double* a)   /* a20 a11 a02 a10 a01 a00 */
{
    coefs c;
    c.c1 = (a[0] + a[2] - a[1]) / (2.0 * p->eps);
    c.c2 = a[1] / (2.0 * p->eps);
    c.c3 = (a[0] - a[2]) / (2.0 * p->eps);
    c.c4 = (a[3] + a[4]) / 2.0;
    c.c5 = (a[3] - a[4]) / 2.0;
    c.c6 = a[5] * p->eps;
    return c;
}

/* The coefficients at voxel i: the constant a, or a(x) of Sec. 5.2. */
static coefs coefs_at(const pfo_problem* p, long i)
{
    if (!p->a_field) return make_coefs(p, p->a);
    const long N = (long)p->nx * p->ny * p->nz;
    double a[6];
    for (int k = 0; k < 6; ++k) a[k] = p->a_field[k * N + i];
    return make_coefs(p, a);
}

/* Finite differences of Sec. 4.1 (reading: second-order central stencils). */
static void stencils(const pfo_problem* p, const double* u, int x, int y, int z, voxel* v)
{
    const double h = p->h;
    const int e[3][3] = { { 1, 0, 0 }, { 0, 1, 0 }, { 0, 0, 1 } };
    v->u = u[vid(p, x, y, z)];
    for (int c = 0; c < 3; ++c) {
        double up = u[vid(p, x + e[c][0], y + e[c][1], z + e[c][2])];
        double um = u[vid(p, x - e[c][0], y - e[c][1], z - e[c][2])];
        v->G[c] = (up - um) / (2.0 * h);
        v->Hs[c][c] = (up - 2.0 * v->u + um) / (h * h);
    }
    for (int c = 0; c < 3; ++c)
        for (int d = c + 1; d < 3; ++d) {
            int sx = e[c][0], sy = e[c][1], sz = e[c][2];
            int tx = e[d][0], ty = e[d][1], tz = e[d][2];
            double upp = u[vid(p, x + sx + tx, y + sy + ty, z + sz + tz)];
            double upm = u[vid(p, x + sx - tx, y + sy - ty, z + sz - tz)];
            double ump = u[vid(p, x - sx + tx, y - sy + ty, z - sz + tz)];
            double umm = u[vid(p, x - sx - tx, y - sy - ty, z - sz - tz)];
            double hcd = (upp - upm - ump + umm) / (4.0 * h * h);
            v->Hs[c][d] = hcd;
            v->Hs[d][c] = hcd;
        }
}

/* Forward evaluation of one voxel: eq. Meps, the invariants of Sec. 3.1 and
 * the integrand of eq. Feps. */
static void forward(const pfo_problem* p, const double* u, int x, int y, int z, voxel* v)
{
    stencils(p, u, x, y, z, v);
    v->cf = coefs_at(p, vid(p, x, y, z));
    const coefs* cf = &v->cf;
    double g2 = v->G[0] * v->G[0] + v->G[1] * v->G[1] + v->G[2] * v->G[2];
    v->rho = g2 + p->xi * p->xi;
    v->q = sqrt(v->rho);
    v->w = Wp(p->well, v->u) / p->eps;
    if (p->proj) {
        /* M = -eps P Hess u P, P = I - n (x) n with n (x) n = G G^T / rho */
        double P[3][3], PH[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) P[a][b] = (a == b ? 1.0 : 0.0) - v->G[a] * v->G[b] / v->rho;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                PH[a][b] = 0.0;
                for (int c = 0; c < 3; ++c) PH[a][b] += P[a][c] * v->Hs[c][b];
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int c = 0; c < 3; ++c) s += PH[a][c] * P[c][b];
                v->M[a][b] = -p->eps * s;
            }
    } else {
        /* M = -eps Hess u + (W'(u)/eps) n (x) n, with n (x) n = G G^T / rho */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                v->M[a][b] = -p->eps * v->Hs[a][b] + v->w * v->G[a] * v->G[b] / v->rho;
    }
    v->T = v->M[0][0] + v->M[1][1] + v->M[2][2];
    v->S = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) v->S += v->M[a][b] * v->M[a][b];
    v->D = 2.0 * v->S - v->T * v->T;
    v->P = softplus_xi(v->D, p->xi);
    v->r = sqrt(v->P);
    v->e = cf->c1 * v->S + cf->c2 * v->T * v->T + cf->c3 * v->T * v->r
         + cf->c4 * v->q * v->T + cf->c5 * v->q * v->r + cf->c6 * g2;
    /* Sec. 5.2: the orientation term eps mu (theta . grad u)^2 */
    v->tg = p->theta[0] * v->G[0] + p->theta[1] * v->G[1] + p->theta[2] * v->G[2];
    v->e += p->eps * p->mu * v->tg * v->tg;
}

/* Cotangents of one voxel's integrand with respect to its stencil outputs:
 *   ubar = de/du (through W'), Gbar[c] = de/dG_c, Hbar[c][d] = de/dHs_cd
 * (Hbar holds the derivative with respect to each of the nine entries; the
 * stencil transpose below visits each unordered pair once and adds both).
 * Chain: e(S, T, r(D(S,T)), q(G), |G|^2), M(Hs, w(u), G). */
static void local_adjoint(const pfo_problem* p, const voxel* v, double* ubar, double Gbar[3], double Hbar[3][3])
{
    const coefs* cf = &v->cf;
    double rp = 0.0;     /* dr/dD, defined as 0 where r == 0 */
    if (v->r > 0.0) rp = softplus_xi_prime(v->D, p->xi) / (2.0 * v->r);
    double k = (cf->c3 * v->T + cf->c5 * v->q) * rp;   /* de/dD */
    double dS = cf->c1 + 2.0 * k;
    double dT = 2.0 * cf->c2 * v->T + cf->c3 * v->r + cf->c4 * v->q - 2.0 * v->T * k;
    double dq = cf->c4 * v->T + cf->c5 * v->r;

    double L[3][3];      /* de/dM_ab */
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) L[a][b] = 2.0 * dS * v->M[a][b] + (a == b ? dT : 0.0);

    if (p->proj) {
        /* M = P K P with K = -eps Hess u and P = I - G G^T / rho:
         *   dE/dK = P L P;  dE/dP = L P K + K P L =: B;
         *   dP = -(dG G^T + G dG^T)/rho + 2 (G.dG) G G^T / rho^2  gives
         *   dE/dG (through P) = -2 B G / rho + 2 (G^T B G) G / rho^2. */
        double P[3][3], K[3][3], PL[3][3], LP[3][3], B[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                P[a][b] = (a == b ? 1.0 : 0.0) - v->G[a] * v->G[b] / v->rho;
                K[a][b] = -p->eps * v->Hs[a][b];
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                PL[a][b] = 0.0;
                LP[a][b] = 0.0;
                for (int c = 0; c < 3; ++c) {
                    PL[a][b] += P[a][c] * L[c][b];
                    LP[a][b] += L[a][c] * P[c][b];
                }
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0, t = 0.0, q = 0.0;
                for (int c = 0; c < 3; ++c) {
                    s += PL[a][c] * P[c][b];                /* (P L P)_ab     */
                    t += LP[a][c] * K[c][b];                /* (L P K)_ab     */
                    q += K[a][c] * PL[c][b];                /* (K P L)_ab     */
                }
                Hbar[a][b] = -p->eps * s;
                B[a][b] = t + q;
            }
        double BG[3], GBG = 0.0;
        for (int a = 0; a < 3; ++a) {
            BG[a] = 0.0;
            for (int b = 0; b < 3; ++b) BG[a] += B[a][b] * v->G[b];
            GBG += v->G[a] * BG[a];
        }
        *ubar = 0.0;     /* M no longer depends on u itself */
        for (int a = 0; a < 3; ++a)
            Gbar[a] = -2.0 * BG[a] / v->rho + 2.0 * GBG * v->G[a] / (v->rho * v->rho)
                    + dq * v->G[a] / v->q + 2.0 * cf->c6 * v->G[a]
                    + 2.0 * p->eps * p->mu * v->tg * p->theta[a];
        return;
    }

    double LG[3], GLG = 0.0;
    for (int a = 0; a < 3; ++a) {
        LG[a] = 0.0;
        for (int b = 0; b < 3; ++b) LG[a] += L[a][b] * v->G[b];
        GLG += v->G[a] * LG[a];
    }
    /* M depends on u through w = W'(u)/eps */
    *ubar = Wpp(p->well, v->u) / p->eps * GLG / v->rho;
    /* M depends on G through w G G^T / rho; q and |G|^2 depend on G too */
    for (int a = 0; a < 3; ++a)
        Gbar[a] = 2.0 * v->w / v->rho * (LG[a] - GLG / v->rho * v->G[a])
                + dq * v->G[a] / v->q + 2.0 * cf->c6 * v->G[a]
                + 2.0 * p->eps * p->mu * v->tg * p->theta[a];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Hbar[a][b] = -p->eps * L[a][b];
}

/* ------------------------------------------------------------- public API */

int pfo_density(const pfo_problem* p, const double* u, double* e)
{
    if (check(p) || !u || !e) return -1;
    voxel v;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                forward(p, u, x, y, z, &v);
                e[vid(p, x, y, z)] = v.e;
            }
    return 0;
}

int pfo_energy(const pfo_problem* p, const double* u, double* E)
{
    if (check(p) || !u || !E) return -1;
    nsum acc = { 0.0, 0.0 };
    voxel v;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                forward(p, u, x, y, z, &v);
                nsum_add(&acc, v.e);
            }
    *E = p->h * p->h * p->h * nsum_get(&acc);
    return 0;
}

/* cotangent fields, one record per voxel: ubar, Gbar[3], Hbar (xx yy zz xy xz yz) */
enum { CT_U = 0, CT_GX, CT_GY, CT_GZ, CT_HXX, CT_HYY, CT_HZZ, CT_HXY, CT_HXZ, CT_HYZ, CT_N };

static void cotangent_record(const pfo_problem* p, const voxel* v, double* rec)
{
    double ub, Gb[3], Hb[3][3];
    local_adjoint(p, v, &ub, Gb, Hb);
    rec[CT_U] = ub;
    rec[CT_GX] = Gb[0]; rec[CT_GY] = Gb[1]; rec[CT_GZ] = Gb[2];
    rec[CT_HXX] = Hb[0][0]; rec[CT_HYY] = Hb[1][1]; rec[CT_HZZ] = Hb[2][2];
    /* a mixed stencil value feeds both M_cd and M_dc */
    rec[CT_HXY] = Hb[0][1] + Hb[1][0];
    rec[CT_HXZ] = Hb[0][2] + Hb[2][0];
    rec[CT_HYZ] = Hb[1][2] + Hb[2][1];
}

/* Transposed stencils: dE/du_j = h^3 * sum over the voxels i whose stencils
 * read u_j of (cotangent_i * stencil weight of u_j in voxel i). */
static double gather(const pfo_problem* p, const double* ct, int x, int y, int z)
{
    const double h = p->h;
    const int e[3][3] = { { 1, 0, 0 }, { 0, 1, 0 }, { 0, 0, 1 } };
    const int gidx[3] = { CT_GX, CT_GY, CT_GZ };
    const int hdiag[3] = { CT_HXX, CT_HYY, CT_HZZ };
    double s = ct[vid(p, x, y, z) * CT_N + CT_U];
    for (int c = 0; c < 3; ++c) {
        long ip = vid(p, x + e[c][0], y + e[c][1], z + e[c][2]);
        long im = vid(p, x - e[c][0], y - e[c][1], z - e[c][2]);
        long i0 = vid(p, x, y, z);
        /* G_c(i) = (u(i+e_c) - u(i-e_c)) / 2h */
        s += (ct[im * CT_N + gidx[c]] - ct[ip * CT_N + gidx[c]]) / (2.0 * h);
        /* Hs_cc(i) = (u(i+e_c) - 2 u(i) + u(i-e_c)) / h^2 */
        s += (ct[im * CT_N + hdiag[c]] - 2.0 * ct[i0 * CT_N + hdiag[c]]
              + ct[ip * CT_N + hdiag[c]]) / (h * h);
    }
    const int pairs[3][3] = { { 0, 1, CT_HXY }, { 0, 2, CT_HXZ }, { 1, 2, CT_HYZ } };
    for (int k = 0; k < 3; ++k) {
        int c = pairs[k][0], d = pairs[k][1], f = pairs[k][2];
        int sx = e[c][0] + e[d][0], sy = e[c][1] + e[d][1], sz = e[c][2] + e[d][2];
        int tx = e[c][0] - e[d][0], ty = e[c][1] - e[d][1], tz = e[c][2] - e[d][2];
        /* Hs_cd(i) = (u(i+c+d) - u(i+c-d) - u(i-c+d) + u(i-c-d)) / 4h^2 */
        double vmm = ct[vid(p, x - sx, y - sy, z - sz) * CT_N + f];  /* i = j-c-d */
        double vmp = ct[vid(p, x - tx, y - ty, z - tz) * CT_N + f];  /* i = j-c+d */
        double vpm = ct[vid(p, x + tx, y + ty, z + tz) * CT_N + f];  /* i = j+c-d */
        double vpp = ct[vid(p, x + sx, y + sy, z + sz) * CT_N + f];  /* i = j+c+d */
        s += (vmm - vmp - vpm + vpp) / (4.0 * h * h);
    }
    return h * h * h * s;
}

int pfo_energy_and_grad(const pfo_problem* p, const double* u, double* E, double* g)
{
    if (check(p) || !u || !g) return -1;
    long N = (long)p->nx * p->ny * p->nz;
    double* ct = (double*)malloc(sizeof(double) * CT_N * (size_t)N);
    if (!ct) return -1;
    nsum acc = { 0.0, 0.0 };
    voxel v;
    /* pass 1: forward and local reverse mode, voxel by voxel */
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                forward(p, u, x, y, z, &v);
                nsum_add(&acc, v.e);
                cotangent_record(p, &v, ct + vid(p, x, y, z) * CT_N);
            }
    /* pass 2: transposed stencils */
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) g[vid(p, x, y, z)] = gather(p, ct, x, y, z);
    free(ct);
    if (E) *E = p->h * p->h * p->h * nsum_get(&acc);
    return 0;
}

int pfo_grad_sampled(const pfo_problem* p, const double* u, int n, const long* idx, double* g)
{
    if (check(p) || !u || (n > 0 && (!idx || !g))) return -1;
    long N = (long)p->nx * p->ny * p->nz;
    /* the gradient at j reads cotangents at offsets in {-1,0,1}^3 only;
     * compute those 27 records into a small local block */
    double* ct = (double*)malloc(sizeof(double) * CT_N * 27);
    if (!ct) return -1;
    voxel v;
    for (int k = 0; k < n; ++k) {
        if (idx[k] < 0 || idx[k] >= N) { free(ct); return -1; }
        int x = (int)(idx[k] % p->nx);
        int y = (int)((idx[k] / p->nx) % p->ny);
        int z = (int)(idx[k] / ((long)p->nx * p->ny));
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    forward(p, u, x + dx, y + dy, z + dz, &v);
                    int l = ((dz + 1) * 3 + (dy + 1)) * 3 + (dx + 1);
                    cotangent_record(p, &v, ct + l * CT_N);
                }
        /* gather on the 3x3x3 block around its centre: every offset it
         * visits lies inside the block, so its wrap never triggers */
        pfo_problem lp = *p;
        lp.nx = 3; lp.ny = 3; lp.nz = 3;
        g[k] = gather(&lp, ct, 1, 1, 1);
    }
    free(ct);
    return 0;
}

int pfo_step(const pfo_problem* p, const double* u_in, double* u_out, double tau, double* sc)
{
    if (check(p) || !u_in || !u_out) return -1;
    long N = (long)p->nx * p->ny * p->nz;
    double* g = (double*)malloc(sizeof(double) * (size_t)N);
    if (!g) return -1;
    double E = 0.0;
    if (pfo_energy_and_grad(p, u_in, &E, g)) { free(g); return -1; }
    nsum sg = { 0, 0 }, sag = { 0, 0 }, su = { 0, 0 };
    double gmax = 0.0;
    for (long i = 0; i < N; ++i) {
        nsum_add(&sg, g[i]);
        nsum_add(&sag, fabs(g[i]));
        nsum_add(&su, u_in[i]);
        if (fabs(g[i]) > gmax) gmax = fabs(g[i]);
    }
    /* volume constraint: remove the mean of the gradient (Lagrange multiplier) */
    double lambda = nsum_get(&sg) / (double)N;
    for (long i = 0; i < N; ++i) u_out[i] = u_in[i] - tau * (g[i] - lambda);
    if (sc) {
        sc[0] = E;
        sc[1] = nsum_get(&su) / (double)N;
        sc[2] = lambda;
        sc[3] = gmax;
        sc[4] = nsum_get(&sag) / (double)N;
    }
    free(g);
    return 0;
}

int pfo_run(const pfo_problem* p, double* u, int nsteps, double tau, double* trace)
{
    if (check(p) || !u || nsteps < 0) return -1;
    long N = (long)p->nx * p->ny * p->nz;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)N);
    if (!tmp) return -1;
    for (int s = 0; s < nsteps; ++s) {
        if (pfo_step(p, u, tmp, tau, trace ? trace + 5 * (long)s : NULL)) { free(tmp); return -1; }
        memcpy(u, tmp, sizeof(double) * (size_t)N);
    }
    free(tmp);
    return 0;
}

int pfo_curvatures(const pfo_problem* p, const double* u, double* k1, double* k2)
{
    if (check(p) || !u || !k1 || !k2) return -1;
    voxel v;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                forward(p, u, x, y, z, &v);
                double root = sqrt(v.D > 0.0 ? v.D : 0.0);
                double den = 2.0 * p->eps * v.q;
                k1[vid(p, x, y, z)] = (v.T + root) / den;
                k2[vid(p, x, y, z)] = (v.T - root) / den;
            }
    return 0;
}

/* ------------------------------------------ curvature diagram (Sec. 4.1) */

/* Corner c = (i, j, k) of a cube is bit i + 2j + 4k.  The six tetrahedra of
 * the Freudenthal split run from corner 0 to corner 7 along the three axes
 * taken in each of the six orders. */
static const int tet_axes[6][3] = { { 0, 1, 2 }, { 0, 2, 1 }, { 1, 0, 2 }, { 1, 2, 0 }, { 2, 0, 1 }, { 2, 1, 0 } };

static void corner_pos(int c, double q[3])
{
    q[0] = (double)(c & 1);
    q[1] = (double)((c >> 1) & 1);
    q[2] = (double)((c >> 2) & 1);
}

/* the point where u - level changes sign on the edge from corner a (above
 * the level) to corner b (not above), by linear interpolation */
static void edge_point(const double f[8], int a, int b, double q[3])
{
    double qa[3], qb[3];
    corner_pos(a, qa);
    corner_pos(b, qb);
    const double t = f[a] / (f[a] - f[b]);
    for (int k = 0; k < 3; ++k) q[k] = qa[k] + t * (qb[k] - qa[k]);
}

static void emit_triangle(const pfo_problem* p, const double P0[3], const double P1[3], const double P2[3],
                          const double k1c[8], const double k2c[8], long* n, long cap, double* cells)
{
    double a[3], b[3], cr[3], bc[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = P1[k] - P0[k];
        b[k] = P2[k] - P0[k];
        bc[k] = (P0[k] + P1[k] + P2[k]) / 3.0;
    }
    cr[0] = a[1] * b[2] - a[2] * b[1];
    cr[1] = a[2] * b[0] - a[0] * b[2];
    cr[2] = a[0] * b[1] - a[1] * b[0];
    const double area = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) * p->h * p->h;
    /* trilinear interpolation of the corner curvatures at the barycenter */
    double s1 = 0.0, s2 = 0.0;
    for (int c = 0; c < 8; ++c) {
        const double wx = (c & 1) ? bc[0] : 1.0 - bc[0];
        const double wy = ((c >> 1) & 1) ? bc[1] : 1.0 - bc[1];
        const double wz = ((c >> 2) & 1) ? bc[2] : 1.0 - bc[2];
        s1 += wx * wy * wz * k1c[c];
        s2 += wx * wy * wz * k2c[c];
    }
    if (*n < cap) {
        cells[3 * *n + 0] = area;
        cells[3 * *n + 1] = s1;
        cells[3 * *n + 2] = s2;
    }
    *n += 1;
}

int pfo_surface_cells(const pfo_problem* p, const double* u, double level, long cap, double* cells, long* count)
{
    if (check(p) || !u || !count || cap < 0 || (cap > 0 && !cells)) return -1;
    const long N = (long)p->nx * p->ny * p->nz;
    double* k1 = (double*)malloc(sizeof(double) * (size_t)N);
    double* k2 = (double*)malloc(sizeof(double) * (size_t)N);
    if (!k1 || !k2 || pfo_curvatures(p, u, k1, k2)) { free(k1); free(k2); return -1; }
    long n = 0;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double f[8], k1c[8], k2c[8];
                int above[8];
                for (int c = 0; c < 8; ++c) {
                    const long i = vid(p, x + (c & 1), y + ((c >> 1) & 1), z + ((c >> 2) & 1));
                    above[c] = u[i] > level;
                    f[c] = u[i] - level;
                    k1c[c] = k1[i];
                    k2c[c] = k2[i];
                }
                for (int t = 0; t < 6; ++t) {
                    int v[4];
                    v[0] = 0;
                    v[1] = 1 << tet_axes[t][0];
                    v[2] = v[1] | (1 << tet_axes[t][1]);
                    v[3] = 7;
                    int pos[4], neg[4], np = 0, nn = 0;
                    for (int k = 0; k < 4; ++k) {
                        if (above[v[k]]) pos[np++] = v[k];
                        else neg[nn++] = v[k];
                    }
                    double A[3], B[3], C[3], D[3];
                    if (np == 1) {          /* one corner above: a triangle around it */
                        edge_point(f, pos[0], neg[0], A);
                        edge_point(f, pos[0], neg[1], B);
                        edge_point(f, pos[0], neg[2], C);
                        emit_triangle(p, A, B, C, k1c, k2c, &n, cap, cells);
                    } else if (np == 3) {   /* one corner below: a triangle around it */
                        edge_point(f, pos[0], neg[0], A);
                        edge_point(f, pos[1], neg[0], B);
                        edge_point(f, pos[2], neg[0], C);
                        emit_triangle(p, A, B, C, k1c, k2c, &n, cap, cells);
                    } else if (np == 2) {   /* a quadrilateral, split along (p0 q0)-(p1 q1) */
                        edge_point(f, pos[0], neg[0], A);
                        edge_point(f, pos[0], neg[1], B);
                        edge_point(f, pos[1], neg[1], C);
                        edge_point(f, pos[1], neg[0], D);
                        emit_triangle(p, A, B, C, k1c, k2c, &n, cap, cells);
                        emit_triangle(p, A, C, D, k1c, k2c, &n, cap, cells);
                    }
                }
            }
    free(k1);
    free(k2);
    *count = n;
    return 0;
}

static double W(int well, double u)
{
    if (well == 1) return 0.25 * (1.0 - u * u) * (1.0 - u * u);
    return u * u * (1.0 - u) * (1.0 - u);
}

int pfo_diagnostics(const pfo_problem* p, const double* u, double out[5])
{
    if (check(p) || !u || !out) return -1;
    nsum dis = { 0, 0 }, ch = { 0, 0 };
    double umax = -HUGE_VAL, umin = HUGE_VAL;
    voxel v;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                stencils(p, u, x, y, z, &v);
                const double g2 = v.G[0] * v.G[0] + v.G[1] * v.G[1] + v.G[2] * v.G[2];
                const double kin = 0.5 * p->eps * g2, pot = W(p->well, v.u) / p->eps;
                nsum_add(&dis, fabs(kin - pot));
                nsum_add(&ch, kin + pot);
                if (v.u > umax) umax = v.u;
                if (v.u < umin) umin = v.u;
            }
    const double h3 = p->h * p->h * p->h;
    out[0] = h3 * nsum_get(&dis);
    out[1] = h3 * nsum_get(&ch);
    out[2] = out[1] > 0.0 ? out[0] / out[1] : 0.0;
    out[3] = umax;
    out[4] = umin;
    return 0;
}

void pfo_b_to_a(const double b[7], double a[6])
{
    /* h2 (H - H0)^2 + k1 K + alpha (k1 - k1_0)^2 + beta (k2 - k2_0)^2,
     * with H = kappa1 + kappa2 and K = kappa1 kappa2, expanded in monomials */
    double h2 = b[0], H0 = b[1], kK = b[2], al = b[3], k10 = b[4], be = b[5], k20 = b[6];
    a[0] = h2 + al;                                  /* kappa1^2        */
    a[1] = 2.0 * h2 + kK;                            /* kappa1 kappa2   */
    a[2] = h2 + be;                                  /* kappa2^2        */
    a[3] = -2.0 * h2 * H0 - 2.0 * al * k10;          /* kappa1          */
    a[4] = -2.0 * h2 * H0 - 2.0 * be * k20;          /* kappa2          */
    a[5] = h2 * H0 * H0 + al * k10 * k10 + be * k20 * k20;
}

/* ------------------------------------------------------ Alg. 1: H^-1 flow */

void pfo_gauss_weights(double sigma, int R, double* w)
{
    double s = 0.0;
    for (int j = -R; j <= R; ++j) {
        w[j + R] = exp(-(double)(j * j) / (2.0 * sigma * sigma));
        s += w[j + R];
    }
    for (int j = 0; j <= 2 * R; ++j) w[j] /= s;
}

/* periodic 1-D convolution along axis `ax` (0 x, 1 y, 2 z) with weights w[0..2R] */
static void convolve_axis(const pfo_problem* p, const double* in, double* out, int ax, const double* w, int R)
{
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double s = 0.0;
                for (int j = -R; j <= R; ++j) {
                    int xx = x + (ax == 0 ? j : 0), yy = y + (ax == 1 ? j : 0), zz = z + (ax == 2 ? j : 0);
                    s += w[j + R] * in[vid(p, xx, yy, zz)];
                }
                out[vid(p, x, y, z)] = s;
            }
}

/* k * a in place (separable Gaussian, x then y then z); no-op without blur */
static int blur(const pfo_problem* p, const pfo_hflow* f, double* a)
{
    if (!(f->blur_sigma > 0.0)) return 0;
    int R = f->blur_radius;
    long N = (long)p->nx * p->ny * p->nz;
    double* w = (double*)malloc(sizeof(double) * (2 * R + 1));
    double* t = (double*)malloc(sizeof(double) * (size_t)N);
    if (!w || !t) { free(w); free(t); return -1; }
    pfo_gauss_weights(f->blur_sigma, R, w);
    convolve_axis(p, a, t, 0, w, R);
    convolve_axis(p, t, a, 1, w, R);
    convolve_axis(p, a, t, 2, w, R);
    memcpy(a, t, sizeof(double) * (size_t)N);
    free(w);
    free(t);
    return 0;
}

static int check_flow(const pfo_hflow* f)
{
    if (!f) return -1;
    if (f->blur_sigma > 0.0 && f->blur_radius < 1) return -1;
    return 0;
}

int pfo_blur(const pfo_problem* p, const pfo_hflow* f, double* a)
{
    if (check(p) || check_flow(f) || !a) return -1;
    return blur(p, f, a);
}

int pfo_hflow_field(const pfo_problem* p, const pfo_hflow* f, const double* A, double* ut)
{
    if (check(p) || check_flow(f) || !A || !ut) return -1;
    long N = (long)p->nx * p->ny * p->nz;
    const int e[3][3] = { { 1, 0, 0 }, { 0, 1, 0 }, { 0, 0, 1 } };
    /* eq. change_var: u = div A + m0 with periodic central differences
     * (Sec. 5.2: + m(x) when the mass is spatialised) */
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double d = 0.0;
                for (int c = 0; c < 3; ++c)
                    d += (A[c * N + vid(p, x + e[c][0], y + e[c][1], z + e[c][2])]
                          - A[c * N + vid(p, x - e[c][0], y - e[c][1], z - e[c][2])]) / (2.0 * p->h);
                const long i = vid(p, x, y, z);
                ut[i] = d + (f->m_field ? f->m_field[i] : f->m0);
            }
    return blur(p, f, ut);   /* Alg. 1: small blur before the energy */
}

int pfo_hflow_grad(const pfo_problem* p, const pfo_hflow* f, const double* A, double* G, double* gA)
{
    if (check(p) || check_flow(f) || !A || !gA) return -1;
    long N = (long)p->nx * p->ny * p->nz;
    double* ut = (double*)malloc(sizeof(double) * (size_t)N);
    double* g = (double*)malloc(sizeof(double) * (size_t)N);
    if (!ut || !g) { free(ut); free(g); return -1; }
    double E = 0.0;
    if (pfo_hflow_field(p, f, A, ut) || pfo_energy_and_grad(p, ut, &E, g) || blur(p, f, g)) {
        free(ut); free(g); return -1;
    }
    /* the blur is symmetric and periodic, hence self-adjoint: g = k * dF/dut.
     * dG/dA_c(j) = sum_i g_i du_i/dA_c(j) = (g(j - e_c) - g(j + e_c)) / 2h */
    const int e[3][3] = { { 1, 0, 0 }, { 0, 1, 0 }, { 0, 0, 1 } };
    for (int c = 0; c < 3; ++c)
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x)
                    gA[c * N + vid(p, x, y, z)] = (g[vid(p, x - e[c][0], y - e[c][1], z - e[c][2])]
                                                   - g[vid(p, x + e[c][0], y + e[c][1], z + e[c][2])]) / (2.0 * p->h);
    if (G) *G = E;
    free(ut);
    free(g);
    return 0;
}

int pfo_hflow_run(const pfo_problem* p, const pfo_hflow* f, double* A, double* m, double* v, int nsteps, int* t,
                  double* trace)
{
    if (check(p) || check_flow(f) || !A || !m || !v || !t || nsteps < 0) return -1;
    long N = (long)p->nx * p->ny * p->nz;
    double* gA = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* ut = (double*)malloc(sizeof(double) * (size_t)N);
    if (!gA || !ut) { free(gA); free(ut); return -1; }
    for (int s = 0; s < nsteps; ++s) {
        double G = 0.0;
        if (pfo_hflow_grad(p, f, A, &G, gA) || pfo_hflow_field(p, f, A, ut)) { free(gA); free(ut); return -1; }
        *t += 1;
        /* Adam (Kingma and Ba): moment updates with bias correction */
        const double b1t = 1.0 - pow(f->beta1, *t), b2t = 1.0 - pow(f->beta2, *t);
        nsum sa = { 0, 0 }, su = { 0, 0 };
        double gmax = 0.0;
        for (long i = 0; i < 3 * N; ++i) {
            const double g = gA[i];
            if (fabs(g) > gmax) gmax = fabs(g);
            nsum_add(&sa, fabs(g));
            m[i] = f->beta1 * m[i] + (1.0 - f->beta1) * g;
            v[i] = f->beta2 * v[i] + (1.0 - f->beta2) * g * g;
            const double mh = m[i] / b1t, vh = v[i] / b2t;
            A[i] -= f->lr * mh / (sqrt(vh) + f->adam_eps);
        }
        for (long i = 0; i < N; ++i) nsum_add(&su, ut[i]);
        if (trace) {
            double* row = trace + 5 * (long)s;
            row[0] = G;
            row[1] = gmax;
            row[2] = nsum_get(&sa) / (3.0 * (double)N);
            row[3] = nsum_get(&su) / (double)N;
            row[4] = (double)*t;
        }
    }
    free(gA);
    free(ut);
    return 0;
}
