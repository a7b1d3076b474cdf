/*
 * hgks_oracle.c -- plain FP64 CPU restatement of the high-order gas-kinetic
 * scheme with hybrid WENO-AO reconstruction (Mu, Zhuo, Zhang, Liu, Zhong,
 * "An efficient high-order gas-kinetic scheme with hybrid WENO-AO method for
 * the Euler and Navier-Stokes solutions", arXiv 2304.05572).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code, header, table or constant with the CUDA library.
 *
 * It is written to be read against the paper, not to be fast:
 *   - velocity moments of the Maxwellian are taken from the Gaussian-integral
 *     recursions and combined through explicit polynomial products in
 *     (u, v, xi^2), so every moment in Eqs. (8)-(12) is integrated literally;
 *   - the micro-slope and compatibility systems of Eqs. (8)-(9) are solved as
 *     generic dense linear systems (Gaussian elimination, partial pivoting);
 *   - the time integrals of Eq. (10) are written out term by term.
 *
 * Compiled with -ffp-contract=off: a*b+c is a rounded multiply followed by a
 * rounded add unless fma() is written.  The troubled-cell indicator and the
 * normal-direction reconstruction follow one fixed evaluation order (spelled
 * out below) so that a second implementation taking the same decisions in the
 * same FP64 order reproduces the troubled flags bit for bit.
 *
 * Readings of points the paper leaves open are marked "Reading:".
 */
#include <math.h>
#include <stdio.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG 4        /* ghost layers: the widest indicator window (Step 4 spread of a 5-cell test) reaches 4 cells */
#define MAXT 256    /* terms of a polynomial in (u, v, xi^2); the largest product formed (heat
                       weight of 18 terms x slope polynomial of 12 terms) has 216 */
#define NMOM 10     /* highest velocity power needed is u^7 (flux of the slope term) */

enum { BC_PERIODIC = 0, BC_EXTRAP = 1, BC_REFLECT = 2, BC_SYMMETRY = 3, BC_NOSLIP = 4,
       BC_INFLOW = 5, BC_SHOCK_WALL = 6, BC_SHOCK_TRACK = 7 };
enum { RECON_HYBRID = 0, RECON_LINEAR = 1, RECON_WENOAO = 2 };
enum { ZETA1_A = 0, ZETA1_B = 1, ZETA1_C = 2, ZETA1_D = 3 };
enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2, OR_ENONPHYSICAL = -3 };

typedef struct {
    int dim, nx, ny;
    double x0, x1, y0, y1;
    double gamma;
    int viscous;
    double mu, prandtl;
    double c1, c2;
    double cfl, fixed_dt;
    int tau_zero;
    int bc[4];            /* x-lo, x-hi, y-lo, y-hi */
    int recon_mode;
    int zeta1_mode;
    double gamma_hi, gamma_lo, eps;
    int threads;
    /* prescribed boundaries of the double Mach reflection problem (Sec. 3.5) */
    double bc_state[4][4];   /* conservative state per side (inflow; behind the shock) */
    double shock_pre[4];     /* conservative state ahead of the shock */
    double shock_x0, shock_cot, shock_speed;   /* shock line x = shock_x0 + shock_cot (y + shock_speed t) */
} or_config;

/* ------------------------------------------------------------------------ */
/* Kinetic model, Sec. 2.1, Eqs. (3)-(4)                                     */
/* ------------------------------------------------------------------------ */

/* Internal degrees of freedom K.  2D: K = (5-3*gamma)/(gamma-1) + 1 (Sec. 2.1).
 * Reading: 1D uses K = (3-gamma)/(gamma-1), the value that gives the same
 * gamma with one translational degree of freedom (the paper gives only 2D). */
static double dof_K(int dim, double gam)
{
    if (dim == 2) return (5.0 - 3.0 * gam) / (gam - 1.0) + 1.0;
    return (3.0 - gam) / (gam - 1.0);
}

/* A polynomial in the particle velocity (u, v) and xi^2, kept as a term list. */
typedef struct {
    int n;
    double c[MAXT];
    unsigned char pu[MAXT], pv[MAXT], px[MAXT]; /* powers of u, v and of xi^2 */
} poly;

static void p_set(poly* p) { p->n = 0; }
static void p_term(poly* p, double c, int a, int b, int x)
{
    if (p->n >= MAXT) { fprintf(stderr, "hgks oracle: polynomial term overflow\n"); abort(); }
    p->c[p->n] = c; p->pu[p->n] = (unsigned char)a; p->pv[p->n] = (unsigned char)b;
    p->px[p->n] = (unsigned char)x; p->n++;
}
static void p_mul(const poly* a, const poly* b, poly* out)
{
    poly r; p_set(&r);
    for (int i = 0; i < a->n; i++)
        for (int j = 0; j < b->n; j++)
            p_term(&r, a->c[i] * b->c[j], a->pu[i] + b->pu[j], a->pv[i] + b->pv[j], a->px[i] + b->px[j]);
    *out = r;
}
static void p_add(const poly* a, const poly* b, poly* out)
{
    poly r = *a;
    for (int j = 0; j < b->n; j++) p_term(&r, b->c[j], b->pu[j], b->pv[j], b->px[j]);
    *out = r;
}

/* psi_alpha of Eq. (4): (1, u, v, (u^2+v^2+xi^2)/2) in 2D, (1, u, (u^2+xi^2)/2) in 1D. */
static void psi_poly(int dim, int alpha, poly* p)
{
    p_set(p);
    int nv = dim + 2;
    if (alpha == 0) p_term(p, 1.0, 0, 0, 0);
    else if (alpha == 1) p_term(p, 1.0, 1, 0, 0);
    else if (dim == 2 && alpha == 2) p_term(p, 1.0, 0, 1, 0);
    else if (alpha == nv - 1) {
        p_term(p, 0.5, 2, 0, 0);
        if (dim == 2) p_term(p, 0.5, 0, 2, 0);
        p_term(p, 0.5, 0, 0, 1);
    }
}

/* a . psi for a coefficient vector a (the micro-slopes a, A of Eqs. (7)-(9)). */
static void slope_poly(int dim, const double* a, poly* p)
{
    int nv = dim + 2;
    poly t; p_set(p);
    for (int k = 0; k < nv; k++) {
        psi_poly(dim, k, &t);
        for (int j = 0; j < t.n; j++) p_term(p, a[k] * t.c[j], t.pu[j], t.pv[j], t.px[j]);
    }
}

/* Moments of the Maxwellian of Eq. (3), divided by rho:
 *   u[n] = <u^n>,  up[n] = <u^n>_{u>0},  un[n] = <u^n>_{u<0},  v[n] = <v^n>,
 *   x[k] = <xi^(2k)>.
 * From the Gaussian integrals: <u^0>_{u>0} = erfc(-sqrt(lam) U)/2,
 * <u^1>_{u>0} = U <u^0>_{u>0} + exp(-lam U^2)/(2 sqrt(pi lam)), and by parts
 * <u^(n+2)> = U <u^(n+1)> + (n+1)/(2 lam) <u^n> on the full and both half lines. */
typedef struct {
    double rho, U, V, lam, K;
    double u[NMOM], up[NMOM], un[NMOM], v[NMOM], x[4];
} mom;

static void moments(int dim, double K, double rho, double U, double V, double lam, mom* m)
{
    m->rho = rho; m->U = U; m->V = V; m->lam = lam; m->K = K;
    double sl = sqrt(lam);
    double e = exp(-lam * U * U) / (2.0 * sqrt(M_PI * lam));
    m->u[0] = 1.0; m->u[1] = U;
    m->up[0] = 0.5 * erfc(-sl * U); m->up[1] = U * m->up[0] + e;
    m->un[0] = 0.5 * erfc(sl * U);  m->un[1] = U * m->un[0] - e;
    for (int n = 0; n + 2 < NMOM; n++) {
        double f = (double)(n + 1) / (2.0 * lam);
        m->u[n + 2] = U * m->u[n + 1] + f * m->u[n];
        m->up[n + 2] = U * m->up[n + 1] + f * m->up[n];
        m->un[n + 2] = U * m->un[n + 1] + f * m->un[n];
    }
    if (dim == 2) {
        m->v[0] = 1.0; m->v[1] = V;
        for (int n = 0; n + 2 < NMOM; n++) m->v[n + 2] = V * m->v[n + 1] + (double)(n + 1) / (2.0 * lam) * m->v[n];
    } else {
        for (int n = 0; n < NMOM; n++) m->v[n] = (n == 0) ? 1.0 : 0.0;
    }
    /* each of the K internal components is a Gaussian of variance 1/(2 lam):
       <xi^(2k+2)> = <xi^(2k)> (K + 2k)/(2 lam) */
    m->x[0] = 1.0;
    for (int k = 0; k < 3; k++) m->x[k + 1] = m->x[k] * (K + 2.0 * k) / (2.0 * lam);
}

/* int p g dXi over the full line (half = 0), u > 0 (half = +1) or u < 0 (half = -1). */
static double integ(const poly* p, const mom* m, int half)
{
    const double* mu = half > 0 ? m->up : (half < 0 ? m->un : m->u);
    double s = 0.0;
    for (int i = 0; i < p->n; i++) s += p->c[i] * mu[p->pu[i]] * m->v[p->pv[i]] * m->x[p->px[i]];
    return m->rho * s;
}

/* Vector of moments int psi_alpha * p * g dXi. */
static void integ_psi(int dim, const poly* p, const mom* m, int half, double* out)
{
    poly ps, t;
    for (int a = 0; a < dim + 2; a++) {
        psi_poly(dim, a, &ps);
        p_mul(&ps, p, &t);
        out[a] = integ(&t, m, half);
    }
}

/* Dense solve A x = b by Gaussian elimination with partial pivoting (n <= 4). */
static void dense_solve(int n, double A[4][4], const double* b, double* x)
{
    double M[4][5];
    for (int i = 0; i < n; i++) { for (int j = 0; j < n; j++) M[i][j] = A[i][j]; M[i][n] = b[i]; }
    for (int k = 0; k < n; k++) {
        int piv = k;
        for (int i = k + 1; i < n; i++) if (fabs(M[i][k]) > fabs(M[piv][k])) piv = i;
        if (piv != k) for (int j = 0; j <= n; j++) { double t = M[k][j]; M[k][j] = M[piv][j]; M[piv][j] = t; }
        for (int i = k + 1; i < n; i++) {
            double f = M[i][k] / M[k][k];
            for (int j = k; j <= n; j++) M[i][j] -= f * M[k][j];
        }
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = M[i][n];
        for (int j = i + 1; j < n; j++) s -= M[i][j] * x[j];
        x[i] = s / M[i][i];
    }
}

/* Conservative W -> (rho, U, V, lambda) with lambda = rho / (2 p) (Sec. 2.1). */
static void to_prim(int dim, double gam, const double* W, double* rho, double* U, double* V, double* lam, double* p)
{
    *rho = W[0];
    *U = W[1] / W[0];
    *V = (dim == 2) ? W[2] / W[0] : 0.0;
    double E = W[dim + 1];
    *p = (gam - 1.0) * (E - 0.5 * W[0] * ((*U) * (*U) + (*V) * (*V)));
    *lam = W[0] / (2.0 * (*p));
}

/* The moment matrix M[a][b] = int psi_a psi_b g dXi. */
static void moment_matrix(int dim, const mom* m, double M[4][4])
{
    poly pa, pb, t;
    for (int a = 0; a < dim + 2; a++)
        for (int b = 0; b < dim + 2; b++) {
            psi_poly(dim, a, &pa); psi_poly(dim, b, &pb); p_mul(&pa, &pb, &t);
            M[a][b] = integ(&t, m, 0);
        }
}

/* Micro-slope a with <a> = dW (Eq. (8)): int psi (a . psi) g dXi = dW. */
static void micro_slope(int dim, const mom* m, const double* dW, double* a)
{
    double M[4][4];
    moment_matrix(dim, m, M);
    dense_solve(dim + 2, M, dW, a);
}

/* Time slope A from the compatibility condition <a1 u + a2 v + A> = 0 (Eq. (9)). */
static void time_slope(int dim, const mom* m, const double* a1, const double* a2, double* A)
{
    poly s1, s2, uu, vv, t1, t2, t;
    double M[4][4], rhs[4];
    slope_poly(dim, a1, &s1);
    p_set(&uu); p_term(&uu, 1.0, 1, 0, 0);
    p_mul(&s1, &uu, &t1);
    if (dim == 2) {
        slope_poly(dim, a2, &s2);
        p_set(&vv); p_term(&vv, 1.0, 0, 1, 0);
        p_mul(&s2, &vv, &t2);
        p_add(&t1, &t2, &t);
    } else {
        t = t1;
    }
    integ_psi(dim, &t, m, 0, rhs);
    for (int k = 0; k < dim + 2; k++) rhs[k] = -rhs[k];
    moment_matrix(dim, m, M);
    dense_solve(dim + 2, M, rhs, A);
}

/* ------------------------------------------------------------------------ */
/* Gas-kinetic flux at one interface point, Sec. 2.1, Eqs. (6)-(12), (46)-(47)*/
/* ------------------------------------------------------------------------ */

/* Local frame: x is the interface normal.  Inputs are the reconstructed
 * non-equilibrium states on the two sides and their normal (x) and tangential
 * (y, 2D only) derivatives.  Output: the time-integrated fluxes of Eq. (12)
 * for delta = dt and delta = dt/2, each nv components.
 * Returns 0, or OR_ENONPHYSICAL if a side has rho <= 0 or p <= 0. */
static int gks_point_flux(const or_config* cfg, const double* Wl, const double* Wlx, const double* Wly,
                          const double* Wr, const double* Wrx, const double* Wry, double dt,
                          double* F_dt, double* F_half)
{
    int dim = cfg->dim, nv = dim + 2;
    double gam = cfg->gamma, K = dof_K(dim, gam);
    double rl, Ul, Vl, ll, pl, rr, Ur, Vr, lr, pr;
    to_prim(dim, gam, Wl, &rl, &Ul, &Vl, &ll, &pl);
    to_prim(dim, gam, Wr, &rr, &Ur, &Vr, &lr, &pr);
    if (!(rl > 0.0) || !(pl > 0.0) || !(rr > 0.0) || !(pr > 0.0)) return OR_ENONPHYSICAL;
    mom ml, mr, mc;
    moments(dim, K, rl, Ul, Vl, ll, &ml);
    moments(dim, K, rr, Ur, Vr, lr, &mr);

    /* non-equilibrium slopes of each side: <a1^k> = dQ/dn_x, <a2^k> = dQ/dn_y (Eq. (8)),
       A^k from <a1^k u + a2^k v + A^k> = 0 (Eq. (9)) */
    double zero[4] = {0, 0, 0, 0};
    double a1l[4], a2l[4] = {0, 0, 0, 0}, Al[4], a1r[4], a2r[4] = {0, 0, 0, 0}, Ar[4];
    micro_slope(dim, &ml, Wlx, a1l);
    micro_slope(dim, &mr, Wrx, a1r);
    if (dim == 2) { micro_slope(dim, &ml, Wly, a2l); micro_slope(dim, &mr, Wry, a2r); }
    time_slope(dim, &ml, a1l, dim == 2 ? a2l : zero, Al);
    time_slope(dim, &mr, a1r, dim == 2 ? a2r : zero, Ar);

    /* equilibrium state by kinetic weighting, Eqs. (46)-(47) and Eq. (9).
       Reading: the second integral of Eqs. (46)-(47) is over u < 0. */
    poly one, s;
    double Wc[4], Wcx[4], Wcy[4] = {0, 0, 0, 0}, tl[4], tr[4];
    p_set(&one); p_term(&one, 1.0, 0, 0, 0);
    integ_psi(dim, &one, &ml, +1, tl); integ_psi(dim, &one, &mr, -1, tr);
    for (int k = 0; k < nv; k++) Wc[k] = tl[k] + tr[k];
    slope_poly(dim, a1l, &s); integ_psi(dim, &s, &ml, +1, tl);
    slope_poly(dim, a1r, &s); integ_psi(dim, &s, &mr, -1, tr);
    for (int k = 0; k < nv; k++) Wcx[k] = tl[k] + tr[k];
    if (dim == 2) {
        slope_poly(dim, a2l, &s); integ_psi(dim, &s, &ml, +1, tl);
        slope_poly(dim, a2r, &s); integ_psi(dim, &s, &mr, -1, tr);
        for (int k = 0; k < nv; k++) Wcy[k] = tl[k] + tr[k];
    }
    double rc, Uc, Vc, lc, pc;
    to_prim(dim, gam, Wc, &rc, &Uc, &Vc, &lc, &pc);
    if (!(rc > 0.0) || !(pc > 0.0)) return OR_ENONPHYSICAL;
    moments(dim, K, rc, Uc, Vc, lc, &mc);
    double ab1[4], ab2[4] = {0, 0, 0, 0}, Ab[4];
    micro_slope(dim, &mc, Wcx, ab1);
    if (dim == 2) micro_slope(dim, &mc, Wcy, ab2);
    time_slope(dim, &mc, ab1, dim == 2 ? ab2 : zero, Ab);

    /* collision time, Sec. 3 preamble */
    double tau;
    double jump = fabs((pl - pr) / (pl + pr));
    if (cfg->tau_zero) tau = 0.0;
    else if (cfg->viscous) tau = cfg->mu / pc + cfg->c2 * jump * dt;
    else tau = cfg->c1 * dt + cfg->c2 * jump * dt;

    /* the six velocity moments multiplying the time coefficients of Eq. (10), each
       integrated against u psi:  g0;  (ab1 u + ab2 v) g0;  Ab g0;
       and for each side g^k, (a1^k u + a2^k v) g^k, A^k g^k over its half line */
    poly uu, vv, t, t2, pa;
    p_set(&uu); p_term(&uu, 1.0, 1, 0, 0);
    p_set(&vv); p_term(&vv, 1.0, 0, 1, 0);
    double M1[4], M2[4], M3[4], L4[4], L5[4], L6[4], R4[4], R5[4], R6[4];

    integ_psi(dim, &uu, &mc, 0, M1);
    slope_poly(dim, ab1, &pa); p_mul(&pa, &uu, &t);
    if (dim == 2) { slope_poly(dim, ab2, &pa); p_mul(&pa, &vv, &t2); p_add(&t, &t2, &t); }
    p_mul(&t, &uu, &t); integ_psi(dim, &t, &mc, 0, M2);
    slope_poly(dim, Ab, &pa); p_mul(&pa, &uu, &t); integ_psi(dim, &t, &mc, 0, M3);

    integ_psi(dim, &uu, &ml, +1, L4);
    slope_poly(dim, a1l, &pa); p_mul(&pa, &uu, &t);
    if (dim == 2) { slope_poly(dim, a2l, &pa); p_mul(&pa, &vv, &t2); p_add(&t, &t2, &t); }
    p_mul(&t, &uu, &t); integ_psi(dim, &t, &ml, +1, L5);
    slope_poly(dim, Al, &pa); p_mul(&pa, &uu, &t); integ_psi(dim, &t, &ml, +1, L6);

    integ_psi(dim, &uu, &mr, -1, R4);
    slope_poly(dim, a1r, &pa); p_mul(&pa, &uu, &t);
    if (dim == 2) { slope_poly(dim, a2r, &pa); p_mul(&pa, &vv, &t2); p_add(&t, &t2, &t); }
    p_mul(&t, &uu, &t); integ_psi(dim, &t, &mr, -1, R5);
    slope_poly(dim, Ar, &pa); p_mul(&pa, &uu, &t); integ_psi(dim, &t, &mr, -1, R6);

    /* Prandtl-number fix (not in the paper, whose BGK flux has Pr = 1): for a viscous
       run with Pr != 1 the energy flux gains (1/Pr - 1) q, where q is the time-integrated
       heat flux of the interface distribution of Eq. (10),
         q(d) = int_0^d int (u - Uc) (|u - Uc|^2 + xi^2)/2 f dXi dt,
       with (Uc, Vc) the velocity of the equilibrium state W^c: each of the six terms of
       Eq. (10) integrated against h = (u-Uc)((u-Uc)^2 + (v-Vc)^2 + xi^2)/2 instead of u psi. */
    double hM[3] = {0, 0, 0}, hL[3] = {0, 0, 0}, hR[3] = {0, 0, 0};
    int prfix = cfg->viscous && cfg->prandtl != 1.0;
    if (prfix) {
        poly cu, cv, xi2, s2, h, w;
        p_set(&cu); p_term(&cu, 1.0, 1, 0, 0); p_term(&cu, -Uc, 0, 0, 0);
        p_set(&cv); p_term(&cv, 1.0, 0, 1, 0); p_term(&cv, -Vc, 0, 0, 0);
        p_set(&xi2); p_term(&xi2, 1.0, 0, 0, 1);
        p_mul(&cu, &cu, &s2);
        if (dim == 2) { p_mul(&cv, &cv, &w); p_add(&s2, &w, &s2); }
        p_add(&s2, &xi2, &s2);
        p_mul(&cu, &s2, &h);
        for (int i = 0; i < h.n; i++) h.c[i] *= 0.5;
        /* g0, (ab1 u + ab2 v) g0, Ab g0 */
        hM[0] = integ(&h, &mc, 0);
        slope_poly(dim, ab1, &pa); p_mul(&pa, &uu, &t);
        if (dim == 2) { slope_poly(dim, ab2, &pa); p_mul(&pa, &vv, &t2); p_add(&t, &t2, &t); }
        p_mul(&t, &h, &w); hM[1] = integ(&w, &mc, 0);
        slope_poly(dim, Ab, &pa); p_mul(&pa, &h, &w); hM[2] = integ(&w, &mc, 0);
        /* each side over its half line: g^k, (a1^k u + a2^k v) g^k, A^k g^k */
        for (int side = 0; side < 2; side++) {
            const mom* ms = side == 0 ? &ml : &mr;
            int half = side == 0 ? +1 : -1;
            const double* a1 = side == 0 ? a1l : a1r;
            const double* a2 = side == 0 ? a2l : a2r;
            const double* A = side == 0 ? Al : Ar;
            double* out = side == 0 ? hL : hR;
            out[0] = integ(&h, ms, half);
            slope_poly(dim, a1, &pa); p_mul(&pa, &uu, &t);
            if (dim == 2) { slope_poly(dim, a2, &pa); p_mul(&pa, &vv, &t2); p_add(&t, &t2, &t); }
            p_mul(&t, &h, &w); out[1] = integ(&w, ms, half);
            slope_poly(dim, A, &pa); p_mul(&pa, &h, &w); out[2] = integ(&w, ms, half);
        }
    }

    /* Reading: in Eq. (10) particles with u > 0 arrive from the left state (the
       printed H(u) / (1-H(u)) labels are swapped with respect to Eq. (7)). */
    for (int pass = 0; pass < 2; pass++) {
        double d = pass == 0 ? dt : 0.5 * dt;
        double C1, C2, C3, C4, C5, C6;
        if (tau == 0.0) {
            /* the tau -> 0 limit of the integrals below, taken explicitly */
            C1 = d; C2 = 0.0; C3 = 0.5 * d * d; C4 = 0.0; C5 = 0.0; C6 = 0.0;
        } else {
            double e = exp(-d / tau);
            /* int_0^d of each time factor of Eq. (10) */
            C1 = d - tau * (1.0 - e);                                        /* (1 - e^{-t/tau})            */
            C2 = 2.0 * tau * tau * (1.0 - e) - tau * d * (1.0 + e);          /* ((t+tau)e^{-t/tau} - tau)   */
            C3 = 0.5 * d * d - tau * d + tau * tau * (1.0 - e);              /* (t - tau + tau e^{-t/tau})  */
            C4 = tau * (1.0 - e);                                            /* e^{-t/tau}                  */
            C5 = -(2.0 * tau * tau * (1.0 - e) - tau * d * e);               /* -(tau+t) e^{-t/tau}         */
            C6 = -tau * tau * (1.0 - e);                                     /* -tau e^{-t/tau}             */
        }
        double* out = pass == 0 ? F_dt : F_half;
        for (int k = 0; k < nv; k++)
            out[k] = C1 * M1[k] + C2 * M2[k] + C3 * M3[k]
                   + C4 * (L4[k] + R4[k]) + C5 * (L5[k] + R5[k]) + C6 * (L6[k] + R6[k]);
        if (prfix) {
            double q = C1 * hM[0] + C2 * hM[1] + C3 * hM[2]
                     + C4 * (hL[0] + hR[0]) + C5 * (hL[1] + hR[1]) + C6 * (hL[2] + hR[2]);
            out[nv - 1] += (1.0 / cfg->prandtl - 1.0) * q;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Hybrid WENO-AO reconstruction, Sec. 2.3.1                                 */
/* ------------------------------------------------------------------------ */

/* Steps 1-3 for one component on the window q[0..4] = Q_{i-2..i+2}.
 * Returns 1 if the cell is troubled before the Step-4 spreading.
 * Coordinates are in cell units (x/dx), where Eq. (24) reads
 *   abar1 = -N/10,  abar2 = D/34,
 *   N = (2 Q_{i-2} + Q_{i-1}) - (2 Q_{i+2} + Q_{i+1}),
 *   D = (4 Q_{i-2} + Q_{i-1}) + (4 Q_{i+2} + Q_{i+1}) - 10 Q_i.
 * Step 1, |2 abar2| <= zeta1 in physical units, is tested as |D| <= Z1 with
 * Z1 = 17 zeta1 dx^2 precomputed.  Step 3 uses the conservative quadratic on
 * I_{i-1}, I_i, I_{i+1}: ahat1 = (Q_{i+1}-Q_{i-1})/2, ahat2 = ((Q_{i-1}+Q_{i+1}) - 2Q_i)/2.
 * Reading: both intervals are closed (|xbar| <= 5/2 is "inside", |xbar-xhat| <= 1/4
 * is non-troubled); the 1e-30 guard of Step 3 is applied in cell units.
 * hmix > 0 selects reading D of Step 3 (zeta1 reading D): the printed abar1, abar2
 * carry dx, so xbar is a length (xbar dx), while the conservative quadratic of Step 3,
 * whose coefficients are not printed, is taken in cell units, so xhat stays a cell
 * count; the test is then |xbar hmix - xhat| <= hmix/4 with hmix = dx (zeta2 = dx/4). */
static int indicator_raw(const double* q, double Z1, double hmix)
{
    double D = fma(-10.0, q[2], fma(4.0, q[0], q[1]) + fma(4.0, q[4], q[3]));
    if (fabs(D) <= Z1) return 0;                                    /* Step 1 */
    double N = fma(2.0, q[0], q[1]) - fma(2.0, q[4], q[3]);
    double a1 = -(N / 10.0);
    double a2 = D / 34.0;
    double xbar = -a1 / (2.0 * a2);
    if (!(fabs(xbar) <= 2.5)) return 0;                             /* Step 2 */
    double ah1 = 0.5 * (q[3] - q[1]);
    double ah2 = 0.5 * ((q[1] + q[3]) - 2.0 * q[2]);
    double den = 2.0 * ah2 + (ah2 == 0.0 ? 1e-30 : 0.0);
    double xhat = -ah1 / den;
    if (hmix > 0.0) {
        if (fabs(xbar * hmix - xhat) <= 0.25 * hmix) return 0;     /* Step 3, reading D */
    } else if (fabs(xbar - xhat) <= 0.25) {
        return 0;                                                   /* Step 3 */
    }
    return 1;
}

/* Robustness of the decision of indicator_raw under a perturbation of every input by
 * eta = 1e-13 max|q|: the smallest ratio, over the steps taken, of the distance of a
 * tested quantity from its threshold to the first-order change eta can cause in it
 * (D: 20 eta; xbar = 1.7 N/D; xhat = -ahat1/(2 ahat2), whose change grows like
 * 1/|ahat2|).  A ratio below 1 marks a decision that round-off can decide.  Test aid
 * only; it does not change any decision. */
static double indicator_margin(const double* q, double Z1)
{
    double scale = 0.0;
    for (int s = 0; s < 5; s++) scale = fmax(scale, fabs(q[s]));
    double eta = 1e-13 * scale + 1e-300;
    double D = fma(-10.0, q[2], fma(4.0, q[0], q[1]) + fma(4.0, q[4], q[3]));
    double r = fabs(fabs(D) - Z1) / (20.0 * eta);
    if (fabs(D) <= Z1) return r;
    double N = fma(2.0, q[0], q[1]) - fma(2.0, q[4], q[3]);
    double a1 = -(N / 10.0);
    double a2 = D / 34.0;
    double xbar = -a1 / (2.0 * a2);
    double dxbar = 1.7 * eta * (6.0 + 20.0 * fabs(N) / fabs(D)) / fabs(D);
    r = fmin(r, fabs(fabs(xbar) - 2.5) / dxbar);
    if (!(fabs(xbar) <= 2.5)) return r;
    double ah1 = 0.5 * (q[3] - q[1]);
    double ah2 = 0.5 * ((q[1] + q[3]) - 2.0 * q[2]);
    if (fabs(ah2) <= 2.0 * eta) {
        /* xhat = -ahat1/(2 ahat2) can take any value of magnitude >= (|ahat1| - eta)/(8 eta) */
        double lo = (fabs(ah1) - eta) / (8.0 * eta);
        return fmin(r, lo > fabs(xbar) + 0.25 ? (lo - fabs(xbar) - 0.25) / (fabs(xbar) + 0.25) : 0.0);
    }
    double xhat = -ah1 / (2.0 * ah2);
    double dxhat = eta * (1.0 + 4.0 * fabs(xhat)) / (2.0 * fabs(ah2));
    return fmin(r, fabs(fabs(xbar - xhat) - 0.25) / (dxhat + dxbar));
}

/* Step 5, Eqs. (26)-(27) (index typos corrected: Q_1 -> Q_{i+1}):
 * value and derivative at x_{i+1/2} from the window of cell i. */
static void linear_left(const double* q, double inv12h, double* val, double* der)
{
    double t = fma(-13.0, q[1], 2.0 * q[0]);
    t = fma(47.0, q[2], t);
    t = fma(27.0, q[3], t);
    t = fma(-3.0, q[4], t);
    *val = t * (1.0 / 60.0);
    double s = fma(-15.0, q[2], q[1]);
    s = fma(15.0, q[3], s);
    s = s - q[4];
    *der = s * inv12h;
}

/* Eqs. (28)-(29) (typos Q_1 -> Q_{i+1}, Q_0 -> Q_i corrected): value and
 * derivative at x_{i-1/2} from the window of cell i, evaluated as the mirror
 * image of linear_left so that mirrored data give mirrored values exactly. */
static void linear_right(const double* q, double inv12h, double* val, double* der)
{
    double t = fma(-13.0, q[3], 2.0 * q[4]);
    t = fma(47.0, q[2], t);
    t = fma(27.0, q[1], t);
    t = fma(-3.0, q[0], t);
    *val = t * (1.0 / 60.0);
    double s = fma(-15.0, q[2], q[3]);
    s = fma(15.0, q[1], s);
    s = s - q[0];
    *der = -(s * inv12h);
}

/* Linear weights of Eq. (35) (Reading: the printed labels 1,2,3 mean the
 * sub-stencils S0, S1, S2; S1 is the central one) and derived constants. */
typedef struct { double g[4], g3inv, gr[3], eps; } ao_consts;

static void ao_setup(double ghi, double glo, double eps, ao_consts* k)
{
    k->g[3] = ghi;
    k->g[0] = ((1.0 - ghi) * (1.0 - glo)) * 0.5;
    k->g[2] = k->g[0];
    k->g[1] = (1.0 - ghi) * glo;
    k->g3inv = 1.0 / ghi;
    for (int j = 0; j < 3; j++) k->gr[j] = k->g[j] / ghi;
    k->eps = eps;
}

/* Smoothness indicators of Eq. (39) in cell units (the dx^(2q-1) factors make
 * beta scale-free).  Quadratics: int (p')^2 + int (p'')^2 over the cell, in the
 * closed form (13/12) s^2 + (1/4) t^2.  Quartic: p = c0 + c1 xi + ... + c4 xi^4
 * fitted to the five averages (Eq. (33)); summing int (p^(q))^2 for q = 1..4 gives
 * c1^2 + c1 c3/2 + 13 c2^2/3 + 21 c2 c4/5 + 3129 c3^2/80 + 87617 c4^2/140. */
static void ao_betas(const double* q, double* b)
{
    double s0 = (q[0] - 2.0 * q[1]) + q[2], t0 = (q[0] - 4.0 * q[1]) + 3.0 * q[2];
    double s1 = (q[1] - 2.0 * q[2]) + q[3], t1 = q[1] - q[3];
    double s2 = (q[2] - 2.0 * q[3]) + q[4], t2 = (3.0 * q[2] - 4.0 * q[3]) + q[4];
    b[0] = (13.0 / 12.0) * (s0 * s0) + 0.25 * (t0 * t0);
    b[1] = (13.0 / 12.0) * (s1 * s1) + 0.25 * (t1 * t1);
    b[2] = (13.0 / 12.0) * (s2 * s2) + 0.25 * (t2 * t2);
    double c1 = (17.0 / 24.0) * (q[3] - q[1]) - (5.0 / 48.0) * (q[4] - q[0]);
    double c2 = ((0.75 * (q[1] + q[3]) - 0.0625 * (q[0] + q[4])) - 1.375 * q[2]);
    double c3 = (1.0 / 6.0) * (q[1] - q[3]) - (1.0 / 12.0) * (q[0] - q[4]);
    double c4 = ((1.0 / 24.0) * (q[0] + q[4]) - (1.0 / 6.0) * (q[1] + q[3])) + 0.25 * q[2];
    b[3] = ((((c1 * c1 + 0.5 * (c1 * c3)) + (13.0 / 3.0) * (c2 * c2)) + (21.0 / 5.0) * (c2 * c4))
            + (3129.0 / 80.0) * (c3 * c3)) + (87617.0 / 140.0) * (c4 * c4);
}

/* Normalised nonlinear weights, Eqs. (37), (38), (40).
 * Reading: the printed beta_3^{r3} in Eq. (38) is beta_2^{r3}.
 * Reading: the ratio delta/(beta_k + eps) of Eq. (37) enters squared, as in the
 * WENO-Z family the paper cites.  Evidence: with the square (and gamma_Hi =
 * gamma_Lo = 0.85) the WENO-AO/linear error ratio of the 1D sine wave equals the
 * Table 1/Table 2 ratio of Sec. 3.1 to three digits at dx = 1/10 and 1/20; as
 * printed, the weights leave half the weight on the quartic across the pressure
 * step of the blast wave (Sec. 3.2(c)) and the face pressure goes negative. */
static void ao_weights(const double* q, const ao_consts* k, double* wb)
{
    double b[4], w[4];
    ao_betas(q, b);
    double d = ((fabs(b[3] - b[0]) + fabs(b[3] - b[1])) + fabs(b[3] - b[2])) * (1.0 / 3.0);
    for (int j = 0; j < 4; j++) {
        double r = d / (b[j] + k->eps);
        w[j] = k->g[j] * (1.0 + r * r);
    }
    double inv = 1.0 / (((w[0] + w[1]) + w[2]) + w[3]);
    for (int j = 0; j < 4; j++) wb[j] = w[j] * inv;
}

/* The AO(5,3) combination of Eq. (41) applied to point values p[0..3] of the
 * three quadratics and the quartic. */
static double ao_combine(const double* wb, const ao_consts* k, const double* p)
{
    return wb[3] * (p[3] * k->g3inv - ((k->gr[0] * p[0] + k->gr[1] * p[1]) + k->gr[2] * p[2]))
         + ((wb[0] * p[0] + wb[1] * p[1]) + wb[2] * p[2]);
}

/* Point values and cell-unit derivatives at x_{i+1/2} (side = +1) or x_{i-1/2}
 * (side = -1) of the three quadratics (Eqs. (32), (43); typo in p_2(x_{i+1/2})
 * corrected to Q_i/3 + 5Q_{i+1}/6 - Q_{i+2}/6) and of the quartic (Eqs. (36), (44)). */
static void face_polys(const double* q, int side, double* pv, double* pd)
{
    if (side > 0) {
        pv[0] = ((2.0 * q[0] - 7.0 * q[1]) + 11.0 * q[2]) * (1.0 / 6.0);
        pv[1] = ((-q[1] + 5.0 * q[2]) + 2.0 * q[3]) * (1.0 / 6.0);
        pv[2] = ((2.0 * q[2] + 5.0 * q[3]) - q[4]) * (1.0 / 6.0);
        pv[3] = ((((2.0 * q[0] - 13.0 * q[1]) + 47.0 * q[2]) + 27.0 * q[3]) - 3.0 * q[4]) * (1.0 / 60.0);
        pd[0] = (q[0] - 3.0 * q[1]) + 2.0 * q[2];
        pd[1] = q[3] - q[2];
        pd[2] = q[3] - q[2];
        pd[3] = (((q[1] - 15.0 * q[2]) + 15.0 * q[3]) - q[4]) * (1.0 / 12.0);
    } else {
        pv[0] = ((-q[0] + 5.0 * q[1]) + 2.0 * q[2]) * (1.0 / 6.0);
        pv[1] = ((2.0 * q[1] + 5.0 * q[2]) - q[3]) * (1.0 / 6.0);
        pv[2] = ((11.0 * q[2] - 7.0 * q[3]) + 2.0 * q[4]) * (1.0 / 6.0);
        pv[3] = ((((-3.0 * q[0] + 27.0 * q[1]) + 47.0 * q[2]) - 13.0 * q[3]) + 2.0 * q[4]) * (1.0 / 60.0);
        pd[0] = q[2] - q[1];
        pd[1] = q[2] - q[1];
        pd[2] = (-2.0 * q[2] + 3.0 * q[3]) - q[4];
        pd[3] = (((q[0] - 15.0 * q[1]) + 15.0 * q[2]) - q[3]) * (1.0 / 12.0);
    }
}

/* Right eigenvectors R (columns) and left eigenvectors L = R^{-1} (rows) of
 * nx dF/dQ + ny dG/dQ at the state Q (Sec. 2.3.1, local characteristic
 * projection).  Columns: u - c, u (entropy), shear (2D), u + c. */
static void eigvec(int dim, double gam, const double* Q, double nx, double ny, double L[4][4], double R[4][4])
{
    double gm1 = gam - 1.0;
    double rho = Q[0], ri = 1.0 / rho;
    double U = Q[1] * ri;
    if (dim == 2) {
        double V = Q[2] * ri;
        double q2 = U * U + V * V;
        double p = gm1 * (Q[3] - (0.5 * rho) * q2);
        double c2 = (gam * p) * ri, c = sqrt(c2), ci = 1.0 / c;
        double H = (Q[3] + p) * ri;
        double un = U * nx + V * ny, ut = V * nx - U * ny;
        double b1 = gm1 / c2, b2 = (0.5 * b1) * q2;
        R[0][0] = 1.0;           R[0][1] = 1.0;        R[0][2] = 0.0; R[0][3] = 1.0;
        R[1][0] = U - c * nx;    R[1][1] = U;          R[1][2] = -ny; R[1][3] = U + c * nx;
        R[2][0] = V - c * ny;    R[2][1] = V;          R[2][2] = nx;  R[2][3] = V + c * ny;
        R[3][0] = H - un * c;    R[3][1] = 0.5 * q2;   R[3][2] = ut;  R[3][3] = H + un * c;
        L[0][0] = 0.5 * (b2 + un * ci); L[0][1] = -0.5 * (b1 * U + nx * ci); L[0][2] = -0.5 * (b1 * V + ny * ci); L[0][3] = 0.5 * b1;
        L[1][0] = 1.0 - b2;             L[1][1] = b1 * U;                    L[1][2] = b1 * V;                    L[1][3] = -b1;
        L[2][0] = -ut;                  L[2][1] = -ny;                       L[2][2] = nx;                        L[2][3] = 0.0;
        L[3][0] = 0.5 * (b2 - un * ci); L[3][1] = -0.5 * (b1 * U - nx * ci); L[3][2] = -0.5 * (b1 * V - ny * ci); L[3][3] = 0.5 * b1;
    } else {
        (void)ny;
        double q2 = U * U;
        double p = gm1 * (Q[2] - (0.5 * rho) * q2);
        double c2 = (gam * p) * ri, c = sqrt(c2), ci = 1.0 / c;
        double H = (Q[2] + p) * ri;
        double b1 = gm1 / c2, b2 = (0.5 * b1) * q2;
        R[0][0] = 1.0;        R[0][1] = 1.0;       R[0][2] = 1.0;
        R[1][0] = U - c;      R[1][1] = U;         R[1][2] = U + c;
        R[2][0] = H - U * c;  R[2][1] = 0.5 * q2;  R[2][2] = H + U * c;
        L[0][0] = 0.5 * (b2 + U * ci); L[0][1] = -0.5 * (b1 * U + ci); L[0][2] = 0.5 * b1;
        L[1][0] = 1.0 - b2;            L[1][1] = b1 * U;               L[1][2] = -b1;
        L[2][0] = 0.5 * (b2 - U * ci); L[2][1] = -0.5 * (b1 * U - ci); L[2][2] = 0.5 * b1;
    }
}

/* Reading (the paper states no safeguard): a reconstructed state with rho <= 0
 * or p <= 0 is replaced by the first-order one (the average it was reconstructed
 * in, with zero slope).  For rho > 0 and gamma > 1, p = (gamma - 1)(E - ke/rho)
 * is positive exactly when rho E - ke is; the test, in this fixed order:
 *   ke = 0.5 (m_x^2 + m_y^2),  rho E - ke > 0. */
static int nonphysical(int dim, double gam, const double* Q)
{
    (void)gam;
    double ke = dim == 2 ? 0.5 * (Q[1] * Q[1] + Q[2] * Q[2]) : 0.5 * (Q[1] * Q[1]);
    double pr = Q[dim + 1] * Q[0] - ke;
    return !(Q[0] > 0.0) || !(pr > 0.0);
}

/* y = M x with the fixed summation order ((m0 x0 + m1 x1) + m2 x2) + m3 x3. */
static void matvec(int nv, double M[4][4], const double* x, double* y)
{
    for (int r = 0; r < nv; r++) {
        double s = M[r][0] * x[0] + M[r][1] * x[1];
        for (int c = 2; c < nv; c++) s = s + M[r][c] * x[c];
        y[r] = s;
    }
}

/* Characteristic WENO-AO at the face x_{i+1/2} (side = +1) or x_{i-1/2}
 * (side = -1) of the cell whose window is Qw[j][comp], j = 0..4 (cells i-2..i+2),
 * projected with the eigenvectors at state Qs in direction (nx, ny).
 * Returns the conservative value and cell-unit derivative (caller divides by h). */
static void weno_ao_face(int dim, double gam, const ao_consts* k, double Qw[5][4], const double* Qs,
                         double nx, double ny, int side, double* val, double* der)
{
    int nv = dim + 2;
    double L[4][4], R[4][4], Uc[5][4], uv[4], ud[4];
    eigvec(dim, gam, Qs, nx, ny, L, R);
    for (int j = 0; j < 5; j++) matvec(nv, L, Qw[j], Uc[j]);
    for (int c = 0; c < nv; c++) {
        double q[5], wb[4], pv[4], pd[4];
        for (int j = 0; j < 5; j++) q[j] = Uc[j][c];
        ao_weights(q, k, wb);
        face_polys(q, side, pv, pd);
        uv[c] = ao_combine(wb, k, pv);
        ud[c] = ao_combine(wb, k, pd);
    }
    matvec(nv, R, uv, val);
    matvec(nv, R, ud, der);
}

/* ---- tangential (Gauss-point) evaluation: generic polynomial evaluation ---- */

/* Coefficients in cell units of the quadratic through the averages of cells
 * (o, o+1, o+2) relative to the cell (o in {-2,-1,0}), and of the quartic
 * through the five averages.  (Solutions of Eqs. (31) and (33).) */
static void quad_coeffs(const double* q3, int o, double* c)
{
    /* averages of 1, xi, xi^2 over cell m: 1, m, m^2 + 1/12; solve the 3x3 system */
    double A[4][4], b[4];
    for (int r = 0; r < 3; r++) {
        double m = (double)(o + r);
        A[r][0] = 1.0; A[r][1] = m; A[r][2] = m * m + 1.0 / 12.0; b[r] = q3[r];
    }
    dense_solve(3, A, b, c);
}
static void quartic_coeffs(const double* q, double* c)
{
    double c0 = 1067.0 / 960.0 * q[2] - 29.0 / 480.0 * (q[1] + q[3]) + 3.0 / 640.0 * (q[0] + q[4]);
    double c1 = 17.0 / 24.0 * (q[3] - q[1]) - 5.0 / 48.0 * (q[4] - q[0]);
    double c2 = 0.75 * (q[1] + q[3]) - 0.0625 * (q[0] + q[4]) - 1.375 * q[2];
    double c3 = (q[1] - q[3]) / 6.0 - (q[0] - q[4]) / 12.0;
    double c4 = (q[0] + q[4]) / 24.0 - (q[1] + q[3]) / 6.0 + 0.25 * q[2];
    c[0] = c0; c[1] = c1; c[2] = c2; c[3] = c3; c[4] = c4;
}
static double peval(const double* c, int deg, double x)
{
    double s = c[deg];
    for (int k = deg - 1; k >= 0; k--) s = s * x + c[k];
    return s;
}
static double pderiv(const double* c, int deg, double x)
{
    double s = deg * c[deg];
    for (int k = deg - 1; k >= 1; k--) s = s * x + k * c[k];
    return s;
}

/* Values (and cell-unit derivatives) at the two Gauss points xi = -g, +g of a
 * cell from its 5-average window, linear (quartic) or AO(5,3). */
static void gauss_linear(const double* q, double* v, double* d)
{
    double c[5], g = 0.5 / sqrt(3.0);
    quartic_coeffs(q, c);
    v[0] = peval(c, 4, -g); v[1] = peval(c, 4, g);
    d[0] = pderiv(c, 4, -g); d[1] = pderiv(c, 4, g);
}
static void gauss_ao(const double* q, const ao_consts* k, double* v, double* d)
{
    double wb[4], cq[3][3], c4[5], g = 0.5 / sqrt(3.0);
    ao_weights(q, k, wb);
    for (int s = 0; s < 3; s++) quad_coeffs(q + s, s - 2, cq[s]);
    quartic_coeffs(q, c4);
    for (int gp = 0; gp < 2; gp++) {
        double x = gp == 0 ? -g : g, pv[4], pd[4];
        for (int s = 0; s < 3; s++) { pv[s] = peval(cq[s], 2, x); pd[s] = pderiv(cq[s], 2, x); }
        pv[3] = peval(c4, 4, x); pd[3] = pderiv(c4, 4, x);
        v[gp] = ao_combine(wb, k, pv);
        d[gp] = ao_combine(wb, k, pd);
    }
}

/* ------------------------------------------------------------------------ */
/* Grid, boundary conditions, sweeps and the S2O4 step (Sec. 2.2, 2.3.3)      */
/* ------------------------------------------------------------------------ */

typedef struct {
    or_config c;
    int nv, NX, NY;          /* padded extents */
    double dx, dy, K;
    double Z1x, Z1y;         /* Step-1 thresholds in cell units, per direction */
    double hmx, hmy;         /* reading D of Step 3: the cell size per direction, else 0 */
    ao_consts ao;
} grid;

static double zeta1_scaled(int mode, double h)
{
    /* Z1 = 17 zeta1 h^2.  Reading B (default): zeta1 = 5/(17 h).
       A: zeta1 = (5/17) h.  C: zeta1 = 5/17 in cell units.  D: zeta1 as A, and Step 3
       compares a length with a cell count (see indicator_raw). */
    if (mode == ZETA1_A || mode == ZETA1_D) return 5.0 * h * h * h;
    if (mode == ZETA1_C) return 5.0;
    return 5.0 * h;
}

static int grid_setup(const or_config* c, grid* g)
{
    if (c->dim != 1 && c->dim != 2) return OR_EINVAL;
    if (c->nx < 1 || c->ny < 1 || (c->dim == 1 && c->ny != 1)) return OR_EINVAL;
    g->c = *c;
    g->nv = c->dim + 2;
    g->NX = c->nx + 2 * NG;
    g->NY = c->dim == 2 ? c->ny + 2 * NG : 1;
    g->dx = (c->x1 - c->x0) / c->nx;
    g->dy = c->dim == 2 ? (c->y1 - c->y0) / c->ny : 1.0;
    g->K = dof_K(c->dim, c->gamma);
    g->Z1x = zeta1_scaled(c->zeta1_mode, g->dx);
    g->Z1y = zeta1_scaled(c->zeta1_mode, g->dy);
    g->hmx = c->zeta1_mode == ZETA1_D ? g->dx : 0.0;
    g->hmy = c->zeta1_mode == ZETA1_D ? g->dy : 0.0;
    ao_setup(c->gamma_hi, c->gamma_lo, c->eps, &g->ao);
    return OR_OK;
}

/* padded index: comp k, row j (-NG..ny+NG-1), column i */
static inline size_t pidx(const grid* g, int k, int j, int i)
{
    int jj = g->c.dim == 2 ? j + NG : 0;
    return ((size_t)k * g->NY + jj) * g->NX + (size_t)(i + NG);
}

/* Ghost fill: x ghosts on the interior rows, then y ghosts over the full padded
 * width (this fills the corners).  Reading: non-reflecting = zero-gradient copy
 * of the boundary cell; reflecting / symmetric = mirror with the normal
 * momentum negated; no-slip adiabatic = mirror with both momenta negated.
 * Double Mach reflection (Sec. 3.5): the post-shock state flows in on the left
 * and on the bottom up to x = 1/6, the bottom is a slip wall from there on, and
 * the top follows the exact motion of the oblique Mach 10 shock.  Reading: each
 * ghost cell takes the state at its centre (x_c, y_c) at the time of the stage
 * (t^n in the first stage, t^n + dt/2 = t* in the second), the post-shock state
 * where x_c lies behind the shock line x = 1/6 + cot(60 deg) (y + 20 t), the
 * pre-shock state elsewhere.  (The shock moves at 10 along its normal, so its
 * trace on a horizontal line moves at 10 / sin 60 deg = cot 60 deg x 20.)  The
 * line's data are configuration values (shock_x0, shock_cot, shock_speed). */
static double cell_centre(double origin, int i, double h) { return origin + ((double)i + 0.5) * h; }

static void ghost_value(const grid* g, const double* Wp, int bc, int axis, int side, int k, int j, int i,
                        int src_j, int src_i, int mirror_j, int mirror_i, double t, double* out)
{
    int nv = g->nv;
    const or_config* c = &g->c;
    int sidx = 2 * axis + side;
    double v;
    if (bc == BC_INFLOW) { *out = c->bc_state[sidx][k]; return; }
    if (bc == BC_SHOCK_TRACK) {
        double xc = cell_centre(c->x0, i, g->dx), yc = cell_centre(c->y0, j, g->dy);
        double xs = c->shock_x0 + c->shock_cot * (yc + c->shock_speed * t);
        *out = xc < xs ? c->bc_state[sidx][k] : c->shock_pre[k];
        return;
    }
    if (bc == BC_SHOCK_WALL && cell_centre(c->x0, i, g->dx) < c->shock_x0) { *out = c->bc_state[sidx][k]; return; }
    if (bc == BC_PERIODIC || bc == BC_EXTRAP) v = Wp[pidx(g, k, src_j, src_i)];
    else {
        v = Wp[pidx(g, k, mirror_j, mirror_i)];
        int normal_mom = 1 + axis;                  /* rho U for x, rho V for y */
        if (k == normal_mom) v = -v;
        if (bc == BC_NOSLIP && k >= 1 && k <= nv - 2) { if (k != normal_mom) v = -v; }
    }
    *out = v;
}

static void fill_ghosts(const grid* g, double* Wp, double t)
{
    int nx = g->c.nx, ny = g->c.ny, nv = g->nv, dim = g->c.dim;
    int jlo = 0, jhi = dim == 2 ? ny : 1;
    for (int k = 0; k < nv; k++)
        for (int j = jlo; j < jhi; j++)
            for (int l = 1; l <= NG; l++) {
                int jr = dim == 2 ? j : 0;
                double v;
                int bl = g->c.bc[0], bh = g->c.bc[1];
                int srcL = bl == BC_PERIODIC ? nx - l : 0;
                ghost_value(g, Wp, bl, 0, 0, k, jr, -l, jr, srcL, jr, l - 1, t, &v);
                Wp[pidx(g, k, jr, -l)] = v;
                int srcH = bh == BC_PERIODIC ? l - 1 : nx - 1;
                ghost_value(g, Wp, bh, 0, 1, k, jr, nx - 1 + l, jr, srcH, jr, nx - l, t, &v);
                Wp[pidx(g, k, jr, nx - 1 + l)] = v;
            }
    if (dim == 1) return;
    for (int k = 0; k < nv; k++)
        for (int i = -NG; i < nx + NG; i++)
            for (int l = 1; l <= NG; l++) {
                double v;
                int bl = g->c.bc[2], bh = g->c.bc[3];
                int srcL = bl == BC_PERIODIC ? ny - l : 0;
                ghost_value(g, Wp, bl, 1, 0, k, -l, i, srcL, i, l - 1, i, t, &v);
                Wp[pidx(g, k, -l, i)] = v;
                int srcH = bh == BC_PERIODIC ? l - 1 : ny - 1;
                ghost_value(g, Wp, bh, 1, 1, k, ny - 1 + l, i, srcH, i, ny - l, i, t, &v);
                Wp[pidx(g, k, ny - 1 + l, i)] = v;
            }
}

/* Flag layout (per stage, per sweep):
 *   normal[(t + 3) * (nn + 2) + (n + 1)]   final flag of cell n in the line t,
 *                                          t in [-3, nt+2] (2D) or t = 0 (1D), n in [-1, nn]
 *   tang[t * (nn + 1) + m]                 bits 0..3 = final flags of the tangential
 *                                          passes of Q^l, Q^r, Q^l_n, Q^r_n at interface m,
 *                                          t in [0, nt), m in [0, nn]
 * where nn / nt are the cell counts normal / tangential to the sweep. */
typedef struct { uint8_t* normal; uint8_t* tang; double* nmargin; double* tmargin; } flag_out;

/* One sweep (dir 0: x-interfaces, dir 1: y-interfaces).  Writes, per interface
 * line segment, the line-averaged dt- and dt/2-integrated fluxes (global
 * component order) into Fdt, Fhalf laid out [nv][nt][nn+1]. */
static int sweep(const grid* g, const double* Wp, int dir, double dt, double* Fdt, double* Fhalf, flag_out* fo)
{
    const or_config* c = &g->c;
    int dim = c->dim, nv = g->nv;
    int nn = dir == 0 ? c->nx : c->ny;
    int nt = dim == 2 ? (dir == 0 ? c->ny : c->nx) : 1;
    double hn = dir == 0 ? g->dx : g->dy, ht = dir == 0 ? g->dy : g->dx;
    double Z1n = dir == 0 ? g->Z1x : g->Z1y, Z1t = dir == 0 ? g->Z1y : g->Z1x;
    double Hn = dir == 0 ? g->hmx : g->hmy, Ht = dir == 0 ? g->hmy : g->hmx;
    double inv12hn = 1.0 / (12.0 * hn);
    int th = dim == 2 ? 3 : 0;                 /* ghost lines needed tangentially */
    int tlo = -th, thi = nt + th;              /* lines [tlo, thi) */
    int nlines = thi - tlo;
    int perm[4] = {0, 1, 2, 3};                /* local (normal, tangential) momentum order */
    if (dim == 2 && dir == 1) { perm[1] = 2; perm[2] = 1; }
    int nm = nn + 1;                           /* interfaces m = 0..nn, between cells m-1 and m */
    int mode = c->recon_mode;

    /* local accessor: component k (local order) of cell n in line t */
#define QL(k, t, n) (dir == 0 ? Wp[pidx(g, perm[k], (t), (n))] : Wp[pidx(g, perm[k], (n), (t))])

    size_t nline = (size_t)nlines * nm;
    double* line = (double*)malloc(sizeof(double) * nline * 4 * nv);  /* [line][m][4 quantities][nv] */
    uint8_t* nflag = (uint8_t*)calloc((size_t)nlines * (nn + 2), 1);
    if (!line || !nflag) { free(line); free(nflag); return OR_ENOMEM; }
    int status = OR_OK;

    /* Step 1 of Sec. 2.3.3: normal reconstruction on every line, with the
       troubled-cell indicator (Steps 1-4 of Sec. 2.3.1) on the cell averages. */
#pragma omp parallel for schedule(dynamic)
    for (int t = tlo; t < thi; t++) {
        int L = t - tlo;
        uint8_t raw[4096 + 8];
        double rmar[4096 + 8];
        uint8_t* rawp = nn + 4 <= 4096 ? raw : (uint8_t*)malloc((size_t)nn + 8);
        double* rmp = nn + 4 <= 4096 ? rmar : (double*)malloc(sizeof(double) * ((size_t)nn + 8));
        for (int n = -2; n <= nn + 1; n++) {
            int tr = 0;
            double mg = INFINITY;
            if (mode == RECON_HYBRID)
                for (int k = 0; k < nv; k++) {
                    double q[5];
                    for (int s = 0; s < 5; s++) q[s] = QL(k, t, n - 2 + s);
                    tr |= indicator_raw(q, Z1n, Hn);
                    if (fo && fo->nmargin) mg = fmin(mg, indicator_margin(q, Z1n));
                }
            rawp[n + 2] = (uint8_t)tr;
            rmp[n + 2] = mg;
        }
        for (int n = -1; n <= nn; n++) {
            uint8_t f;
            if (mode == RECON_LINEAR) f = 0;
            else if (mode == RECON_WENOAO) f = 1;
            else f = rawp[n + 1] | rawp[n + 2] | rawp[n + 3];        /* Step 4 */
            nflag[(size_t)L * (nn + 2) + (n + 1)] = f;
            if (fo && fo->nmargin)
                fo->nmargin[(size_t)L * (nn + 2) + (n + 1)] = fmin(rmp[n + 1], fmin(rmp[n + 2], rmp[n + 3]));
        }
        if (rawp != raw) free(rawp);
        if (rmp != rmar) free(rmp);
        for (int m = 0; m < nm; m++) {
            double* out = line + ((size_t)L * nm + m) * 4 * nv;
            int il = m - 1, ir = m;                                   /* left cell, right cell */
            double Qs[4];
            for (int k = 0; k < nv; k++) Qs[k] = (QL(k, t, il) + QL(k, t, ir)) * 0.5;
            for (int side = 0; side < 2; side++) {
                int ic = side == 0 ? il : ir;
                uint8_t f = nflag[(size_t)L * (nn + 2) + (ic + 1)];
                double* val = out + (side == 0 ? 0 : 1) * nv;          /* Q^l, Q^r */
                double* der = out + (side == 0 ? 2 : 3) * nv;          /* Q^l_n, Q^r_n */
                if (!f) {
                    for (int k = 0; k < nv; k++) {
                        double q[5];
                        for (int s = 0; s < 5; s++) q[s] = QL(k, t, ic - 2 + s);
                        if (side == 0) linear_left(q, inv12hn, &val[k], &der[k]);
                        else linear_right(q, inv12hn, &val[k], &der[k]);
                    }
                } else {
                    double Qw[5][4], d[4];
                    for (int s = 0; s < 5; s++) for (int k = 0; k < nv; k++) Qw[s][k] = QL(k, t, ic - 2 + s);
                    weno_ao_face(dim, c->gamma, &g->ao, Qw, Qs, 1.0, 0.0, side == 0 ? +1 : -1, val, d);
                    for (int k = 0; k < nv; k++) der[k] = d[k] * (1.0 / hn);
                }
                if (nonphysical(dim, c->gamma, val))
                    for (int k = 0; k < nv; k++) { val[k] = QL(k, t, ic); der[k] = 0.0; }
            }
        }
    }
    if (fo && fo->normal)
        for (int L = 0; L < nlines; L++)
            for (int n = 0; n < nn + 2; n++) fo->normal[(size_t)L * (nn + 2) + n] = nflag[(size_t)L * (nn + 2) + n];

    /* Step 2-3 of Sec. 2.3.3 and the flux at the Gauss points */
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < nt; t++) {
        for (int m = 0; m < nm; m++) {
            double gW[2][6][4];   /* per Gauss point: Wl, Wlx, Wly, Wr, Wrx, Wry (local order) */
            uint8_t tbits = 0;
            double tmg = INFINITY;
            if (dim == 1) {
                const double* ln = line + ((size_t)(t - tlo) * nm + m) * 4 * nv;
                for (int k = 0; k < nv; k++) {
                    gW[0][0][k] = ln[0 * nv + k]; gW[0][1][k] = ln[2 * nv + k]; gW[0][2][k] = 0.0;
                    gW[0][3][k] = ln[1 * nv + k]; gW[0][4][k] = ln[3 * nv + k]; gW[0][5][k] = 0.0;
                }
            } else {
                /* tangential state for the characteristic projection.  Reading: the
                   average of the two cell averages beside the segment, direction = tangent */
                double Qs[4];
                for (int k = 0; k < nv; k++) Qs[k] = (QL(k, t, m - 1) + QL(k, t, m)) * 0.5;
                for (int X = 0; X < 4; X++) {
                    /* tangential troubled flags on the line values of quantity X */
                    int raw3[3];
                    for (int dt3 = -1; dt3 <= 1; dt3++) {
                        int tr = 0;
                        if (mode == RECON_HYBRID)
                            for (int k = 0; k < nv; k++) {
                                double q[5];
                                for (int s = 0; s < 5; s++) {
                                    int tt = t + dt3 - 2 + s;
                                    q[s] = line[((size_t)(tt - tlo) * nm + m) * 4 * nv + X * nv + k];
                                }
                                tr |= indicator_raw(q, Z1t, Ht);
                                if (fo && fo->tmargin) tmg = fmin(tmg, indicator_margin(q, Z1t));
                            }
                        raw3[dt3 + 1] = tr;
                    }
                    int f = mode == RECON_LINEAR ? 0 : (mode == RECON_WENOAO ? 1 : (raw3[0] | raw3[1] | raw3[2]));
                    if (f) tbits |= (uint8_t)(1u << X);
                    double v[4][2], d[4][2];
                    if (!f) {
                        for (int k = 0; k < nv; k++) {
                            double q[5];
                            for (int s = 0; s < 5; s++) q[s] = line[((size_t)(t - 2 + s - tlo) * nm + m) * 4 * nv + X * nv + k];
                            gauss_linear(q, v[k], d[k]);
                        }
                    } else {
                        double Lm[4][4], Rm[4][4], Uc[5][4];
                        eigvec(dim, c->gamma, Qs, 0.0, 1.0, Lm, Rm);
                        for (int s = 0; s < 5; s++) {
                            const double* src = line + ((size_t)(t - 2 + s - tlo) * nm + m) * 4 * nv + X * nv;
                            double tmp[4];
                            for (int k = 0; k < nv; k++) tmp[k] = src[k];
                            matvec(nv, Lm, tmp, Uc[s]);
                        }
                        double cv[4][2], cd[4][2];
                        for (int k = 0; k < nv; k++) {
                            double q[5];
                            for (int s = 0; s < 5; s++) q[s] = Uc[s][k];
                            gauss_ao(q, &g->ao, cv[k], cd[k]);
                        }
                        for (int gp = 0; gp < 2; gp++) {
                            double a[4], b[4], ra[4], rb[4];
                            for (int k = 0; k < nv; k++) { a[k] = cv[k][gp]; b[k] = cd[k][gp]; }
                            matvec(nv, Rm, a, ra); matvec(nv, Rm, b, rb);
                            for (int k = 0; k < nv; k++) { v[k][gp] = ra[k]; d[k][gp] = rb[k]; }
                        }
                    }
                    if (X <= 1)
                        for (int gp = 0; gp < 2; gp++) {
                            double Qg[4];
                            for (int k = 0; k < nv; k++) Qg[k] = v[k][gp];
                            if (nonphysical(dim, c->gamma, Qg))
                                for (int k = 0; k < nv; k++) {
                                    v[k][gp] = line[((size_t)(t - tlo) * nm + m) * 4 * nv + X * nv + k];
                                    d[k][gp] = 0.0;
                                }
                        }
                    for (int gp = 0; gp < 2; gp++)
                        for (int k = 0; k < nv; k++) {
                            if (X == 0) { gW[gp][0][k] = v[k][gp]; gW[gp][2][k] = d[k][gp] / ht; }
                            if (X == 1) { gW[gp][3][k] = v[k][gp]; gW[gp][5][k] = d[k][gp] / ht; }
                            if (X == 2) gW[gp][1][k] = v[k][gp];
                            if (X == 3) gW[gp][4][k] = v[k][gp];
                        }
                }
                if (fo && fo->tang) fo->tang[(size_t)t * nm + m] = tbits;
                if (fo && fo->tmargin) fo->tmargin[(size_t)t * nm + m] = tmg;
            }
            /* gas-kinetic flux at the Gauss points and the line average (weights 1/2) */
            int ngp = dim == 2 ? 2 : 1;
            double acc_dt[4] = {0, 0, 0, 0}, acc_h[4] = {0, 0, 0, 0};
            for (int gp = 0; gp < ngp; gp++) {
                double fd[4], fh[4];
                int st = gks_point_flux(c, gW[gp][0], gW[gp][1], gW[gp][2], gW[gp][3], gW[gp][4], gW[gp][5], dt, fd, fh);
                if (st != OR_OK) {
#pragma omp atomic write
                    status = st;
                }
                double wgt = dim == 2 ? 0.5 : 1.0;
                for (int k = 0; k < nv; k++) { acc_dt[k] += wgt * fd[k]; acc_h[k] += wgt * fh[k]; }
            }
            for (int k = 0; k < nv; k++) {
                size_t o = ((size_t)perm[k] * nt + t) * nm + m;
                Fdt[o] = acc_dt[k];
                Fhalf[o] = acc_h[k];
            }
        }
    }
#undef QL
    free(line); free(nflag);
    return status;
}

/* Time step, Sec. 3 preamble: dt = CFL min(h/(|U| + a), h^2/(4 nu)) with
 * h = min(dx, dy).  Reading: nu = mu/rho (the kinematic viscosity). */
static double cfl_dt(const grid* g, const double* Wp)
{
    const or_config* c = &g->c;
    if (c->fixed_dt > 0.0) return c->fixed_dt;
    double h = c->dim == 2 ? fmin(g->dx, g->dy) : g->dx;
    double gm1 = c->gamma - 1.0;
    double best = INFINITY;
    int jhi = c->dim == 2 ? c->ny : 1;
    for (int j = 0; j < jhi; j++)
        for (int i = 0; i < c->nx; i++) {
            double rho = Wp[pidx(g, 0, j, i)], ri = 1.0 / rho;
            double U = Wp[pidx(g, 1, j, i)] * ri;
            double V = c->dim == 2 ? Wp[pidx(g, 2, j, i)] * ri : 0.0;
            double q2 = U * U + V * V;
            double p = gm1 * (Wp[pidx(g, g->nv - 1, j, i)] - (0.5 * rho) * q2);
            double a = sqrt((c->gamma * p) * ri);
            double d = h / (sqrt(q2) + a);
            if (c->viscous) {
                double nu = c->mu * ri;
                double dv = (h * h) / (4.0 * nu);
                if (dv < d) d = dv;
            }
            if (d < best) best = d;
        }
    return c->cfl * best;
}

static int check_physical(const grid* g, const double* Wp)
{
    const or_config* c = &g->c;
    int jhi = c->dim == 2 ? c->ny : 1;
    for (int j = 0; j < jhi; j++)
        for (int i = 0; i < c->nx; i++) {
            double rho = Wp[pidx(g, 0, j, i)];
            double ke = 0.0;
            for (int k = 1; k <= c->dim; k++) ke += Wp[pidx(g, k, j, i)] * Wp[pidx(g, k, j, i)];
            double p = (c->gamma - 1.0) * (Wp[pidx(g, g->nv - 1, j, i)] - 0.5 * ke / rho);
            if (!(rho > 0.0) || !(p > 0.0) || !isfinite(rho) || !isfinite(p)) return OR_ENONPHYSICAL;
        }
    return OR_OK;
}

typedef struct {
    uint8_t* flags[2][2][2];   /* [stage][dir][0 normal, 1 tangential]; any may be NULL */
    double* margins[2][2][2];  /* decision margins, same layout; any may be NULL */
    double* wstar;             /* if not NULL: receives W* ([nv][ny][nx]) */
} step_flags;

/* One S2O4 step (Sec. 2.2): stage 1 with the dt and dt/2 fluxes at t_n gives
 * F^n, dF^n (Eqs. (17)-(18)) and W* (Eq. (19)); stage 2 at t* gives dF*, then
 * the fluxes of Eqs. (20)-(21) and W^{n+1} (Eq. (22)). */
static int s2o4_step(const grid* g, double* Wp, double t, double dt, step_flags* sf)
{
    const or_config* c = &g->c;
    int nx = c->nx, ny = c->ny, nv = g->nv, dim = c->dim;
    int ndir = dim;
    size_t nF[2];
    nF[0] = (size_t)nv * (dim == 2 ? ny : 1) * (nx + 1);
    nF[1] = dim == 2 ? (size_t)nv * nx * (ny + 1) : 0;
    size_t npad = (size_t)nv * g->NY * g->NX;
    double* Wn = (double*)malloc(sizeof(double) * npad);
    double* Ws = (double*)malloc(sizeof(double) * npad);
    double *Fdt[2] = {0, 0}, *Fh[2] = {0, 0}, *Fn[2] = {0, 0}, *dFn[2] = {0, 0};
    int st = OR_OK;
    for (int d = 0; d < ndir; d++) {
        Fdt[d] = (double*)malloc(sizeof(double) * nF[d]); Fh[d] = (double*)malloc(sizeof(double) * nF[d]);
        Fn[d] = (double*)malloc(sizeof(double) * nF[d]); dFn[d] = (double*)malloc(sizeof(double) * nF[d]);
        if (!Fdt[d] || !Fh[d] || !Fn[d] || !dFn[d]) st = OR_ENOMEM;
    }
    if (!Wn || !Ws) st = OR_ENOMEM;
    if (st != OR_OK) goto done;
    memcpy(Wn, Wp, sizeof(double) * npad);

    /* ---- stage 1 ---- */
    fill_ghosts(g, Wn, t);
    for (int d = 0; d < ndir && st == OR_OK; d++) {
        flag_out fo = {sf ? sf->flags[0][d][0] : NULL, sf ? sf->flags[0][d][1] : NULL,
                       sf ? sf->margins[0][d][0] : NULL, sf ? sf->margins[0][d][1] : NULL};
        st = sweep(g, Wn, d, dt, Fdt[d], Fh[d], &fo);
        for (size_t o = 0; o < nF[d]; o++) {
            Fn[d][o] = (4.0 * Fh[d][o] - Fdt[d][o]) / dt;                 /* Eq. (17) */
            dFn[d][o] = 4.0 * (Fdt[d][o] - 2.0 * Fh[d][o]) / (dt * dt);   /* Eq. (18) */
        }
    }
    if (st != OR_OK) goto done;
    memcpy(Ws, Wn, sizeof(double) * npad);
    for (int k = 0; k < nv; k++)
        for (int j = 0; j < (dim == 2 ? ny : 1); j++)
            for (int i = 0; i < nx; i++) {
                int jj = dim == 2 ? j : 0;
                double w = Wn[pidx(g, k, jj, i)];
                w = w - (Fh[0][((size_t)k * (dim == 2 ? ny : 1) + j) * (nx + 1) + i + 1]
                       - Fh[0][((size_t)k * (dim == 2 ? ny : 1) + j) * (nx + 1) + i]) / g->dx;   /* Eq. (19) */
                if (dim == 2)
                    w = w - (Fh[1][((size_t)k * nx + i) * (ny + 1) + j + 1]
                           - Fh[1][((size_t)k * nx + i) * (ny + 1) + j]) / g->dy;
                Ws[pidx(g, k, jj, i)] = w;
            }
    st = check_physical(g, Ws);
    if (st != OR_OK) goto done;
    if (sf && sf->wstar)
        for (int k = 0; k < nv; k++)
            for (int j = 0; j < (dim == 2 ? ny : 1); j++)
                for (int i = 0; i < nx; i++)
                    sf->wstar[((size_t)k * (dim == 2 ? ny : 1) + j) * nx + i] = Ws[pidx(g, k, dim == 2 ? j : 0, i)];

    /* ---- stage 2 (at t* = t^n + dt/2) ---- */
    fill_ghosts(g, Ws, t + 0.5 * dt);
    for (int d = 0; d < ndir && st == OR_OK; d++) {
        flag_out fo = {sf ? sf->flags[1][d][0] : NULL, sf ? sf->flags[1][d][1] : NULL,
                       sf ? sf->margins[1][d][0] : NULL, sf ? sf->margins[1][d][1] : NULL};
        st = sweep(g, Ws, d, dt, Fdt[d], Fh[d], &fo);
        for (size_t o = 0; o < nF[d]; o++) {
            double dFs = 4.0 * (Fdt[d][o] - 2.0 * Fh[d][o]) / (dt * dt);    /* Eq. (18) at t* */
            Fdt[d][o] = Fn[d][o] + dt / 6.0 * (dFn[d][o] + 2.0 * dFs);      /* Eqs. (20)-(21) */
        }
    }
    if (st != OR_OK) goto done;
    for (int k = 0; k < nv; k++)
        for (int j = 0; j < (dim == 2 ? ny : 1); j++)
            for (int i = 0; i < nx; i++) {
                int jj = dim == 2 ? j : 0;
                double w = Wn[pidx(g, k, jj, i)];
                w = w - dt / g->dx * (Fdt[0][((size_t)k * (dim == 2 ? ny : 1) + j) * (nx + 1) + i + 1]
                                    - Fdt[0][((size_t)k * (dim == 2 ? ny : 1) + j) * (nx + 1) + i]);   /* Eq. (22) */
                if (dim == 2)
                    w = w - dt / g->dy * (Fdt[1][((size_t)k * nx + i) * (ny + 1) + j + 1]
                                        - Fdt[1][((size_t)k * nx + i) * (ny + 1) + j]);
                Wp[pidx(g, k, jj, i)] = w;
            }
    st = check_physical(g, Wp);
done:
    free(Wn); free(Ws);
    for (int d = 0; d < 2; d++) { free(Fdt[d]); free(Fh[d]); free(Fn[d]); free(dFn[d]); }
    return st;
}

static void set_threads(const or_config* c)
{
#ifdef _OPENMP
    if (c->threads > 0) omp_set_num_threads(c->threads);
#else
    (void)c;
#endif
}

static void to_padded(const grid* g, const double* W, double* Wp)
{
    int nx = g->c.nx, ny = g->c.dim == 2 ? g->c.ny : 1;
    for (int k = 0; k < g->nv; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) Wp[pidx(g, k, j, i)] = W[((size_t)k * ny + j) * nx + i];
}
static void from_padded(const grid* g, const double* Wp, double* W)
{
    int nx = g->c.nx, ny = g->c.dim == 2 ? g->c.ny : 1;
    for (int k = 0; k < g->nv; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) W[((size_t)k * ny + j) * nx + i] = Wp[pidx(g, k, j, i)];
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (loaded through ctypes by the tests)                */
/* ------------------------------------------------------------------------ */

int or_threads_used(int requested)
{
#ifdef _OPENMP
    if (requested > 0) return requested;
    return omp_get_max_threads();
#else
    (void)requested;
    return 1;
#endif
}

/* Advance W ([nv][ny][nx], C order) from time *t to t_end by whole S2O4 steps,
 * at most max_steps.  The last step is shortened to land on t_end.
 * Reading: the run stops once t_end - t <= 1e-12 max(1, |t_end|). */
int or_run(const or_config* cfg, double* W, double* t, double t_end, int max_steps, int* steps_done, double* last_dt)
{
    grid g;
    int st = grid_setup(cfg, &g);
    if (st != OR_OK) return st;
    set_threads(cfg);
    size_t npad = (size_t)g.nv * g.NY * g.NX;
    double* Wp = (double*)calloc(npad, sizeof(double));
    if (!Wp) return OR_ENOMEM;
    to_padded(&g, W, Wp);
    int n = 0;
    double tol = 1e-12 * fmax(1.0, fabs(t_end));
    while (n < max_steps && t_end - *t > tol) {
        double dt = cfl_dt(&g, Wp);
        if (*t + dt > t_end) dt = t_end - *t;
        st = s2o4_step(&g, Wp, *t, dt, NULL);
        if (st != OR_OK) break;
        *t += dt;
        n++;
        if (last_dt) *last_dt = dt;
    }
    from_padded(&g, Wp, W);
    free(Wp);
    if (steps_done) *steps_done = n;
    return st;
}

/* One step from time t with flag capture.  dt <= 0 selects the CFL time step.
 * flags, margins: arrays of 8 pointers [stage][dir][normal/tangential], each may be NULL. */
int or_step_flags(const or_config* cfg, double* W, double t, double dt, double* dt_used, uint8_t** flags, double** margins,
                  double* wstar)
{
    grid g;
    int st = grid_setup(cfg, &g);
    if (st != OR_OK) return st;
    set_threads(cfg);
    size_t npad = (size_t)g.nv * g.NY * g.NX;
    double* Wp = (double*)calloc(npad, sizeof(double));
    if (!Wp) return OR_ENOMEM;
    to_padded(&g, W, Wp);
    if (dt <= 0.0) dt = cfl_dt(&g, Wp);
    step_flags sf;
    for (int s = 0; s < 2; s++) for (int d = 0; d < 2; d++) for (int k = 0; k < 2; k++) {
        sf.flags[s][d][k] = flags ? flags[(s * 2 + d) * 2 + k] : NULL;
        sf.margins[s][d][k] = margins ? margins[(s * 2 + d) * 2 + k] : NULL;
    }
    sf.wstar = wstar;
    st = s2o4_step(&g, Wp, t, dt, &sf);
    from_padded(&g, Wp, W);
    free(Wp);
    if (dt_used) *dt_used = dt;
    return st;
}

/* CFL time step of a state (same rule as or_run). */
double or_cfl_dt(const or_config* cfg, const double* W)
{
    grid g;
    if (grid_setup(cfg, &g) != OR_OK) return -1.0;
    size_t npad = (size_t)g.nv * g.NY * g.NX;
    double* Wp = (double*)calloc(npad, sizeof(double));
    to_padded(&g, W, Wp);
    double dt = cfl_dt(&g, Wp);
    free(Wp);
    return dt;
}

/* ---- pieces exposed for the unit tests ---- */

void or_moments(int dim, double K, double U, double V, double lam, double* u, double* up, double* un, double* v, double* x)
{
    mom m;
    moments(dim, K, 1.0, U, V, lam, &m);
    for (int n = 0; n < NMOM; n++) { u[n] = m.u[n]; up[n] = m.up[n]; un[n] = m.un[n]; v[n] = m.v[n]; }
    for (int k = 0; k < 4; k++) x[k] = m.x[k];
}

double or_dof_K(int dim, double gam) { return dof_K(dim, gam); }

/* micro-slope a with <a> = dW at state W */
int or_micro_slope(int dim, double gam, const double* W, const double* dW, double* a)
{
    double rho, U, V, lam, p;
    to_prim(dim, gam, W, &rho, &U, &V, &lam, &p);
    if (!(rho > 0.0) || !(p > 0.0)) return OR_ENONPHYSICAL;
    mom m;
    moments(dim, dof_K(dim, gam), rho, U, V, lam, &m);
    micro_slope(dim, &m, dW, a);
    return OR_OK;
}

int or_time_slope(int dim, double gam, const double* W, const double* a1, const double* a2, double* A)
{
    double rho, U, V, lam, p;
    to_prim(dim, gam, W, &rho, &U, &V, &lam, &p);
    if (!(rho > 0.0) || !(p > 0.0)) return OR_ENONPHYSICAL;
    mom m;
    moments(dim, dof_K(dim, gam), rho, U, V, lam, &m);
    double z[4] = {0, 0, 0, 0};
    time_slope(dim, &m, a1, dim == 2 ? a2 : z, A);
    return OR_OK;
}

/* int psi (a . psi) g over the full line (half=0) or a half line (+1 / -1) */
int or_slope_moment(int dim, double gam, const double* W, const double* a, int half, double* out)
{
    double rho, U, V, lam, p;
    to_prim(dim, gam, W, &rho, &U, &V, &lam, &p);
    mom m;
    moments(dim, dof_K(dim, gam), rho, U, V, lam, &m);
    poly s;
    slope_poly(dim, a, &s);
    integ_psi(dim, &s, &m, half, out);
    return OR_OK;
}

int or_point_flux(const or_config* cfg, const double* Wl, const double* Wlx, const double* Wly,
                  const double* Wr, const double* Wrx, const double* Wry, double dt, double* Fdt, double* Fhalf)
{
    return gks_point_flux(cfg, Wl, Wlx, Wly, Wr, Wrx, Wry, dt, Fdt, Fhalf);
}

int or_indicator(const double* q5, double Z1) { return indicator_raw(q5, Z1, 0.0); }
double or_zeta1_scaled(int mode, double h) { return zeta1_scaled(mode, h); }

void or_linear_face(const double* q5, double inv12h, int side, double* val, double* der)
{
    if (side > 0) linear_left(q5, inv12h, val, der);
    else linear_right(q5, inv12h, val, der);
}

void or_ao_betas(const double* q5, double* b) { ao_betas(q5, b); }

void or_ao_face_scalar(const double* q5, double ghi, double glo, double eps, int side, double* val, double* der)
{
    ao_consts k; double wb[4], pv[4], pd[4];
    ao_setup(ghi, glo, eps, &k);
    ao_weights(q5, &k, wb);
    face_polys(q5, side, pv, pd);
    *val = ao_combine(wb, &k, pv);
    *der = ao_combine(wb, &k, pd);
}

void or_gauss_scalar(const double* q5, int use_ao, double ghi, double glo, double eps, double* v2, double* d2)
{
    ao_consts k;
    ao_setup(ghi, glo, eps, &k);
    if (use_ao) gauss_ao(q5, &k, v2, d2);
    else gauss_linear(q5, v2, d2);
}

void or_eigvec(int dim, double gam, const double* Q, double nx, double ny, double* L16, double* R16)
{
    double L[4][4], R[4][4];
    memset(L, 0, sizeof L); memset(R, 0, sizeof R);
    eigvec(dim, gam, Q, nx, ny, L, R);
    for (int i = 0; i < 4; i++) for (int j = 0; j < 4; j++) { L16[i * 4 + j] = L[i][j]; R16[i * 4 + j] = R[i][j]; }
}

void or_weno_ao_face(int dim, double gam, double ghi, double glo, double eps, const double* Qw20, const double* Qs,
                     double nx, double ny, int side, double* val, double* der)
{
    ao_consts k; double Qw[5][4];
    ao_setup(ghi, glo, eps, &k);
    for (int j = 0; j < 5; j++) for (int c = 0; c < 4; c++) Qw[j][c] = Qw20[j * 4 + c];
    weno_ao_face(dim, gam, &k, Qw, Qs, nx, ny, side, val, der);
}

/* Ghost-filled padded state (for the boundary-condition tests). */
int or_fill_ghosts(const or_config* cfg, const double* W, double t, double* Wpad)
{
    grid g;
    int st = grid_setup(cfg, &g);
    if (st != OR_OK) return st;
    size_t npad = (size_t)g.nv * g.NY * g.NX;
    memset(Wpad, 0, sizeof(double) * npad);
    to_padded(&g, W, Wpad);
    fill_ghosts(&g, Wpad, t);
    return OR_OK;
}

int or_ghost_layers(void) { return NG; }
