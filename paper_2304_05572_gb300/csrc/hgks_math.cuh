// hgks_math.cuh -- device arithmetic of the hybrid WENO-AO gas-kinetic scheme
// (arXiv 2304.05572) for sm_103a, FP64.
//
// Two kinds of code live here:
//  * decision-carrying reconstruction (troubled-cell indicator, normal-direction
//    linear and characteristic WENO-AO reconstruction, positivity test).  Its
//    outputs feed later troubled-cell decisions, so it is evaluated in one fixed
//    IEEE order with no FMA contraction: every operation goes through the
//    `ex` wrapper, whose operators map to __dadd_rn / __dmul_rn / __ddiv_rn and
//    whose fma is explicit.  Any implementation that evaluates the same formulas
//    in the same order (as written below) takes bit-identical decisions.
//  * the Gauss-point (tangential) reconstruction and the gas-kinetic flux, which
//    only feed the update and are written for few FP64 instructions: closed-form
//    micro-slope solves, one erfc and one exp per side, exp(-dt/(2 tau)) squared
//    for exp(-dt/tau), and the S2O4 flux combinations formed on scalar
//    coefficients before the moment vectors are combined.
#pragma once

#include <cstdint>

namespace hgks {

// ---------------------------------------------------------------- exact-order FP64
struct ex {
    double v;
    __device__ __forceinline__ ex() {}
    __device__ __forceinline__ ex(double x) : v(x) {}
};
__device__ __forceinline__ ex operator+(ex a, ex b) { return ex(__dadd_rn(a.v, b.v)); }
__device__ __forceinline__ ex operator-(ex a, ex b) { return ex(__dsub_rn(a.v, b.v)); }
__device__ __forceinline__ ex operator*(ex a, ex b) { return ex(__dmul_rn(a.v, b.v)); }
__device__ __forceinline__ ex operator/(ex a, ex b) { return ex(__ddiv_rn(a.v, b.v)); }
__device__ __forceinline__ ex operator-(ex a) { return ex(-a.v); }
__device__ __forceinline__ ex xfma(ex a, ex b, ex c) { return ex(__fma_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ ex xabs(ex a) { return ex(fabs(a.v)); }
__device__ __forceinline__ ex xsqrt(ex a) { return ex(__dsqrt_rn(a.v)); }

// Troubled-cell indicator, Sec. 2.3.1 Steps 1-3, on the window q[0..4] = Q_{i-2..i+2}
// (cell units).  Step 1: |D| <= Z1 with D = (4Q_{i-2}+Q_{i-1}) + (4Q_{i+2}+Q_{i+1}) - 10 Q_i
// and Z1 = 17 zeta1 dx^2 (Eq. (24): abar2 = D/34).  Step 2: xbar = -abar1/(2 abar2) with
// abar1 = -N/10, N = (2Q_{i-2}+Q_{i-1}) - (2Q_{i+2}+Q_{i+1}); inside iff |xbar| <= 5/2.
// Step 3: xhat from the conservative 3-cell quadratic; non-troubled iff |xbar - xhat| <= 1/4.
__device__ __forceinline__ int indicator_raw(const double* q, double Z1)
{
    ex q0(q[0]), q1(q[1]), q2(q[2]), q3(q[3]), q4(q[4]);
    ex D = xfma(ex(-10.0), q2, xfma(ex(4.0), q0, q1) + xfma(ex(4.0), q4, q3));
    if (fabs(D.v) <= Z1) return 0;
    ex N = xfma(ex(2.0), q0, q1) - xfma(ex(2.0), q4, q3);
    ex a1 = -(N / ex(10.0));
    ex a2 = D / ex(34.0);
    ex xbar = (-a1) / (ex(2.0) * a2);
    if (!(fabs(xbar.v) <= 2.5)) return 0;
    ex ah1 = ex(0.5) * (q3 - q1);
    ex ah2 = ex(0.5) * ((q1 + q3) - ex(2.0) * q2);
    ex den = ex(2.0) * ah2 + ex(ah2.v == 0.0 ? 1e-30 : 0.0);
    ex xhat = (-ah1) / den;
    if (fabs((xbar - xhat).v) <= 0.25) return 0;
    return 1;
}

// Step 5, Eqs. (26)-(27): value and derivative at x_{i+1/2} from cell i's window.
__device__ __forceinline__ void linear_left(const double* q, double inv12h, double& val, double& der)
{
    ex t = xfma(ex(-13.0), ex(q[1]), ex(2.0) * ex(q[0]));
    t = xfma(ex(47.0), ex(q[2]), t);
    t = xfma(ex(27.0), ex(q[3]), t);
    t = xfma(ex(-3.0), ex(q[4]), t);
    val = (t * ex(1.0 / 60.0)).v;
    ex s = xfma(ex(-15.0), ex(q[2]), ex(q[1]));
    s = xfma(ex(15.0), ex(q[3]), s);
    s = s - ex(q[4]);
    der = (s * ex(inv12h)).v;
}

// Eqs. (28)-(29): value and derivative at x_{i-1/2}, the mirror image of linear_left.
__device__ __forceinline__ void linear_right(const double* q, double inv12h, double& val, double& der)
{
    ex t = xfma(ex(-13.0), ex(q[3]), ex(2.0) * ex(q[4]));
    t = xfma(ex(47.0), ex(q[2]), t);
    t = xfma(ex(27.0), ex(q[1]), t);
    t = xfma(ex(-3.0), ex(q[0]), t);
    val = (t * ex(1.0 / 60.0)).v;
    ex s = xfma(ex(-15.0), ex(q[2]), ex(q[3]));
    s = xfma(ex(15.0), ex(q[1]), s);
    s = s - ex(q[0]);
    der = (-(s * ex(inv12h))).v;
}

// WENO-AO constants: linear weights of Eq. (35) and derived ratios.
struct AOConst {
    double g[4];      // gamma_0..2 (sub-stencils, S1 central), gamma_3 (large stencil)
    double g3inv;     // 1/gamma_3
    double gr[3];     // gamma_k / gamma_3
    double eps;
};

// Smoothness indicators of Eq. (39) in cell units (same evaluation order as the decisions need).
__device__ __forceinline__ void ao_betas(const ex* q, ex* b)
{
    ex s0 = (q[0] - ex(2.0) * q[1]) + q[2], t0 = (q[0] - ex(4.0) * q[1]) + ex(3.0) * q[2];
    ex s1 = (q[1] - ex(2.0) * q[2]) + q[3], t1 = q[1] - q[3];
    ex s2 = (q[2] - ex(2.0) * q[3]) + q[4], t2 = (ex(3.0) * q[2] - ex(4.0) * q[3]) + q[4];
    b[0] = ex(13.0 / 12.0) * (s0 * s0) + ex(0.25) * (t0 * t0);
    b[1] = ex(13.0 / 12.0) * (s1 * s1) + ex(0.25) * (t1 * t1);
    b[2] = ex(13.0 / 12.0) * (s2 * s2) + ex(0.25) * (t2 * t2);
    ex c1 = ex(17.0 / 24.0) * (q[3] - q[1]) - ex(5.0 / 48.0) * (q[4] - q[0]);
    ex c2 = ((ex(0.75) * (q[1] + q[3]) - ex(0.0625) * (q[0] + q[4])) - ex(1.375) * q[2]);
    ex c3 = ex(1.0 / 6.0) * (q[1] - q[3]) - ex(1.0 / 12.0) * (q[0] - q[4]);
    ex c4 = ((ex(1.0 / 24.0) * (q[0] + q[4]) - ex(1.0 / 6.0) * (q[1] + q[3])) + ex(0.25) * q[2]);
    b[3] = ((((c1 * c1 + ex(0.5) * (c1 * c3)) + ex(13.0 / 3.0) * (c2 * c2)) + ex(21.0 / 5.0) * (c2 * c4))
            + ex(3129.0 / 80.0) * (c3 * c3)) + ex(87617.0 / 140.0) * (c4 * c4);
}

// Normalised nonlinear weights, Eqs. (37), (38), (40), with the ratio delta/(beta_k + eps) squared.
__device__ __forceinline__ void ao_weights(const ex* q, const AOConst& k, ex* wb)
{
    ex b[4], w[4];
    ao_betas(q, b);
    ex d = ((xabs(b[3] - b[0]) + xabs(b[3] - b[1])) + xabs(b[3] - b[2])) * ex(1.0 / 3.0);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        ex r = d / (b[j] + ex(k.eps));
        w[j] = ex(k.g[j]) * (ex(1.0) + r * r);
    }
    ex inv = ex(1.0) / (((w[0] + w[1]) + w[2]) + w[3]);
#pragma unroll
    for (int j = 0; j < 4; j++) wb[j] = w[j] * inv;
}

// AO(5,3) polynomial of Eq. (41) applied to point values p[0..3].
__device__ __forceinline__ ex ao_combine(const ex* wb, const AOConst& k, const ex* p)
{
    return wb[3] * (p[3] * ex(k.g3inv) - ((ex(k.gr[0]) * p[0] + ex(k.gr[1]) * p[1]) + ex(k.gr[2]) * p[2]))
         + ((wb[0] * p[0] + wb[1] * p[1]) + wb[2] * p[2]);
}

// Face values / cell-unit derivatives of the three quadratics (Eqs. (32), (43), with the
// p_2(x_{i+1/2}) coefficient corrected to -1/6) and of the quartic (Eqs. (36), (44)).
__device__ __forceinline__ void face_polys(const ex* q, int side, ex* pv, ex* pd)
{
    if (side > 0) {
        pv[0] = ((ex(2.0) * q[0] - ex(7.0) * q[1]) + ex(11.0) * q[2]) * ex(1.0 / 6.0);
        pv[1] = ((-q[1] + ex(5.0) * q[2]) + ex(2.0) * q[3]) * ex(1.0 / 6.0);
        pv[2] = ((ex(2.0) * q[2] + ex(5.0) * q[3]) - q[4]) * ex(1.0 / 6.0);
        pv[3] = ((((ex(2.0) * q[0] - ex(13.0) * q[1]) + ex(47.0) * q[2]) + ex(27.0) * q[3]) - ex(3.0) * q[4]) * ex(1.0 / 60.0);
        pd[0] = (q[0] - ex(3.0) * q[1]) + ex(2.0) * q[2];
        pd[1] = q[3] - q[2];
        pd[2] = q[3] - q[2];
        pd[3] = (((q[1] - ex(15.0) * q[2]) + ex(15.0) * q[3]) - q[4]) * ex(1.0 / 12.0);
    } else {
        pv[0] = ((-q[0] + ex(5.0) * q[1]) + ex(2.0) * q[2]) * ex(1.0 / 6.0);
        pv[1] = ((ex(2.0) * q[1] + ex(5.0) * q[2]) - q[3]) * ex(1.0 / 6.0);
        pv[2] = ((ex(11.0) * q[2] - ex(7.0) * q[3]) + ex(2.0) * q[4]) * ex(1.0 / 6.0);
        pv[3] = ((((-ex(3.0) * q[0] + ex(27.0) * q[1]) + ex(47.0) * q[2]) - ex(13.0) * q[3]) + ex(2.0) * q[4]) * ex(1.0 / 60.0);
        pd[0] = q[2] - q[1];
        pd[1] = q[2] - q[1];
        pd[2] = (-ex(2.0) * q[2] + ex(3.0) * q[3]) - q[4];
        pd[3] = (((q[0] - ex(15.0) * q[1]) + ex(15.0) * q[2]) - q[3]) * ex(1.0 / 12.0);
    }
}

// Left (L = R^{-1}, rows) and right (R, columns) eigenvectors of nx dF/dQ + ny dG/dQ at Q.
template <int NV>
__device__ __forceinline__ void eigvec(double gam, const ex* Q, double nxd, double nyd, ex (*L)[NV], ex (*R)[NV])
{
    ex gm1 = ex(gam) - ex(1.0);
    ex rho = Q[0], ri = ex(1.0) / rho;
    ex U = Q[1] * ri;
    if constexpr (NV == 4) {
        ex nx(nxd), ny(nyd);
        ex V = Q[2] * ri;
        ex q2 = U * U + V * V;
        ex p = gm1 * (Q[3] - (ex(0.5) * rho) * q2);
        ex c2 = (ex(gam) * p) * ri, c = xsqrt(c2), ci = ex(1.0) / c;
        ex H = (Q[3] + p) * ri;
        ex un = U * nx + V * ny, ut = V * nx - U * ny;
        ex b1 = gm1 / c2, b2 = (ex(0.5) * b1) * q2;
        R[0][0] = ex(1.0);    R[0][1] = ex(1.0);       R[0][2] = ex(0.0); R[0][3] = ex(1.0);
        R[1][0] = U - c * nx; R[1][1] = U;             R[1][2] = -ny;     R[1][3] = U + c * nx;
        R[2][0] = V - c * ny; R[2][1] = V;             R[2][2] = nx;      R[2][3] = V + c * ny;
        R[3][0] = H - un * c; R[3][1] = ex(0.5) * q2;  R[3][2] = ut;      R[3][3] = H + un * c;
        L[0][0] = ex(0.5) * (b2 + un * ci); L[0][1] = -(ex(0.5) * (b1 * U + nx * ci)); L[0][2] = -(ex(0.5) * (b1 * V + ny * ci)); L[0][3] = ex(0.5) * b1;
        L[1][0] = ex(1.0) - b2;             L[1][1] = b1 * U;                          L[1][2] = b1 * V;                          L[1][3] = -b1;
        L[2][0] = -ut;                      L[2][1] = -ny;                             L[2][2] = nx;                              L[2][3] = ex(0.0);
        L[3][0] = ex(0.5) * (b2 - un * ci); L[3][1] = -(ex(0.5) * (b1 * U - nx * ci)); L[3][2] = -(ex(0.5) * (b1 * V - ny * ci)); L[3][3] = ex(0.5) * b1;
    } else {
        ex q2 = U * U;
        ex p = gm1 * (Q[2] - (ex(0.5) * rho) * q2);
        ex c2 = (ex(gam) * p) * ri, c = xsqrt(c2), ci = ex(1.0) / c;
        ex H = (Q[2] + p) * ri;
        ex b1 = gm1 / c2, b2 = (ex(0.5) * b1) * q2;
        R[0][0] = ex(1.0);    R[0][1] = ex(1.0);      R[0][2] = ex(1.0);
        R[1][0] = U - c;      R[1][1] = U;            R[1][2] = U + c;
        R[2][0] = H - U * c;  R[2][1] = ex(0.5) * q2; R[2][2] = H + U * c;
        L[0][0] = ex(0.5) * (b2 + U * ci); L[0][1] = -(ex(0.5) * (b1 * U + ci)); L[0][2] = ex(0.5) * b1;
        L[1][0] = ex(1.0) - b2;            L[1][1] = b1 * U;                     L[1][2] = -b1;
        L[2][0] = ex(0.5) * (b2 - U * ci); L[2][1] = -(ex(0.5) * (b1 * U - ci)); L[2][2] = ex(0.5) * b1;
    }
}

// y = M x with the summation order ((m0 x0 + m1 x1) + m2 x2) + m3 x3.
template <int NV>
__device__ __forceinline__ void matvec(const ex (*M)[NV], const ex* x, ex* y)
{
#pragma unroll
    for (int r = 0; r < NV; r++) {
        ex s = M[r][0] * x[0] + M[r][1] * x[1];
#pragma unroll
        for (int c = 2; c < NV; c++) s = s + M[r][c] * x[c];
        y[r] = s;
    }
}

// Characteristic WENO-AO at the face of side (+1: x_{i+1/2}, -1: x_{i-1/2}) of the cell whose
// window (cells i-2..i+2) is Qw[j][comp], projected with the eigenvectors at Qs in the local
// normal direction.  Returns conservative value and cell-unit derivative.
template <int NV>
__device__ __forceinline__ void weno_ao_face(double gam, const AOConst& k, const double (*Qw)[NV], const double* Qs,
                                             int side, double* val, double* der)
{
    ex L[NV][NV], R[NV][NV], Uc[5][NV], uv[NV], ud[NV], qs[NV];
#pragma unroll
    for (int c = 0; c < NV; c++) qs[c] = ex(Qs[c]);
    eigvec<NV>(gam, qs, 1.0, 0.0, L, R);
#pragma unroll
    for (int j = 0; j < 5; j++) {
        ex x[NV];
#pragma unroll
        for (int c = 0; c < NV; c++) x[c] = ex(Qw[j][c]);
        matvec<NV>(L, x, Uc[j]);
    }
#pragma unroll
    for (int c = 0; c < NV; c++) {
        ex q[5], wb[4], pv[4], pd[4];
#pragma unroll
        for (int j = 0; j < 5; j++) q[j] = Uc[j][c];
        ao_weights(q, k, wb);
        face_polys(q, side, pv, pd);
        uv[c] = ao_combine(wb, k, pv);
        ud[c] = ao_combine(wb, k, pd);
    }
    ex v[NV], d[NV];
    matvec<NV>(R, uv, v);
    matvec<NV>(R, ud, d);
#pragma unroll
    for (int c = 0; c < NV; c++) { val[c] = v[c].v; der[c] = d[c].v; }
}

// Reading (no safeguard is printed): rho <= 0 or p <= 0 after reconstruction -> first order.
// ke = 0.5 (m_x^2 + m_y^2), p = (gamma-1)(E - ke/rho), in this order.
template <int NV>
__device__ __forceinline__ bool nonphysical(double gam, const double* Q)
{
    ex ke;
    if constexpr (NV == 4) ke = ex(0.5) * (ex(Q[1]) * ex(Q[1]) + ex(Q[2]) * ex(Q[2]));
    else ke = ex(0.5) * (ex(Q[1]) * ex(Q[1]));
    ex p = (ex(gam) - ex(1.0)) * (ex(Q[NV - 1]) - ke / ex(Q[0]));
    return !(Q[0] > 0.0) || !(p.v > 0.0);
}

// ---------------------------------------------------------------- Gauss-point reconstruction
// Coefficients (cell units) of the three quadratics and the quartic through the averages of
// cells i-2..i+2, evaluated at xi = +-1/(2 sqrt 3): values V and derivatives D, at +g (P) and -g (M).
struct GaussCoef { double VP[4][5], DP[4][5], VM[4][5], DM[4][5]; };
__device__ __constant__ GaussCoef c_gauss = {
    {{1.44337567297406433e-01, -5.77350269189625731e-01, 1.43301270189221941e+00, 0.0, 0.0},
     {0.0, -1.44337567297406433e-01, 1.00000000000000000e+00, 1.44337567297406433e-01, 0.0},
     {0.0, 0.0, 5.66987298107780702e-01, 5.77350269189625731e-01, -1.44337567297406433e-01},
     {2.78341566041253249e-02, -1.99542917542694126e-01, 9.98611111111111116e-01, 2.01394769394545980e-01, -2.82971195670882886e-02}},
    {{7.88675134594812866e-01, -2.57735026918962573e+00, 1.78867513459481287e+00, 0.0, 0.0},
     {0.0, -2.11324865405187107e-01, -5.77350269189625731e-01, 7.88675134594812866e-01, 0.0},
     {0.0, 0.0, -1.21132486540518713e+00, 1.42264973081037427e+00, -2.11324865405187107e-01},
     {5.12583183783541230e-02, -2.49691472251936941e-01, -7.69800358919501049e-01, 1.08364186108139648e+00, -1.15408348288312548e-01}},
    {{-1.44337567297406433e-01, 5.77350269189625731e-01, 5.66987298107780702e-01, 0.0, 0.0},
     {0.0, 1.44337567297406433e-01, 1.00000000000000000e+00, -1.44337567297406433e-01, 0.0},
     {0.0, 0.0, 1.43301270189221941e+00, -5.77350269189625731e-01, 1.44337567297406433e-01},
     {-2.82971195670882886e-02, 2.01394769394545980e-01, 9.98611111111111116e-01, -1.99542917542694126e-01, 2.78341566041253249e-02}},
    {{2.11324865405187107e-01, -1.42264973081037427e+00, 1.21132486540518713e+00, 0.0, 0.0},
     {0.0, -7.88675134594812866e-01, 5.77350269189625731e-01, 2.11324865405187107e-01, 0.0},
     {0.0, 0.0, -1.78867513459481287e+00, 2.57735026918962573e+00, -7.88675134594812866e-01},
     {1.15408348288312548e-01, -1.08364186108139648e+00, 7.69800358919501049e-01, 2.49691472251936941e-01, -5.12583183783541230e-02}},
};

// quartic at the two Gauss points: v[0] at -g, v[1] at +g (and cell-unit derivatives)
__device__ __forceinline__ void gauss_linear(const double* q, double* v, double* d)
{
    const double* vm = c_gauss.VM[3]; const double* vp = c_gauss.VP[3];
    const double* dm = c_gauss.DM[3]; const double* dp = c_gauss.DP[3];
    double a = vm[2] * q[2], b = vp[2] * q[2], e = dm[2] * q[2], f = dp[2] * q[2];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        if (j == 2) continue;
        a = fma(vm[j], q[j], a); b = fma(vp[j], q[j], b);
        e = fma(dm[j], q[j], e); f = fma(dp[j], q[j], f);
    }
    v[0] = a; v[1] = b; d[0] = e; d[1] = f;
}

__device__ __forceinline__ void gauss_ao(const ex* q, const AOConst& k, double* v, double* d)
{
    ex wb[4];
    ao_weights(q, k, wb);
    double w3 = wb[3].v * k.g3inv;
    // weight of each polynomial in the AO combination (Eq. (41)):
    //   quartic: wb3/g3;   quadratic s: wb_s - wb3 g_s/g3
    double ws[4] = {wb[0].v - wb[3].v * k.gr[0], wb[1].v - wb[3].v * k.gr[1], wb[2].v - wb[3].v * k.gr[2], w3};
    double a = 0.0, b = 0.0, e = 0.0, f = 0.0;
#pragma unroll
    for (int s = 0; s < 4; s++) {
        double pa = 0.0, pb = 0.0, pe = 0.0, pf = 0.0;
#pragma unroll
        for (int j = 0; j < 5; j++) {
            if (c_gauss.VM[s][j] == 0.0 && c_gauss.DM[s][j] == 0.0) continue;
            pa = fma(c_gauss.VM[s][j], q[j].v, pa); pb = fma(c_gauss.VP[s][j], q[j].v, pb);
            pe = fma(c_gauss.DM[s][j], q[j].v, pe); pf = fma(c_gauss.DP[s][j], q[j].v, pf);
        }
        a = fma(ws[s], pa, a); b = fma(ws[s], pb, b); e = fma(ws[s], pe, e); f = fma(ws[s], pf, f);
    }
    v[0] = a; v[1] = b; d[0] = e; d[1] = f;
}

// ---------------------------------------------------------------- gas-kinetic flux
// Normalised moments of a Maxwellian: u^n (full or one half line), v^m (full), xi^2, xi^4.
template <int DIM>
struct Mom {
    double u[8];
    double v[DIM == 2 ? 7 : 1];
    double x2, x4;
};

// T(n, m) = <u^n v^m (a.psi)>; Tx = <u^n v^m xi^2 (a.psi)>
template <int DIM, int N, int M>
__device__ __forceinline__ double Tm(const double* a, const Mom<DIM>& m)
{
    if constexpr (DIM == 2) {
        double um = m.u[N] * m.v[M];
        double s = a[0] * um;
        s = fma(a[1], m.u[N + 1] * m.v[M], s);
        s = fma(a[2], m.u[N] * m.v[M + 1], s);
        double e = fma(m.u[N + 2], m.v[M], fma(m.u[N], m.v[M + 2], um * m.x2));
        return fma(0.5 * a[3], e, s);
    } else {
        double s = a[0] * m.u[N];
        s = fma(a[1], m.u[N + 1], s);
        double e = fma(m.u[N], m.x2, m.u[N + 2]);
        return fma(0.5 * a[2], e, s);
    }
}
template <int DIM, int N, int M>
__device__ __forceinline__ double Tx(const double* a, const Mom<DIM>& m)
{
    if constexpr (DIM == 2) {
        double um = m.u[N] * m.v[M];
        double s = a[0] * um;
        s = fma(a[1], m.u[N + 1] * m.v[M], s);
        s = fma(a[2], m.u[N] * m.v[M + 1], s);
        double e = fma(m.x2, fma(m.u[N + 2], m.v[M], m.u[N] * m.v[M + 2]), um * m.x4);
        return fma(0.5 * a[3], e, s * m.x2);
    } else {
        double s = fma(a[1], m.u[N + 1], a[0] * m.u[N]);
        double e = fma(m.x2, m.u[N + 2], m.u[N] * m.x4);
        return fma(0.5 * a[2], e, s * m.x2);
    }
}
// G(a; n, m) = <u^n v^m psi (a.psi)> (NV components)
template <int DIM, int N, int M>
__device__ __forceinline__ void Gm(const double* a, const Mom<DIM>& m, double* out)
{
    if constexpr (DIM == 2) {
        out[0] = Tm<2, N, M>(a, m);
        out[1] = Tm<2, N + 1, M>(a, m);
        out[2] = Tm<2, N, M + 1>(a, m);
        out[3] = 0.5 * (Tm<2, N + 2, M>(a, m) + Tm<2, N, M + 2>(a, m) + Tx<2, N, M>(a, m));
    } else {
        out[0] = Tm<1, N, 0>(a, m);
        out[1] = Tm<1, N + 1, 0>(a, m);
        out[2] = 0.5 * (Tm<1, N + 2, 0>(a, m) + Tx<1, N, 0>(a, m));
    }
}

// Micro-slope a with <a> = b (b = dW / rho), closed form of the moment system of Eq. (8).
template <int DIM>
__device__ __forceinline__ void slope_solve(const double* b, double U, double V, double lam, double K, double* a)
{
    if constexpr (DIM == 2) {
        double q = fma(U, U, fma(V, V, (K + 2.0) / (2.0 * lam)));
        double R4 = fma(-q, b[0], 2.0 * b[3]);
        double R3 = fma(-V, b[0], b[2]);
        double R2 = fma(-U, b[0], b[1]);
        double a4 = (4.0 * lam * lam / (K + 2.0)) * fma(-2.0 * V, R3, fma(-2.0 * U, R2, R4));
        double a3 = fma(-V, a4, 2.0 * lam * R3);
        double a2 = fma(-U, a4, 2.0 * lam * R2);
        a[3] = a4; a[2] = a3; a[1] = a2;
        a[0] = fma(-0.5 * a4, q, fma(-V, a3, fma(-U, a2, b[0])));
    } else {
        double q = fma(U, U, (K + 1.0) / (2.0 * lam));
        double R3 = fma(-q, b[0], 2.0 * b[2]);
        double R2 = fma(-U, b[0], b[1]);
        double a3 = (4.0 * lam * lam / (K + 1.0)) * fma(-2.0 * U, R2, R3);
        double a2 = fma(-U, a3, 2.0 * lam * R2);
        a[2] = a3; a[1] = a2;
        a[0] = fma(-0.5 * a3, q, fma(-U, a2, b[0]));
    }
}

struct FluxConst {
    double gamma, K, mu, c1, c2;
    int viscous, tau_zero;
};

// Primitive state; returns false if rho <= 0 or p <= 0.
template <int DIM>
__device__ __forceinline__ bool prim(const double* W, double gam, double& rho, double& U, double& V, double& lam, double& p)
{
    rho = W[0];
    double ri = 1.0 / rho;
    U = W[1] * ri;
    V = DIM == 2 ? W[2] * ri : 0.0;
    double ke = DIM == 2 ? fma(U, W[1], V * W[2]) : U * W[1];
    p = (gam - 1.0) * fma(-0.5, ke, W[DIM + 1]);
    lam = 0.5 * rho / p;
    return rho > 0.0 && p > 0.0;
}

template <int DIM>
__device__ __forceinline__ void full_moments(double U, double V, double lam, double K, Mom<DIM>& m)
{
    double h = 0.5 / lam;
    m.u[0] = 1.0; m.u[1] = U;
#pragma unroll
    for (int n = 0; n < 6; n++) m.u[n + 2] = fma(U, m.u[n + 1], (n + 1) * h * m.u[n]);
    if constexpr (DIM == 2) {
        m.v[0] = 1.0; m.v[1] = V;
#pragma unroll
        for (int n = 0; n < 5; n++) m.v[n + 2] = fma(V, m.v[n + 1], (n + 1) * h * m.v[n]);
    } else {
        m.v[0] = 1.0;
    }
    m.x2 = K * h;
    m.x4 = m.x2 * (K + 2.0) * h;
}

// Half-line moments: sign > 0 for u > 0 (left state), < 0 for u < 0 (right state).
template <int DIM>
__device__ __forceinline__ void half_moments(double U, double V, double lam, double K, int sign, Mom<DIM>& m)
{
    double h = 0.5 / lam;
    double sl = sqrt(lam);
    double x = sl * U;
    double e = 0.5 * exp(-x * x) * (0.56418958354775628695 / sl);   // exp(-lam U^2) / (2 sqrt(pi lam))
    if (sign > 0) { m.u[0] = 0.5 * erfc(-x); m.u[1] = fma(U, m.u[0], e); }
    else          { m.u[0] = 0.5 * erfc(x);  m.u[1] = fma(U, m.u[0], -e); }
#pragma unroll
    for (int n = 0; n < 6; n++) m.u[n + 2] = fma(U, m.u[n + 1], (n + 1) * h * m.u[n]);
    if constexpr (DIM == 2) {
        m.v[0] = 1.0; m.v[1] = V;
#pragma unroll
        for (int n = 0; n < 5; n++) m.v[n + 2] = fma(V, m.v[n + 1], (n + 1) * h * m.v[n]);
    } else {
        m.v[0] = 1.0;
    }
    m.x2 = K * h;
    m.x4 = m.x2 * (K + 2.0) * h;
}

// Gas-kinetic flux at one Gauss point in the local frame (x = normal).
// Inputs: side states and their normal (x) and tangential (y, 2D) derivatives.
// Outputs for the S2O4 stages, with Fd = F(dt), Fh = F(dt/2) of Eq. (12):
//   STAGE 0: o0 = Fh (for W*, Eq. (19)), o1 = (8 Fh - Fd)/3 = dt F^n + dt^2/6 dF^n (Eqs. (17),(18),(20))
//   STAGE 1: o0 = (4/3)(Fd - 2 Fh) = dt^2/3 dF* (Eqs. (18), (20))
// Returns false if a side or the equilibrium state is non-physical.
template <int DIM, int STAGE>
__device__ __forceinline__ bool gks_flux(const FluxConst& fc, const double* Wl, const double* Wlx, const double* Wly,
                                         const double* Wr, const double* Wrx, const double* Wry, double dt,
                                         double* o0, double* o1)
{
    constexpr int NV = DIM + 2;
    const double K = fc.K;
    double rl, Ul, Vl, ll, pl, rr, Ur, Vr, lr, pr;
    bool ok = prim<DIM>(Wl, fc.gamma, rl, Ul, Vl, ll, pl);
    ok = prim<DIM>(Wr, fc.gamma, rr, Ur, Vr, lr, pr) && ok;
    if (!ok) return false;
    Mom<DIM> ml, mr;
    half_moments<DIM>(Ul, Vl, ll, K, +1, ml);
    half_moments<DIM>(Ur, Vr, lr, K, -1, mr);
    const double ril = 1.0 / rl, rir = 1.0 / rr;

    // micro-slopes of each side (Eq. (8)): b = dW / rho
    double a1l[NV], a1r[NV], a2l[NV], a2r[NV], b[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) b[k] = Wlx[k] * ril;
    slope_solve<DIM>(b, Ul, Vl, ll, K, a1l);
#pragma unroll
    for (int k = 0; k < NV; k++) b[k] = Wrx[k] * rir;
    slope_solve<DIM>(b, Ur, Vr, lr, K, a1r);
    if constexpr (DIM == 2) {
#pragma unroll
        for (int k = 0; k < NV; k++) b[k] = Wly[k] * ril;
        slope_solve<DIM>(b, Ul, Vl, ll, K, a2l);
#pragma unroll
        for (int k = 0; k < NV; k++) b[k] = Wry[k] * rir;
        slope_solve<DIM>(b, Ur, Vr, lr, K, a2r);
    }

    // equilibrium state and slopes by kinetic weighting, Eqs. (46)-(47)
    double Wc[NV], Wcx[NV], Wcy[NV], t1[NV], t2[NV];
    {
        double one[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) one[k] = k == 0 ? 1.0 : 0.0;
        Gm<DIM, 0, 0>(one, ml, t1);
        Gm<DIM, 0, 0>(one, mr, t2);
#pragma unroll
        for (int k = 0; k < NV; k++) Wc[k] = fma(rl, t1[k], rr * t2[k]);
        Gm<DIM, 0, 0>(a1l, ml, t1);
        Gm<DIM, 0, 0>(a1r, mr, t2);
#pragma unroll
        for (int k = 0; k < NV; k++) Wcx[k] = fma(rl, t1[k], rr * t2[k]);
        if constexpr (DIM == 2) {
            Gm<DIM, 0, 0>(a2l, ml, t1);
            Gm<DIM, 0, 0>(a2r, mr, t2);
#pragma unroll
            for (int k = 0; k < NV; k++) Wcy[k] = fma(rl, t1[k], rr * t2[k]);
        }
    }
    double rc, Uc, Vc, lc, pc;
    if (!prim<DIM>(Wc, fc.gamma, rc, Uc, Vc, lc, pc)) return false;
    Mom<DIM> mc;
    full_moments<DIM>(Uc, Vc, lc, K, mc);
    const double ric = 1.0 / rc;
    double ab1[NV], ab2[NV], Ab[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) b[k] = Wcx[k] * ric;
    slope_solve<DIM>(b, Uc, Vc, lc, K, ab1);
    if constexpr (DIM == 2) {
#pragma unroll
        for (int k = 0; k < NV; k++) b[k] = Wcy[k] * ric;
        slope_solve<DIM>(b, Uc, Vc, lc, K, ab2);
    }
    // compatibility for the equilibrium time slope (Eq. (9))
    Gm<DIM, 1, 0>(ab1, mc, t1);
    if constexpr (DIM == 2) {
        Gm<DIM, 0, 1>(ab2, mc, t2);
#pragma unroll
        for (int k = 0; k < NV; k++) b[k] = -(t1[k] + t2[k]);
    } else {
#pragma unroll
        for (int k = 0; k < NV; k++) b[k] = -t1[k];
    }
    slope_solve<DIM>(b, Uc, Vc, lc, K, Ab);

    // collision time (Sec. 3 preamble)
    const double jump = fabs((pl - pr) / (pl + pr));
    double tau;
    if (fc.tau_zero) tau = 0.0;
    else if (fc.viscous) tau = fma(fc.c2 * jump, dt, fc.mu / pc);
    else tau = (fc.c1 + fc.c2 * jump) * dt;

    // time coefficients of Eq. (10) integrated over [0, d], for d = dt and dt/2
    double Cd[6], Ch[6];
    if (tau == 0.0) {
        Cd[0] = dt; Cd[1] = 0.0; Cd[2] = 0.5 * dt * dt; Cd[3] = 0.0; Cd[4] = 0.0; Cd[5] = 0.0;
        Ch[0] = 0.5 * dt; Ch[1] = 0.0; Ch[2] = 0.125 * dt * dt; Ch[3] = 0.0; Ch[4] = 0.0; Ch[5] = 0.0;
    } else {
        const double eh = exp(-0.5 * dt / tau);
        const double ed = eh * eh;
        const double tt = tau * tau;
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const double d = s == 0 ? dt : 0.5 * dt;
            const double e = s == 0 ? ed : eh;
            const double om = 1.0 - e;
            double* C = s == 0 ? Cd : Ch;
            C[0] = fma(-tau, om, d);
            C[1] = fma(2.0 * tt, om, -tau * d * (1.0 + e));
            C[2] = fma(tt, om, d * fma(0.5, d, -tau));
            C[3] = tau * om;
            C[4] = fma(tau * d, e, -2.0 * tt * om);
            C[5] = -tt * om;
        }
    }
    // combined coefficients of the stage outputs
    double A0[6], A1[6];
#pragma unroll
    for (int j = 0; j < 6; j++) {
        if (STAGE == 0) { A0[j] = Ch[j]; A1[j] = (8.0 * Ch[j] - Cd[j]) * (1.0 / 3.0); }
        else            { A0[j] = (4.0 / 3.0) * fma(-2.0, Ch[j], Cd[j]); A1[j] = 0.0; }
    }

    // moment vectors multiplying the coefficients (all integrated against u psi)
    double acc0[NV], acc1[NV];
    {
        double one[NV], M1[NV], M2[NV], M3[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) one[k] = k == 0 ? 1.0 : 0.0;
        Gm<DIM, 1, 0>(one, mc, M1);
        Gm<DIM, 1, 0>(Ab, mc, M3);
#pragma unroll
        for (int k = 0; k < NV; k++) {
            acc0[k] = rc * fma(A0[0], M1[k], A0[2] * M3[k]);
            acc1[k] = rc * fma(A1[0], M1[k], A1[2] * M3[k]);
        }
        if (tau != 0.0) {
            Gm<DIM, 2, 0>(ab1, mc, M2);
            if constexpr (DIM == 2) {
                Gm<DIM, 1, 1>(ab2, mc, t1);
#pragma unroll
                for (int k = 0; k < NV; k++) M2[k] += t1[k];
            }
#pragma unroll
            for (int k = 0; k < NV; k++) {
                acc0[k] = fma(rc * A0[1], M2[k], acc0[k]);
                acc1[k] = fma(rc * A1[1], M2[k], acc1[k]);
            }
        }
    }
    if (tau != 0.0) {
        // non-equilibrium initial parts: left state over u > 0, right state over u < 0
        // (time slopes from <a1 u + a2 v + A> = 0, Eq. (9), with full-line moments)
#pragma unroll
        for (int side = 0; side < 2; side++) {
            const Mom<DIM>& mh = side == 0 ? ml : mr;
            const double* a1 = side == 0 ? a1l : a1r;
            const double* a2 = side == 0 ? a2l : a2r;
            const double rs = side == 0 ? rl : rr;
            Mom<DIM> mf;
            if (side == 0) full_moments<DIM>(Ul, Vl, ll, K, mf);
            else full_moments<DIM>(Ur, Vr, lr, K, mf);
            double As[NV], L4[NV], L5[NV], L6[NV];
            Gm<DIM, 1, 0>(a1, mf, t1);
            if constexpr (DIM == 2) {
                Gm<DIM, 0, 1>(a2, mf, t2);
#pragma unroll
                for (int k = 0; k < NV; k++) b[k] = -(t1[k] + t2[k]);
            } else {
#pragma unroll
                for (int k = 0; k < NV; k++) b[k] = -t1[k];
            }
            if (side == 0) slope_solve<DIM>(b, Ul, Vl, ll, K, As);
            else slope_solve<DIM>(b, Ur, Vr, lr, K, As);
            double one[NV];
#pragma unroll
            for (int k = 0; k < NV; k++) one[k] = k == 0 ? 1.0 : 0.0;
            Gm<DIM, 1, 0>(one, mh, L4);
            Gm<DIM, 2, 0>(a1, mh, L5);
            if constexpr (DIM == 2) {
                Gm<DIM, 1, 1>(a2, mh, t1);
#pragma unroll
                for (int k = 0; k < NV; k++) L5[k] += t1[k];
            }
            Gm<DIM, 1, 0>(As, mh, L6);
#pragma unroll
            for (int k = 0; k < NV; k++) {
                acc0[k] = fma(rs, fma(A0[3], L4[k], fma(A0[4], L5[k], A0[5] * L6[k])), acc0[k]);
                acc1[k] = fma(rs, fma(A1[3], L4[k], fma(A1[4], L5[k], A1[5] * L6[k])), acc1[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NV; k++) { o0[k] = acc0[k]; if (STAGE == 0) o1[k] = acc1[k]; }
    return true;
}

}  // namespace hgks
