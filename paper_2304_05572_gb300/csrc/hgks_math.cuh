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
#include <cmath>

// flux arithmetic is also compiled for the host (unit checks of the formulas)
#define HGKS_HD __host__ __device__

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

// 1/x in free-order arithmetic (the flux, the tangential WENO-AO pass): the hardware's approximate reciprocal refined by two
// Newton-Raphson steps for 1/x, r <- r + r (1 - x r), each of which squares the relative error;
// within 1 ulp of the correctly rounded quotient for the normal x the flux meets (checked against
// IEEE division by hgks_check_reciprocal).  A zero x gives a NaN, which the flux's physical-state
// tests reject as they rejected the infinity of 1/0.  The host build divides.
HGKS_HD __forceinline__ double rcp_nr(double x)
{
#ifdef __CUDA_ARCH__
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
#else
    return 1.0 / x;
#endif
}

// 1/sqrt(x), x > 0, likewise: the hardware's approximation refined by two Newton-Raphson steps
// for 1/sqrt(x), y <- y + y (1 - x y^2) / 2 (each roughly squares the relative error).  The host
// build divides by the square root.
HGKS_HD __forceinline__ double rsqrt_nr(double x)
{
#ifdef __CUDA_ARCH__
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double hx = 0.5 * x;
    double t = fma(-hx * y, y, 0.5);
    y = fma(y, t, y);
    t = fma(-hx * y, y, 0.5);
    return fma(y, t, y);
#else
    return 1.0 / sqrt(x);
#endif
}

// Free-order FP64 with the same interface: the compiler may contract a*b + c into an FMA, and
// divisions and square roots go through the Newton-refined reciprocals above.  Used where the
// outputs only feed the flux (the tangential WENO-AO pass), never a flag decision.
struct fx {
    double v;
    __device__ __forceinline__ fx() {}
    __device__ __forceinline__ fx(double x) : v(x) {}
};
__device__ __forceinline__ fx operator+(fx a, fx b) { return fx(a.v + b.v); }
__device__ __forceinline__ fx operator-(fx a, fx b) { return fx(a.v - b.v); }
__device__ __forceinline__ fx operator*(fx a, fx b) { return fx(a.v * b.v); }
__device__ __forceinline__ fx operator/(fx a, fx b) { return fx(a.v * rcp_nr(b.v)); }
__device__ __forceinline__ fx operator-(fx a) { return fx(-a.v); }
__device__ __forceinline__ fx xfma(fx a, fx b, fx c) { return fx(fma(a.v, b.v, c.v)); }
__device__ __forceinline__ fx xabs(fx a) { return fx(fabs(a.v)); }
__device__ __forceinline__ fx xsqrt(fx a) { return fx(a.v * rsqrt_nr(a.v)); }

template <typename T> struct exact_order { static constexpr bool value = false; };
template <> struct exact_order<ex> { static constexpr bool value = true; };

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

// Smoothness indicators of Eq. (39) in cell units (with T = ex: the evaluation order the
// decisions need).
template <typename T>
__device__ __forceinline__ void ao_betas(const T* q, T* b)
{
    T s0 = (q[0] - T(2.0) * q[1]) + q[2], t0 = (q[0] - T(4.0) * q[1]) + T(3.0) * q[2];
    T s1 = (q[1] - T(2.0) * q[2]) + q[3], t1 = q[1] - q[3];
    T s2 = (q[2] - T(2.0) * q[3]) + q[4], t2 = (T(3.0) * q[2] - T(4.0) * q[3]) + q[4];
    b[0] = T(13.0 / 12.0) * (s0 * s0) + T(0.25) * (t0 * t0);
    b[1] = T(13.0 / 12.0) * (s1 * s1) + T(0.25) * (t1 * t1);
    b[2] = T(13.0 / 12.0) * (s2 * s2) + T(0.25) * (t2 * t2);
    T c1 = T(17.0 / 24.0) * (q[3] - q[1]) - T(5.0 / 48.0) * (q[4] - q[0]);
    T c2 = ((T(0.75) * (q[1] + q[3]) - T(0.0625) * (q[0] + q[4])) - T(1.375) * q[2]);
    T c3 = T(1.0 / 6.0) * (q[1] - q[3]) - T(1.0 / 12.0) * (q[0] - q[4]);
    T c4 = ((T(1.0 / 24.0) * (q[0] + q[4]) - T(1.0 / 6.0) * (q[1] + q[3])) + T(0.25) * q[2]);
    b[3] = ((((c1 * c1 + T(0.5) * (c1 * c3)) + T(13.0 / 3.0) * (c2 * c2)) + T(21.0 / 5.0) * (c2 * c4))
            + T(3129.0 / 80.0) * (c3 * c3)) + T(87617.0 / 140.0) * (c4 * c4);
}

// Normalised nonlinear weights, Eqs. (37), (38), (40), with the ratio delta/(beta_k + eps) squared.
// With T = fx the four ratios share one division (1/(e0 e1 e2 e3) times the other three factors)
// whenever that product is a finite positive number.
template <typename T>
__device__ __forceinline__ void ao_weights(const T* q, const AOConst& k, T* wb)
{
    T b[4], w[4], r[4];
    ao_betas(q, b);
    T d = ((xabs(b[3] - b[0]) + xabs(b[3] - b[1])) + xabs(b[3] - b[2])) * T(1.0 / 3.0);
    bool done = false;
    if constexpr (!exact_order<T>::value) {
        const double e0 = b[0].v + k.eps, e1 = b[1].v + k.eps, e2 = b[2].v + k.eps, e3 = b[3].v + k.eps;
        const double e01 = e0 * e1, e23 = e2 * e3, prod = e01 * e23;
        if (prod > 0.0 && prod < 1e300) {
            const double di = d.v * rcp_nr(prod);
            r[0] = T(di * (e1 * e23)); r[1] = T(di * (e0 * e23));
            r[2] = T(di * (e3 * e01)); r[3] = T(di * (e2 * e01));
            done = true;
        }
    }
    if (!done) {
#pragma unroll
        for (int j = 0; j < 4; j++) r[j] = d / (b[j] + T(k.eps));
    }
#pragma unroll
    for (int j = 0; j < 4; j++) w[j] = T(k.g[j]) * (T(1.0) + r[j] * r[j]);
    T inv = T(1.0) / (((w[0] + w[1]) + w[2]) + w[3]);
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
template <int NV, typename T>
__device__ __forceinline__ void eigvec(double gam, const T* Q, double nxd, double nyd, T (*L)[NV], T (*R)[NV])
{
    T gm1 = T(gam) - T(1.0);
    T rho = Q[0], ri = T(1.0) / rho;
    T U = Q[1] * ri;
    if constexpr (NV == 4) {
        T nx(nxd), ny(nyd);
        T V = Q[2] * ri;
        T q2 = U * U + V * V;
        T p = gm1 * (Q[3] - (T(0.5) * rho) * q2);
        T c2 = (T(gam) * p) * ri, c = xsqrt(c2), ci = T(1.0) / c;
        T H = (Q[3] + p) * ri;
        T un = U * nx + V * ny, ut = V * nx - U * ny;
        T b1 = gm1 / c2, b2 = (T(0.5) * b1) * q2;
        R[0][0] = T(1.0);    R[0][1] = T(1.0);       R[0][2] = T(0.0); R[0][3] = T(1.0);
        R[1][0] = U - c * nx; R[1][1] = U;             R[1][2] = -ny;     R[1][3] = U + c * nx;
        R[2][0] = V - c * ny; R[2][1] = V;             R[2][2] = nx;      R[2][3] = V + c * ny;
        R[3][0] = H - un * c; R[3][1] = T(0.5) * q2;  R[3][2] = ut;      R[3][3] = H + un * c;
        L[0][0] = T(0.5) * (b2 + un * ci); L[0][1] = -(T(0.5) * (b1 * U + nx * ci)); L[0][2] = -(T(0.5) * (b1 * V + ny * ci)); L[0][3] = T(0.5) * b1;
        L[1][0] = T(1.0) - b2;             L[1][1] = b1 * U;                          L[1][2] = b1 * V;                          L[1][3] = -b1;
        L[2][0] = -ut;                      L[2][1] = -ny;                             L[2][2] = nx;                              L[2][3] = T(0.0);
        L[3][0] = T(0.5) * (b2 - un * ci); L[3][1] = -(T(0.5) * (b1 * U - nx * ci)); L[3][2] = -(T(0.5) * (b1 * V - ny * ci)); L[3][3] = T(0.5) * b1;
    } else {
        T q2 = U * U;
        T p = gm1 * (Q[2] - (T(0.5) * rho) * q2);
        T c2 = (T(gam) * p) * ri, c = xsqrt(c2), ci = T(1.0) / c;
        T H = (Q[2] + p) * ri;
        T b1 = gm1 / c2, b2 = (T(0.5) * b1) * q2;
        R[0][0] = T(1.0);    R[0][1] = T(1.0);      R[0][2] = T(1.0);
        R[1][0] = U - c;      R[1][1] = U;            R[1][2] = U + c;
        R[2][0] = H - U * c;  R[2][1] = T(0.5) * q2; R[2][2] = H + U * c;
        L[0][0] = T(0.5) * (b2 + U * ci); L[0][1] = -(T(0.5) * (b1 * U + ci)); L[0][2] = T(0.5) * b1;
        L[1][0] = T(1.0) - b2;            L[1][1] = b1 * U;                     L[1][2] = -b1;
        L[2][0] = T(0.5) * (b2 - U * ci); L[2][1] = -(T(0.5) * (b1 * U - ci)); L[2][2] = T(0.5) * b1;
    }
}

// y = M x with the summation order ((m0 x0 + m1 x1) + m2 x2) + m3 x3.
template <int NV, typename T>
__device__ __forceinline__ void matvec(const T (*M)[NV], const T* x, T* y)
{
#pragma unroll
    for (int r = 0; r < NV; r++) {
        T s = M[r][0] * x[0] + M[r][1] * x[1];
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

#if defined(__CUDACC__)   // lane-group functions: device code only (the host count compiles the flux alone)
// Row r of M for a per-lane r, selected without indexing local memory.
template <int NV, typename T>
__device__ __forceinline__ void select_row(const T (*M)[NV], int r, T* row)
{
#pragma unroll
    for (int c = 0; c < NV; c++) {
        T v = M[0][c];
#pragma unroll
        for (int k = 1; k < NV; k++) v = r == k ? M[k][c] : v;
        row[c] = v;
    }
}

// The characteristic WENO-AO face reconstruction of weno_ao_face, spread over the 4 lanes of an
// aligned lane group (lane q = threadIdx.x & 3): lane q projects the window onto characteristic
// field q (row q of L), runs the nonlinear weights and the AO combination of that field alone,
// the 4 fields' results are exchanged with shuffles, and lane q projects back component q (row q
// of R); the components are exchanged again so that every lane returns the whole state val[]
// (for the positivity test) and its own component's derivative derq.  Every value is formed by
// the same operations in the same order as in weno_ao_face, so the results are bit-identical;
// the per-lane work, and so the latency of an item on the narrow FP64 pipe, is about a quarter.
// Lanes q >= NV (1D) duplicate field NV-1.  All 4 lanes of the group must call this together
// (mask gmask).
template <int NV>
__device__ __forceinline__ void weno_ao_face_x4(double gam, const AOConst& k, const double (*Qw)[NV], const double* Qs,
                                                int side, unsigned gmask, double* val, double& derq)
{
    const int q = threadIdx.x & 3;
    const int qc = q < NV ? q : NV - 1;
    const int lane0 = threadIdx.x & 28;
    ex L[NV][NV], R[NV][NV], qs[NV];
#pragma unroll
    for (int c = 0; c < NV; c++) qs[c] = ex(Qs[c]);
    eigvec<NV>(gam, qs, 1.0, 0.0, L, R);
    ex Lq[NV], Rq[NV];
    select_row<NV>(L, qc, Lq);
    select_row<NV>(R, qc, Rq);
    ex u[5], wb[4], pv[4], pd[4];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        ex s = Lq[0] * ex(Qw[j][0]) + Lq[1] * ex(Qw[j][1]);
#pragma unroll
        for (int c = 2; c < NV; c++) s = s + Lq[c] * ex(Qw[j][c]);
        u[j] = s;
    }
    ao_weights(u, k, wb);
    face_polys(u, side, pv, pd);
    const double uvq = ao_combine(wb, k, pv).v, udq = ao_combine(wb, k, pd).v;
    ex uv[NV], ud[NV];
#pragma unroll
    for (int c = 0; c < NV; c++) {
        uv[c] = ex(__shfl_sync(gmask, uvq, lane0 + c));
        ud[c] = ex(__shfl_sync(gmask, udq, lane0 + c));
    }
    // row qc of R times uv and ud, in the summation order of matvec
    ex v = Rq[0] * uv[0] + Rq[1] * uv[1], d = Rq[0] * ud[0] + Rq[1] * ud[1];
#pragma unroll
    for (int c = 2; c < NV; c++) { v = v + Rq[c] * uv[c]; d = d + Rq[c] * ud[c]; }
#pragma unroll
    for (int c = 0; c < NV; c++) val[c] = __shfl_sync(gmask, v.v, lane0 + c);
    derq = d.v;
}
#endif

// Reading (no safeguard is printed): rho <= 0 or p <= 0 after reconstruction -> first order.
// For rho > 0 (and gamma > 1), p > 0 exactly when rho E - ke > 0, ke = 0.5 (m_x^2 + m_y^2);
// tested in that division-free form, in this order.
template <int NV>
__device__ __forceinline__ bool nonphysical(double gam, const double* Q)
{
    (void)gam;
    ex ke;
    if constexpr (NV == 4) ke = ex(0.5) * (ex(Q[1]) * ex(Q[1]) + ex(Q[2]) * ex(Q[2]));
    else ke = ex(0.5) * (ex(Q[1]) * ex(Q[1]));
    ex pr = ex(Q[NV - 1]) * ex(Q[0]) - ke;
    return !(Q[0] > 0.0) || !(pr.v > 0.0);
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

__device__ __forceinline__ void gauss_ao(const fx* q, const AOConst& k, double* v, double* d)
{
    fx wb[4];
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

// Tangential WENO-AO of one pass (4 components, one lane) at the two Gauss points: projection of
// the 5 line values x[s][] onto the characteristic fields (rows of Lm), gauss_ao per field, and
// the projection back with Rm.  Free-order arithmetic (the outputs only feed the flux).
__device__ __forceinline__ void tang_ao(const fx (*Lm)[4], const fx (*Rm)[4], const fx (*x)[4], const AOConst& ak,
                                        double (*v)[2], double (*d)[2])
{
    // all 20 projections first: the line values are dead before the four fields' weights are
    // formed (134 registers against 170 with the projection inside the field loop)
    fx uc[4][5];
#pragma unroll
    for (int s = 0; s < 5; s++)
#pragma unroll
        for (int c = 0; c < 4; c++)
            uc[c][s] = xfma(Lm[c][3], x[s][3], xfma(Lm[c][2], x[s][2], xfma(Lm[c][1], x[s][1], Lm[c][0] * x[s][0])));
    double cv[4][2], cd[4][2];
#pragma unroll
    for (int c = 0; c < 4; c++) gauss_ao(uc[c], ak, cv[c], cd[c]);
#pragma unroll
    for (int g = 0; g < 2; g++)
#pragma unroll
        for (int r = 0; r < 4; r++) {
            double a = 0.0, b = 0.0;
#pragma unroll
            for (int c = 0; c < 4; c++) { a = fma(Rm[r][c].v, cv[c][g], a); b = fma(Rm[r][c].v, cd[c][g], b); }
            v[r][g] = a; d[r][g] = b;
        }
}

#if defined(__CUDACC__)
// The same pass spread over the 4 lanes of an aligned lane group like weno_ao_face_x4: lane q
// projects the 5 line values onto field q (row q of Lm), runs gauss_ao for it, the fields'
// Gauss-point values and derivatives are exchanged with shuffles, and lane q projects back its
// own component (row q of Rm): vq[g], dq[g] at the two Gauss points.
__device__ __forceinline__ void tang_ao_x4(const fx (*Lm)[4], const fx (*Rm)[4], const fx (*x)[4], const AOConst& ak,
                                           unsigned gmask, double* vq, double* dq)
{
    const int q = threadIdx.x & 3;
    const int lane0 = threadIdx.x & 28;
    fx Lq[4], Rq[4];
    select_row<4>(Lm, q, Lq);
    select_row<4>(Rm, q, Rq);
    fx u[5];
#pragma unroll
    for (int s = 0; s < 5; s++) u[s] = xfma(Lq[3], x[s][3], xfma(Lq[2], x[s][2], xfma(Lq[1], x[s][1], Lq[0] * x[s][0])));
    double cvq[2], cdq[2];
    gauss_ao(u, ak, cvq, cdq);
#pragma unroll
    for (int g = 0; g < 2; g++) {
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            a = fma(Rq[c].v, __shfl_sync(gmask, cvq[g], lane0 + c), a);
            b = fma(Rq[c].v, __shfl_sync(gmask, cdq[g], lane0 + c), b);
        }
        vq[g] = a; dq[g] = b;
    }
}
#endif

// ---------------------------------------------------------------- gas-kinetic flux
// Moments of a Maxwellian: u^n on one half line times the density (n <= 6), normalised v^m
// (full line, m <= 5), xi^2, xi^4.  Powers beyond these are never contracted.
template <int DIM>
struct Mom {
    double u[7];
    double v[DIM == 2 ? 6 : 1];
    double x2, x4;
};

// Primitive description of one Maxwellian (Eq. (3)): h = 1/(2 lambda) = p/rho.
template <int DIM>
struct MState {
    double rho, ri, U, V, p, h, lam, sl, E;
    double q, lam2c, two_lam;      // slope-solve constants: q = |U|^2 + Kq h, lam2c = lam^2 (4/Kq)/rho,
                                   // two_lam = 2 lam/rho (the 1/rho of <a> = dW/rho folded in)
};

struct FluxConst {
    double gamma, gm1, K, Kq, cslope, mu, c1, c2;   // Kq = K + D (D = 2 in 2D, 1 in 1D), cslope = 4/Kq
    double prfix;                                    // 1/Pr - 1 for viscous runs with Pr != 1, else 0
    int viscous, tau_zero;
};

template <int NV>
HGKS_HD __forceinline__ double dotv(const double* a, const double* b)
{
    double s = a[0] * b[0];
#pragma unroll
    for (int k = 1; k < NV; k++) s = fma(a[k], b[k], s);
    return s;
}

template <int DIM>
HGKS_HD __forceinline__ bool make_state(const double* W, const FluxConst& fc, MState<DIM>& s)
{
    s.rho = W[0];
    s.ri = rcp_nr(s.rho);
    s.U = W[1] * s.ri;
    s.V = DIM == 2 ? W[2] * s.ri : 0.0;
    s.E = W[DIM + 1];
    double mu2 = DIM == 2 ? fma(W[1], s.U, W[2] * s.V) : W[1] * s.U;
    s.p = fc.gm1 * fma(-0.5, mu2, s.E);
    s.h = s.p * s.ri;
    s.sl = rsqrt_nr(2.0 * s.h);                 // sqrt(lambda), lambda = 1/(2h)
    s.lam = s.sl * s.sl;
    s.q = fma(s.U, s.U, fma(s.V, s.V, fc.Kq * s.h));
    s.two_lam = 2.0 * s.lam * s.ri;
    s.lam2c = s.lam * fc.cslope * (0.5 * s.two_lam);
    return s.rho > 0.0 && s.p > 0.0;
}

// Micro-slope a with <a> = dW/rho: closed-form inverse of the moment system of Eq. (8), on the
// unscaled derivative dW (the 1/rho is carried by lam2c, two_lam and the last line).
template <int DIM>
HGKS_HD __forceinline__ void slope_solve(const double* dW, const MState<DIM>& s, double* a)
{
    if constexpr (DIM == 2) {
        double R4 = fma(-s.q, dW[0], 2.0 * dW[3]);
        double R3 = fma(-s.V, dW[0], dW[2]);
        double R2 = fma(-s.U, dW[0], dW[1]);
        double a4 = s.lam2c * fma(-2.0 * s.V, R3, fma(-2.0 * s.U, R2, R4));
        double a3 = fma(-s.V, a4, s.two_lam * R3);
        double a2 = fma(-s.U, a4, s.two_lam * R2);
        a[3] = a4; a[2] = a3; a[1] = a2;
        a[0] = fma(-0.5 * s.q, a4, fma(-s.V, a3, fma(-s.U, a2, dW[0] * s.ri)));
    } else {
        double R3 = fma(-s.q, dW[0], 2.0 * dW[2]);
        double R2 = fma(-s.U, dW[0], dW[1]);
        double a3 = s.lam2c * fma(-2.0 * s.U, R2, R3);
        double a2 = fma(-s.U, a3, s.two_lam * R2);
        a[2] = a3; a[1] = a2;
        a[0] = fma(-0.5 * s.q, a3, fma(-s.U, a2, dW[0] * s.ri));
    }
}

// Euler flux Jacobians applied to a direction: dF/dW d (x) and dG/dW d (y).
// For a Maxwellian g and a slope a with <a> = d, int u psi (a.psi) g = dF/dW d, so these
// give the moments int psi (a1 u + a2 v) g of the compatibility condition (Eq. (9)) and the
// flux moment of the equilibrium time slope in closed form.
template <int DIM>
HGKS_HD __forceinline__ void jac_x(const MState<DIM>& s, const double* d, const double gm1, double* out)
{
    const double g = s.E + s.p;     // rho H
    if constexpr (DIM == 2) {
        const double hq = 0.5 * fma(s.U, s.U, s.V * s.V);
        const double dp = gm1 * fma(hq, d[0], fma(-s.U, d[1], fma(-s.V, d[2], d[3])));
        const double dU = fma(-s.U, d[0], d[1]) * s.ri;
        out[0] = d[1];
        out[1] = fma(s.U, fma(-s.U, d[0], 2.0 * d[1]), dp);
        out[2] = fma(s.V, d[1], s.U * fma(-s.V, d[0], d[2]));
        out[3] = fma(dU, g, s.U * (d[3] + dp));
    } else {
        const double hq = 0.5 * s.U * s.U;
        const double dp = gm1 * fma(hq, d[0], fma(-s.U, d[1], d[2]));
        const double dU = fma(-s.U, d[0], d[1]) * s.ri;
        out[0] = d[1];
        out[1] = fma(s.U, fma(-s.U, d[0], 2.0 * d[1]), dp);
        out[2] = fma(dU, g, s.U * (d[2] + dp));
    }
}

HGKS_HD __forceinline__ void jac_y(const MState<2>& s, const double* e, const double gm1, double* out)
{
    const double g = s.E + s.p;
    const double hq = 0.5 * fma(s.U, s.U, s.V * s.V);
    const double dp = gm1 * fma(hq, e[0], fma(-s.U, e[1], fma(-s.V, e[2], e[3])));
    const double dV = fma(-s.V, e[0], e[2]) * s.ri;
    out[0] = e[2];
    out[1] = fma(s.U, e[2], s.V * fma(-s.U, e[0], e[1]));
    out[2] = fma(s.V, fma(-s.V, e[0], 2.0 * e[2]), dp);
    out[3] = fma(dV, g, s.V * (e[3] + dp));
}

// Time derivative of the conserved variables for the slopes d (x) and e (y) from the Euler
// compatibility (Eq. (9)): W_t = -(dF/dW d + dG/dW e).
template <int DIM>
HGKS_HD __forceinline__ void w_t(const MState<DIM>& s, const double* d, const double* e, const double gm1, double* out)
{
    jac_x<DIM>(s, d, gm1, out);
    if constexpr (DIM == 2) {
        double t[4];
        jac_y(s, e, gm1, t);
#pragma unroll
        for (int k = 0; k < 4; k++) out[k] = -(out[k] + t[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 3; k++) out[k] = -out[k];
    }
}

// Directional derivatives of Pi(W) = int u^2 psi g and Sigma(W) = int u v psi g (g the Maxwellian
// of W) along d (and e).  Since <abar> = d makes (abar.psi) g0 the derivative of g0 along d,
// int u psi (abar1 u + abar2 v) g0 = Pi'(W) d + Sigma'(W) e: the (abar1 u + abar2 v) g0 flux
// moment of Eq. (10) without solving for abar.  With h = p/rho and chain rule through (rho, U, V, h).
template <int DIM>
HGKS_HD __forceinline__ void pi_sigma_dir(const MState<DIM>& s, const double* d, const double* e, const double gm1,
                                          const double K, double* out)
{
    const double U = s.U, V = s.V, h = s.h, r = s.rho;
    const double U2 = U * U;
    if constexpr (DIM == 2) {
        const double V2 = V * V;
        const double hq = 0.5 * fma(U, U, V2);
        // Pi along d
        double dU = fma(-U, d[0], d[1]) * s.ri, dV = fma(-V, d[0], d[2]) * s.ri;
        double dp = gm1 * fma(hq, d[0], fma(-U, d[1], fma(-V, d[2], d[3])));
        double dh = fma(-h, d[0], dp) * s.ri;
        const double u2 = fma(U, U, h), v2 = fma(V, V, h);
        const double p0 = u2, p1 = U * fma(3.0, h, U2), p2 = u2 * V;
        const double p3 = 0.5 * fma(u2 * K, h, fma(u2, v2, fma(U2, fma(6.0, h, U2), 3.0 * h * h)));
        const double p3U = U * fma(K, h, fma(6.0, h, 2.0 * U2) + v2);
        const double p3h = 0.5 * fma(K, fma(2.0, h, U2), fma(8.0, h, fma(7.0, U2, V2)));
        out[0] = fma(p0, d[0], r * fma(2.0 * U, dU, dh));
        out[1] = fma(p1, d[0], r * fma(3.0 * u2, dU, 3.0 * U * dh));
        out[2] = fma(p2, d[0], r * fma(2.0 * U * V, dU, fma(u2, dV, V * dh)));
        out[3] = fma(p3, d[0], r * fma(p3U, dU, fma(u2 * V, dV, p3h * dh)));
        // Sigma along e
        dU = fma(-U, e[0], e[1]) * s.ri; dV = fma(-V, e[0], e[2]) * s.ri;
        dp = gm1 * fma(hq, e[0], fma(-U, e[1], fma(-V, e[2], e[3])));
        dh = fma(-h, e[0], dp) * s.ri;
        const double UV = U * V, k6 = 6.0 + K;
        const double s0 = UV, s1 = u2 * V, s2 = U * v2, s3 = 0.5 * UV * fma(k6, h, fma(U, U, V2));
        const double s3U = 0.5 * V * fma(k6, h, fma(3.0, U2, V2));
        const double s3V = 0.5 * U * fma(k6, h, fma(3.0, V2, U2));
        const double s3h = 0.5 * k6 * UV;
        out[0] += fma(s0, e[0], r * fma(V, dU, U * dV));
        out[1] += fma(s1, e[0], r * fma(2.0 * UV, dU, fma(u2, dV, V * dh)));
        out[2] += fma(s2, e[0], r * fma(v2, dU, fma(2.0 * UV, dV, U * dh)));
        out[3] += fma(s3, e[0], r * fma(s3U, dU, fma(s3V, dV, s3h * dh)));
    } else {
        (void)e;
        const double hq = 0.5 * U2;
        const double dU = fma(-U, d[0], d[1]) * s.ri;
        const double dp = gm1 * fma(hq, d[0], fma(-U, d[1], d[2]));
        const double dh = fma(-h, d[0], dp) * s.ri;
        const double u2 = fma(U, U, h);
        const double p0 = u2, p1 = U * fma(3.0, h, U2);
        const double p2 = 0.5 * fma(u2 * K, h, fma(U2, fma(6.0, h, U2), 3.0 * h * h));
        const double p2U = U * fma(K, h, fma(6.0, h, 2.0 * U2));
        const double p2h = 0.5 * fma(K, fma(2.0, h, U2), fma(6.0, h, 6.0 * U2));
        out[0] = fma(p0, d[0], r * fma(2.0 * U, dU, dh));
        out[1] = fma(p1, d[0], r * fma(3.0 * u2, dU, 3.0 * U * dh));
        out[2] = fma(p2, d[0], r * fma(p2U, dU, p2h * dh));
    }
}

// T(n, m) = <u^n v^m (a.psi)>, Tx(n, m) = <u^n v^m xi^2 (a.psi)>, G = <u^n v^m psi (a.psi)>.
template <int DIM, int N, int M>
HGKS_HD __forceinline__ void Gm(const double* a, const Mom<DIM>& m, double* out)
{
    if constexpr (DIM == 2) {
        const double ha3 = 0.5 * a[3];
        // Au(n) = a0 u_n + a1 u_{n+1} + a3/2 u_{n+2};  Bv(k) = a2 v_{k+1} + a3/2 (v_{k+2} + x2 v_k)
        const double Au0 = fma(a[1], m.u[N + 1], fma(ha3, m.u[N + 2], a[0] * m.u[N]));
        const double Au1 = fma(a[1], m.u[N + 2], fma(ha3, m.u[N + 3], a[0] * m.u[N + 1]));
        const double Au2 = fma(a[1], m.u[N + 3], fma(ha3, m.u[N + 4], a[0] * m.u[N + 2]));
        const double Bv0 = fma(a[2], m.v[M + 1], ha3 * fma(m.x2, m.v[M], m.v[M + 2]));
        const double Bv1 = fma(a[2], m.v[M + 2], ha3 * fma(m.x2, m.v[M + 1], m.v[M + 3]));
        const double Bv2 = fma(a[2], m.v[M + 3], ha3 * fma(m.x2, m.v[M + 2], m.v[M + 4]));
        out[0] = fma(m.v[M], Au0, m.u[N] * Bv0);                        // T(n, m)
        out[1] = fma(m.v[M], Au1, m.u[N + 1] * Bv0);                    // T(n+1, m)
        out[2] = fma(m.v[M + 1], Au0, m.u[N] * Bv1);                    // T(n, m+1)
        const double Tn2 = fma(m.v[M], Au2, m.u[N + 2] * Bv0);          // T(n+2, m)
        const double Tm2 = fma(m.v[M + 2], Au0, m.u[N] * Bv2);          // T(n, m+2)
        const double Tx = fma(m.x2, fma(m.v[M], Au0, m.u[N] * fma(a[2], m.v[M + 1], ha3 * m.v[M + 2])),
                              ha3 * m.x4 * (m.u[N] * m.v[M]));           // Tx(n, m)
        out[3] = 0.5 * (Tn2 + Tm2 + Tx);
    } else {
        const double ha2 = 0.5 * a[2];
        // T(n) = a0 u_n + a1 u_{n+1} + a2/2 (u_{n+2} + x2 u_n)
        const double c0 = fma(ha2, m.x2, a[0]);
        const double T0 = fma(a[1], m.u[N + 1], fma(ha2, m.u[N + 2], c0 * m.u[N]));
        const double T1 = fma(a[1], m.u[N + 2], fma(ha2, m.u[N + 3], c0 * m.u[N + 1]));
        const double T2 = fma(a[1], m.u[N + 3], fma(ha2, m.u[N + 4], c0 * m.u[N + 2]));
        const double Tx = fma(m.x2, fma(a[1], m.u[N + 1], fma(ha2, m.u[N + 2], a[0] * m.u[N])), ha2 * m.x4 * m.u[N]);
        out[0] = T0; out[1] = T1; out[2] = 0.5 * (T2 + Tx);
    }
}

// The two slope moments of one side that share a slope, 2D, in one pass over the shared sums:
//   Gm_x: G(0,0) and G(2,0) of the normal slope a1 (the x-slope of the equilibrium, Eq. (47), and
//         the u^2 part of the (a1 u + a2 v) g flux moment of Eq. (10));
//   Gm_y: G(0,0) and G(1,1) of the tangential slope a2 (the y-slope of the equilibrium and the
//         u v part of the same flux moment).
// Au(n) = a0 u_n + a1 u_{n+1} + a3/2 u_{n+2} and Bv(m) = a2 v_{m+1} + a3/2 (v_{m+2} + x2 v_m) are
// formed once for both moments (and T(2,0) once for both in Gm_x).
HGKS_HD __forceinline__ void Gm_x(const double* a, const Mom<2>& m, double* g00, double* g20)
{
    const double ha3 = 0.5 * a[3];
    double Au[5], Bv[3];
#pragma unroll
    for (int n = 0; n < 5; n++) Au[n] = fma(a[1], m.u[n + 1], fma(ha3, m.u[n + 2], a[0] * m.u[n]));
#pragma unroll
    for (int k = 0; k < 3; k++) Bv[k] = fma(a[2], m.v[k + 1], ha3 * fma(m.x2, m.v[k], m.v[k + 2]));
    auto T = [&](int n, int k) { return fma(m.v[k], Au[n], m.u[n] * Bv[k]); };
    const double bx = fma(a[2], m.v[1], ha3 * m.v[2]);
    auto Tx = [&](int n) { return fma(m.x2, fma(m.v[0], Au[n], m.u[n] * bx), ha3 * m.x4 * (m.u[n] * m.v[0])); };
    const double T20 = T(2, 0);
    g00[0] = T(0, 0); g00[1] = T(1, 0); g00[2] = T(0, 1);
    g00[3] = 0.5 * (T20 + T(0, 2) + Tx(0));
    g20[0] = T20; g20[1] = T(3, 0); g20[2] = T(2, 1);
    g20[3] = 0.5 * (T(4, 0) + T(2, 2) + Tx(2));
}

HGKS_HD __forceinline__ void Gm_y(const double* a, const Mom<2>& m, double* g00, double* g11)
{
    const double ha3 = 0.5 * a[3];
    double Au[4], Bv[4];
#pragma unroll
    for (int n = 0; n < 4; n++) Au[n] = fma(a[1], m.u[n + 1], fma(ha3, m.u[n + 2], a[0] * m.u[n]));
#pragma unroll
    for (int k = 0; k < 4; k++) Bv[k] = fma(a[2], m.v[k + 1], ha3 * fma(m.x2, m.v[k], m.v[k + 2]));
    auto T = [&](int n, int k) { return fma(m.v[k], Au[n], m.u[n] * Bv[k]); };
    auto Tx = [&](int n, int k) {
        return fma(m.x2, fma(m.v[k], Au[n], m.u[n] * fma(a[2], m.v[k + 1], ha3 * m.v[k + 2])),
                   ha3 * m.x4 * (m.u[n] * m.v[k]));
    };
    g00[0] = T(0, 0); g00[1] = T(1, 0); g00[2] = T(0, 1);
    g00[3] = 0.5 * (T(2, 0) + T(0, 2) + Tx(0, 0));
    g11[0] = T(1, 1); g11[1] = T(2, 1); g11[2] = T(1, 2);
    g11[3] = 0.5 * (T(3, 1) + T(1, 3) + Tx(1, 1));
}

template <int DIM>
HGKS_HD __forceinline__ void fill_vx(const MState<DIM>& s, const FluxConst& fc, Mom<DIM>& m)
{
    if constexpr (DIM == 2) {
        m.v[0] = 1.0;
        m.v[1] = s.V;
        m.v[2] = fma(s.V, m.v[1], s.h);
        m.v[3] = fma(s.V, m.v[2], 2.0 * s.h * m.v[1]);
        m.v[4] = fma(s.V, m.v[3], 3.0 * s.h * m.v[2]);
        m.v[5] = fma(s.V, m.v[4], 4.0 * s.h * m.v[3]);
    } else {
        m.v[0] = 1.0;
    }
    m.x2 = fc.K * s.h;
    m.x4 = m.x2 * (fc.K + 2.0) * s.h;
}

// <u^(n+2)> = U <u^(n+1)> + (n+1) h <u^n>, on the full line or either half line.
template <int DIM>
HGKS_HD __forceinline__ void recur_u(const MState<DIM>& s, Mom<DIM>& m)
{
#pragma unroll
    for (int n = 0; n < 5; n++) m.u[n + 2] = fma(s.U, m.u[n + 1], ((double)(n + 1) * s.h) * m.u[n]);
}

#include "erfcx_table.inc"

// erfcx(y) = exp(y^2) erfc(y) on [0, 8): per interval [k/4, (k+1)/4) a degree-11 polynomial in
// y - (k + 1/2)/4 (Chebyshev interpolant, relative error 2.1e-16; gen_erfcx_table.py).
// Read by device code only.
__device__ const double c_erfcx[HGKS_ERFCX_INTERVALS * (HGKS_ERFCX_DEGREE + 1)] = HGKS_ERFCX_TABLE;

// erfc(y) for y >= 0, given ey = exp(-y^2): ey erfcx(y) from the table below y = 8 (17 FP64
// operations instead of a full erfc, which recomputes the exponential), the library erfc above.
HGKS_HD __forceinline__ double erfc_nonneg(double y, double ey)
{
#ifdef __CUDA_ARCH__
    if (y < 8.0) {
        // k = round(4y - 1/2) in 0..31 (the interval whose centre is nearest): adding 1.5 2^52
        // leaves the rounded integer in the low mantissa bits
        constexpr double kRound = 6755399441055744.0;
        const double z = fma(y, 4.0, -0.5) + kRound;
        const int k = __double2loint(z);
        const double t = y - fma(z - kRound, 0.25, 0.125);
        const double* a = c_erfcx + k * (HGKS_ERFCX_DEGREE + 1);
        double p = __ldg(a + HGKS_ERFCX_DEGREE);
#pragma unroll
        for (int j = HGKS_ERFCX_DEGREE - 1; j >= 0; j--) p = fma(p, t, __ldg(a + j));
        return ey * p;
    }
#endif
    (void)ey;
    return erfc(y);
}

// Half-line moments of the left state over u > 0 (sign = +1) or of the right state over
// u < 0 (sign = -1), carrying the density: u[n] = rho <u^n> on the half line, with
// <1> = erfc(-+sqrt(lam) U)/2, <u> = U <1> +- exp(-lam U^2)/(2 sqrt(pi lam)).  Every moment
// product formed from them (psi_mom, Gm) has exactly one u-factor and so carries rho too.
// With x = sqrt(lam) U, erfc(-+x) is formed from E = erfc(|x|): the half line that the mean
// velocity points into holds 1 - E/2 of the mass, the other E/2.
template <int DIM>
HGKS_HD __forceinline__ void half_moments(const MState<DIM>& s, int sign, const FluxConst& fc, Mom<DIM>& m)
{
    const double sl = s.sl;
    const double x = sl * s.U;
    const double ex2 = exp(-x * x);
    const double e = ex2 * (0.56418958354775628695 * s.p * sl);   // rho h sqrt(lam)/sqrt(pi), rho h = p
    const double E = erfc_nonneg(fabs(x), ex2);
    const bool into = sign > 0 ? x >= 0.0 : x < 0.0;
    const double hr = 0.5 * s.rho;
    m.u[0] = into ? fma(-hr, E, s.rho) : hr * E;
    m.u[1] = fma(s.U, m.u[0], sign > 0 ? e : -e);
    recur_u<DIM>(s, m);
    fill_vx<DIM>(s, fc, m);
}

// <psi> and <u psi> of one (half-line) Maxwellian, normalised.
template <int DIM>
HGKS_HD __forceinline__ void psi_mom(const Mom<DIM>& m, double* out0, double* out1)
{
    if constexpr (DIM == 2) {
        const double w = m.v[2] + m.x2;
        out0[0] = m.u[0]; out0[1] = m.u[1]; out0[2] = m.u[0] * m.v[1]; out0[3] = 0.5 * fma(m.u[0], w, m.u[2]);
        out1[0] = m.u[1]; out1[1] = m.u[2]; out1[2] = m.u[1] * m.v[1]; out1[3] = 0.5 * fma(m.u[1], w, m.u[3]);
    } else {
        out0[0] = m.u[0]; out0[1] = m.u[1]; out0[2] = 0.5 * fma(m.u[0], m.x2, m.u[2]);
        out1[0] = m.u[1]; out1[1] = m.u[2]; out1[2] = 0.5 * fma(m.u[1], m.x2, m.u[3]);
    }
}

// Gas-kinetic flux at one Gauss point in the local frame (x = normal); Sec. 2.1, Eqs. (6)-(12),
// (46)-(47), collision time of Sec. 3.  Inputs: side states and their normal (x) and tangential
// (y, 2D) derivatives.  With Fd = F(dt), Fh = F(dt/2) of Eq. (12):
//   STAGE 0: o0 = Fh (for W*, Eq. (19)),  o1 = (8 Fh - Fd)/3 = dt F^n + dt^2/6 dF^n (Eqs. (17)-(18), (20))
//   STAGE 1: o0 = (4/3)(Fd - 2 Fh) = dt^2/3 dF* (Eqs. (18), (20))
// Returns false if a side or the equilibrium state is non-physical.
template <int DIM, int STAGE, bool PRFIX = false>
HGKS_HD __forceinline__ bool gks_flux(const FluxConst& fc, const double* Wl, const double* Wlx, const double* Wly,
                                         const double* Wr, const double* Wrx, const double* Wry, double dt,
                                         double* o0, double* o1)
{
    constexpr int NV = DIM + 2;
    MState<DIM> sl, sr;
    bool okl = make_state<DIM>(Wl, fc, sl);
    bool okr = make_state<DIM>(Wr, fc, sr);
    if (!(okl && okr)) return false;
    Mom<DIM> ml, mr;
    half_moments<DIM>(sl, +1, fc, ml);
    half_moments<DIM>(sr, -1, fc, mr);

    // micro-slopes of each side, Eq. (8)
    double a1l[NV], a1r[NV], a2l[NV], a2r[NV];
    slope_solve<DIM>(Wlx, sl, a1l);
    slope_solve<DIM>(Wrx, sr, a1r);
    if constexpr (DIM == 2) {
        slope_solve<DIM>(Wly, sl, a2l);
        slope_solve<DIM>(Wry, sr, a2r);
    }

    // equilibrium state and its slopes by kinetic weighting, Eqs. (46)-(47)
    double Wc[NV], Wcx[NV], Wcy[NV], pl0[NV], pl1[NV], pr0[NV], pr1[NV], t1[NV], t2[NV];
    psi_mom<DIM>(ml, pl0, pl1);
    psi_mom<DIM>(mr, pr0, pr1);
#pragma unroll
    for (int k = 0; k < NV; k++) Wc[k] = pl0[k] + pr0[k];
    // (2D: the u^2 and u v flux moments of the side slopes, L5 of Eq. (10), come out of the same
    // passes and are kept for the non-equilibrium terms below)
    double L5l[NV], L5r[NV];
    if (DIM == 2 && fc.tau_zero) {
        // tau = 0: no non-equilibrium terms, only the equilibrium slopes
        Gm<DIM, 0, 0>(a1l, ml, t1);
        Gm<DIM, 0, 0>(a1r, mr, t2);
#pragma unroll
        for (int k = 0; k < NV; k++) Wcx[k] = t1[k] + t2[k];
        Gm<DIM, 0, 0>(a2l, ml, t1);
        Gm<DIM, 0, 0>(a2r, mr, t2);
#pragma unroll
        for (int k = 0; k < NV; k++) Wcy[k] = t1[k] + t2[k];
    } else if constexpr (DIM == 2) {
        double u1[NV], u2[NV];
        Gm_x(a1l, ml, t1, L5l);
        Gm_x(a1r, mr, t2, L5r);
#pragma unroll
        for (int k = 0; k < NV; k++) Wcx[k] = t1[k] + t2[k];
        Gm_y(a2l, ml, t1, u1);
        Gm_y(a2r, mr, t2, u2);
#pragma unroll
        for (int k = 0; k < NV; k++) { Wcy[k] = t1[k] + t2[k]; L5l[k] += u1[k]; L5r[k] += u2[k]; }
    } else {
        Gm<DIM, 0, 0>(a1l, ml, t1);
        Gm<DIM, 0, 0>(a1r, mr, t2);
#pragma unroll
        for (int k = 0; k < NV; k++) Wcx[k] = t1[k] + t2[k];
        if (!fc.tau_zero) {
            Gm<DIM, 2, 0>(a1l, ml, L5l);
            Gm<DIM, 2, 0>(a1r, mr, L5r);
        }
    }
    MState<DIM> sc;
    if (!make_state<DIM>(Wc, fc, sc)) return false;

    // equilibrium flux moments: M1 = int u psi g0 = F(Wc);  M3 = int u psi Abar g0 = dF/dW Wc_t
    double M1[NV], M3[NV], Wct[NV];
    M1[0] = Wc[1];
    M1[1] = fma(Wc[1], sc.U, sc.p);
    if constexpr (DIM == 2) M1[2] = Wc[1] * sc.V;
    M1[NV - 1] = sc.U * (sc.E + sc.p);
    w_t<DIM>(sc, Wcx, Wcy, fc.gm1, Wct);
    jac_x<DIM>(sc, Wct, fc.gm1, M3);

    // collision time (Sec. 3 preamble)
    const double jump = fabs((sl.p - sr.p) * rcp_nr(sl.p + sr.p));
    double tau;
    if (fc.tau_zero) tau = 0.0;
    else if (fc.viscous) tau = fma(fc.c2 * jump, dt, fc.mu * rcp_nr(sc.p));
    else tau = fma(fc.c2, jump, fc.c1) * dt;

    // time integrals of the factors of Eq. (10) over [0, d], d = dt and dt/2
    double Cd[6], Ch[6];
    if (tau == 0.0) {
        Cd[0] = dt; Cd[1] = 0.0; Cd[2] = 0.5 * dt * dt; Cd[3] = 0.0; Cd[4] = 0.0; Cd[5] = 0.0;
        Ch[0] = 0.5 * dt; Ch[1] = 0.0; Ch[2] = 0.125 * dt * dt; Ch[3] = 0.0; Ch[4] = 0.0; Ch[5] = 0.0;
    } else {
        const double eh = exp(-0.5 * dt * rcp_nr(tau));
        const double ed = eh * eh;
        const double tt = tau * tau;
#pragma unroll
        for (int s2 = 0; s2 < 2; s2++) {
            const double d = s2 == 0 ? dt : 0.5 * dt;
            const double e = s2 == 0 ? ed : eh;
            const double om = 1.0 - e;
            double* C = s2 == 0 ? Cd : Ch;
            C[0] = fma(-tau, om, d);
            C[1] = fma(2.0 * tt, om, -tau * d * (1.0 + e));
            C[2] = fma(tt, om, d * fma(0.5, d, -tau));
            C[3] = tau * om;
            C[4] = fma(tau * d, e, -2.0 * tt * om);
            C[5] = -tt * om;
        }
    }
    double A0[6], A1[6];
#pragma unroll
    for (int j = 0; j < 6; j++) {
        if constexpr (STAGE == 0) { A0[j] = Ch[j]; A1[j] = fma(8.0, Ch[j], -Cd[j]) * (1.0 / 3.0); }
        else                      { A0[j] = (4.0 / 3.0) * fma(-2.0, Ch[j], Cd[j]); A1[j] = 0.0; }
    }

    double acc0[NV], acc1[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) {
        acc0[k] = fma(A0[0], M1[k], A0[2] * M3[k]);
        if constexpr (STAGE == 0) acc1[k] = fma(A1[0], M1[k], A1[2] * M3[k]);
    }
    if (tau != 0.0) {
        // (abar1 u + abar2 v) g0 term: Pi'(Wc) Wcx + Sigma'(Wc) Wcy
        double M2[NV];
        pi_sigma_dir<DIM>(sc, Wcx, Wcy, fc.gm1, fc.K, M2);
#pragma unroll
        for (int k = 0; k < NV; k++) {
            acc0[k] = fma(A0[1], M2[k], acc0[k]);
            if constexpr (STAGE == 0) acc1[k] = fma(A1[1], M2[k], acc1[k]);
        }
        // Prandtl-number fix (an extension: the paper's BGK flux has Pr = 1).  The energy flux
        // gains (1/Pr - 1) q, q the time-integrated heat flux of the distribution of Eq. (10)
        // relative to the equilibrium velocity (Uc, Vc).  With l = (|Uc|^2/2, -Uc, -Vc, 1),
        // int (u - Uc)(|u - Uc|^2 + xi^2)/2 phi = l.(int u psi phi) - Uc l.(int psi phi) for
        // every term phi of Eq. (10); the g0 term carries no heat flux, the density moments of
        // the (abar u) g0 and Abar g0 terms are -Wc_t and Wc_t (compatibility, Eq. (9)).
        // (a compile-time variant, so that the Pr = 1 flux keeps its register allocation)
        double lv[NV], Qh[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if constexpr (PRFIX) {
            lv[0] = 0.5 * fma(sc.U, sc.U, sc.V * sc.V);
            lv[1] = -sc.U;
            if constexpr (DIM == 2) lv[2] = -sc.V;
            lv[NV - 1] = 1.0;
            const double lWt = dotv<NV>(lv, Wct);
            Qh[1] = fma(sc.U, lWt, dotv<NV>(lv, M2));
            Qh[2] = fma(-sc.U, lWt, dotv<NV>(lv, M3));
        }
        // non-equilibrium initial parts: left state over u > 0, right state over u < 0, with the
        // time slope A from the compatibility condition <a1 u + a2 v + A> = 0 (Eq. (9)).  The three
        // terms of the two sides share their time coefficients, so their moments are summed over
        // the sides first: S4 (g^k), S5 ((a1 u + a2 v) g^k, formed with the equilibrium slopes
        // above) and S6 (A^k g^k)
        double S4[NV], S5[NV], S6[NV], D5s[NV], D6s[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            S4[k] = pl1[k] + pr1[k]; S5[k] = L5l[k] + L5r[k]; S6[k] = 0.0;
            if constexpr (PRFIX) { D5s[k] = 0.0; D6s[k] = 0.0; }
        }
#pragma unroll
        for (int side = 0; side < 2; side++) {
            const MState<DIM>& st = side == 0 ? sl : sr;
            const Mom<DIM>& mh = side == 0 ? ml : mr;
            double Wt[NV], As[NV], L6[NV];
            w_t<DIM>(st, side == 0 ? Wlx : Wrx, side == 0 ? Wly : Wry, fc.gm1, Wt);
            slope_solve<DIM>(Wt, st, As);
            Gm<DIM, 1, 0>(As, mh, L6);
#pragma unroll
            for (int k = 0; k < NV; k++) S6[k] += L6[k];
            if constexpr (PRFIX) {
                // density moments of the side's slope terms over its half line
                const double* a1 = side == 0 ? a1l : a1r;
                const double* a2 = side == 0 ? a2l : a2r;
                double D5[NV], D6[NV];
                Gm<DIM, 1, 0>(a1, mh, D5);
                if constexpr (DIM == 2) {
                    Gm<DIM, 0, 1>(a2, mh, t1);
#pragma unroll
                    for (int k = 0; k < NV; k++) D5[k] += t1[k];
                }
                Gm<DIM, 0, 0>(As, mh, D6);
#pragma unroll
                for (int k = 0; k < NV; k++) { D5s[k] += D5[k]; D6s[k] += D6[k]; }
            }
        }
#pragma unroll
        for (int k = 0; k < NV; k++) {
            acc0[k] = fma(A0[3], S4[k], fma(A0[4], S5[k], fma(A0[5], S6[k], acc0[k])));
            if constexpr (STAGE == 0) acc1[k] = fma(A1[3], S4[k], fma(A1[4], S5[k], fma(A1[5], S6[k], acc1[k])));
        }
        if constexpr (PRFIX) {
            // the g^k terms' density moments sum to Wc (Eq. (46))
            Qh[3] = fma(-sc.U, dotv<NV>(lv, Wc), dotv<NV>(lv, S4));
            Qh[4] = fma(-sc.U, dotv<NV>(lv, D5s), dotv<NV>(lv, S5));
            Qh[5] = fma(-sc.U, dotv<NV>(lv, D6s), dotv<NV>(lv, S6));
        }
        if constexpr (PRFIX) {
            double q0 = 0.0, q1 = 0.0;
#pragma unroll
            for (int j = 1; j < 6; j++) {
                q0 = fma(A0[j], Qh[j], q0);
                if constexpr (STAGE == 0) q1 = fma(A1[j], Qh[j], q1);
            }
            acc0[NV - 1] = fma(fc.prfix, q0, acc0[NV - 1]);
            if constexpr (STAGE == 0) acc1[NV - 1] = fma(fc.prfix, q1, acc1[NV - 1]);
        }
    }
#pragma unroll
    for (int k = 0; k < NV; k++) { o0[k] = acc0[k]; if (STAGE == 0) o1[k] = acc1[k]; }
    return true;
}

}  // namespace hgks
