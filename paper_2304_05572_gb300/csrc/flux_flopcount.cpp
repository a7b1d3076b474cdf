// flux_flopcount.cpp -- counts the FP64 operations of the closed-form gas-kinetic flux of
// hgks_math.cuh (Sec. 2.1, Eqs. (6)-(12), (46)-(47)) per Gauss point, on the host.
//
// The flux functions of hgks_math.cuh are host/device functions written on `double`; this
// translation unit compiles them for the host with every double replaced by a counting
// stand-in, so each evaluation reports how many operations of each kind the closed form
// takes: add / sub, mul, div, sqrt, exp and erfc one each, fma two (the convention of the
// roofline's algorithmic count).  The device's own instruction sequences for division, square
// root and the exponential, and the erfc table, are not counted: each is one operation.
// Built and run by paper_2304_05572_gb300/flopcount.py; not part of the library.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

namespace {
enum { K_ADD = 0, K_MUL, K_FMA, K_DIV, K_SQRT, K_EXP, K_ERFC, K_N };
unsigned long long g_n[K_N];
}  // namespace

struct cnt_double {
    double v;
    constexpr cnt_double() : v(0.0) {}
    constexpr cnt_double(double x) : v(x) {}
    template <class T> explicit operator T() const { return (T)v; }
    cnt_double& operator+=(cnt_double o) { g_n[K_ADD]++; v += o.v; return *this; }
    cnt_double& operator-=(cnt_double o) { g_n[K_ADD]++; v -= o.v; return *this; }
    cnt_double& operator*=(cnt_double o) { g_n[K_MUL]++; v *= o.v; return *this; }
};
inline cnt_double operator+(cnt_double a, cnt_double b) { g_n[K_ADD]++; return cnt_double(a.v + b.v); }
inline cnt_double operator-(cnt_double a, cnt_double b) { g_n[K_ADD]++; return cnt_double(a.v - b.v); }
inline cnt_double operator*(cnt_double a, cnt_double b) { g_n[K_MUL]++; return cnt_double(a.v * b.v); }
inline cnt_double operator/(cnt_double a, cnt_double b) { g_n[K_DIV]++; return cnt_double(a.v / b.v); }
inline cnt_double operator-(cnt_double a) { return cnt_double(-a.v); }
inline bool operator<(cnt_double a, cnt_double b) { return a.v < b.v; }
inline bool operator>(cnt_double a, cnt_double b) { return a.v > b.v; }
inline bool operator<=(cnt_double a, cnt_double b) { return a.v <= b.v; }
inline bool operator>=(cnt_double a, cnt_double b) { return a.v >= b.v; }
inline bool operator==(cnt_double a, cnt_double b) { return a.v == b.v; }
inline bool operator!=(cnt_double a, cnt_double b) { return a.v != b.v; }
inline cnt_double fabs(cnt_double a) { return cnt_double(std::fabs(a.v)); }
inline cnt_double sqrt(cnt_double a) { g_n[K_SQRT]++; return cnt_double(std::sqrt(a.v)); }
inline cnt_double exp(cnt_double a) { g_n[K_EXP]++; return cnt_double(std::exp(a.v)); }
inline cnt_double erfc(cnt_double a) { g_n[K_ERFC]++; return cnt_double(std::erfc(a.v)); }
inline cnt_double fma(cnt_double a, cnt_double b, cnt_double c) { g_n[K_FMA]++; return cnt_double(std::fma(a.v, b.v, c.v)); }

// the header's device-only helpers, for a host compile (only the flux functions are called)
inline cnt_double __dadd_rn(cnt_double a, cnt_double b) { return a + b; }
inline cnt_double __dsub_rn(cnt_double a, cnt_double b) { return a - b; }
inline cnt_double __dmul_rn(cnt_double a, cnt_double b) { return a * b; }
inline cnt_double __ddiv_rn(cnt_double a, cnt_double b) { return a / b; }
inline cnt_double __fma_rn(cnt_double a, cnt_double b, cnt_double c) { return fma(a, b, c); }
inline cnt_double __dsqrt_rn(cnt_double a) { return sqrt(a); }
template <class T> inline T __ldg(const T* p) { return *p; }
#define __device__
#define __host__
#define __constant__
#define __forceinline__ inline
#define double cnt_double
#include "hgks_math.cuh"
#undef double

using namespace hgks;

template <int DIM, int STAGE, bool PRFIX>
static void count(const char* name, int viscous, int tau_zero, bool last)
{
    FluxConst fc;
    fc.gamma = 1.4; fc.gm1 = 0.4;
    fc.K = DIM == 2 ? 3.0 : 4.0;
    fc.Kq = fc.K.v + DIM;
    fc.cslope = 4.0 / fc.Kq.v;
    fc.mu = 1e-3; fc.c1 = 0.01; fc.c2 = 1.0; fc.viscous = viscous; fc.tau_zero = tau_zero;
    fc.prfix = PRFIX ? 1.0 / 0.73 - 1.0 : 0.0;
    // a generic interface: distinct sides, non-zero slopes (the count does not depend on the data
    // as long as both sides and the equilibrium state are physical)
    cnt_double Wl[4] = {1.0, 0.1, 0.2, 2.5}, Wr[4] = {0.8, -0.1, 0.05, 2.0};
    cnt_double dx[4] = {0.1, 0.05, -0.02, 0.3}, dy[4] = {-0.05, 0.01, 0.03, -0.1};
    if (DIM == 1) { Wl[2] = 2.5; Wr[2] = 2.0; }
    cnt_double o0[4], o1[4];
    memset(g_n, 0, sizeof g_n);
    bool ok = gks_flux<DIM, STAGE, PRFIX>(fc, Wl, dx, dy, Wr, dx, dy, cnt_double(1e-3), o0, o1);
    unsigned long long flop = g_n[K_ADD] + g_n[K_MUL] + 2 * g_n[K_FMA] + g_n[K_DIV] + g_n[K_SQRT] + g_n[K_EXP] + g_n[K_ERFC];
    printf("  \"%s\": {\"ok\": %s, \"flop\": %llu, \"add\": %llu, \"mul\": %llu, \"fma\": %llu, \"div\": %llu, "
           "\"sqrt\": %llu, \"exp\": %llu, \"erfc\": %llu}%s\n", name, ok ? "true" : "false", flop, g_n[K_ADD],
           g_n[K_MUL], g_n[K_FMA], g_n[K_DIV], g_n[K_SQRT], g_n[K_EXP], g_n[K_ERFC], last ? "" : ",");
}

// values mode: flux_flopcount values DIM STAGE VISCOUS TAU_ZERO PRFIX gamma mu c1 c2 prandtl dt
//   followed by the 24 numbers Wl Wlx Wly Wr Wrx Wry (4 each; 1D uses the first 3 of each);
//   prints "ok o0[0..nv) o1[0..nv)" with 17 digits (the closed form evaluated on the host)
template <int DIM, int STAGE, bool PRFIX>
static int values(int viscous, int tau_zero, const double* c, const double* w)
{
    constexpr int NV = DIM + 2;
    FluxConst fc;
    fc.gamma = c[0]; fc.gm1 = c[0] - 1.0;
    fc.K = DIM == 2 ? (5.0 - 3.0 * c[0]) / (c[0] - 1.0) + 1.0 : (3.0 - c[0]) / (c[0] - 1.0);
    fc.Kq = fc.K.v + DIM;
    fc.cslope = 4.0 / fc.Kq.v;
    fc.mu = c[1]; fc.c1 = c[2]; fc.c2 = c[3]; fc.viscous = viscous; fc.tau_zero = tau_zero;
    fc.prfix = PRFIX ? 1.0 / c[4] - 1.0 : 0.0;
    cnt_double in[6][4], o0[4], o1[4];
    for (int q = 0; q < 6; q++)
        for (int k = 0; k < 4; k++) in[q][k] = k < NV ? w[q * 4 + k] : 0.0;
    bool ok = gks_flux<DIM, STAGE, PRFIX>(fc, in[0], in[1], in[2], in[3], in[4], in[5], cnt_double(c[5]), o0, o1);
    printf("%d", ok ? 1 : 0);
    for (int k = 0; k < NV; k++) printf(" %.17g", o0[k].v);
    for (int k = 0; k < NV; k++) printf(" %.17g", STAGE == 0 ? o1[k].v : 0.0);
    printf("\n");
    return 0;
}

int main(int argc, char** argv)
{
    if (argc > 1 && strcmp(argv[1], "values") == 0) {
        if (argc != 2 + 5 + 6 + 24) return 2;
        const int dim = atoi(argv[2]), stage = atoi(argv[3]), visc = atoi(argv[4]), tz = atoi(argv[5]), pr = atoi(argv[6]);
        double c[6], w[24];
        for (int j = 0; j < 6; j++) c[j] = atof(argv[7 + j]);
        for (int j = 0; j < 24; j++) w[j] = atof(argv[13 + j]);
        if (dim == 2 && stage == 0) return pr ? values<2, 0, true>(visc, tz, c, w) : values<2, 0, false>(visc, tz, c, w);
        if (dim == 2 && stage == 1) return pr ? values<2, 1, true>(visc, tz, c, w) : values<2, 1, false>(visc, tz, c, w);
        if (dim == 1 && stage == 0) return pr ? values<1, 0, true>(visc, tz, c, w) : values<1, 0, false>(visc, tz, c, w);
        return pr ? values<1, 1, true>(visc, tz, c, w) : values<1, 1, false>(visc, tz, c, w);
    }
    printf("{\n");
    count<2, 0, false>("2d_euler_stage1", 0, 0, false);
    count<2, 1, false>("2d_euler_stage2", 0, 0, false);
    count<2, 0, false>("2d_tau0_stage1", 0, 1, false);
    count<2, 1, false>("2d_tau0_stage2", 0, 1, false);
    count<2, 0, false>("2d_ns_stage1", 1, 0, false);
    count<2, 1, false>("2d_ns_stage2", 1, 0, false);
    count<2, 0, true>("2d_ns_prfix_stage1", 1, 0, false);
    count<2, 1, true>("2d_ns_prfix_stage2", 1, 0, false);
    count<1, 0, false>("1d_euler_stage1", 0, 0, false);
    count<1, 1, false>("1d_euler_stage2", 0, 0, true);
    printf("}\n");
    return 0;
}
