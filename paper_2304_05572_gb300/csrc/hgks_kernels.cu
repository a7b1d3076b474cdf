// hgks_kernels.cu -- the S2O4 step of the hybrid WENO-AO gas-kinetic scheme as sm_103a
// FP64 kernels (arXiv 2304.05572, Sec. 2), and the host code that enqueues one step.
//
// Per stage: ghost fill -> for each sweep (x, then y in 2D):
//   raw normal flags -> normal reconstruction (linear inline, troubled sides appended to a
//   work list with warp-aggregated atomics) -> dense WENO-AO pass over that list ->
//   [2D: raw tangential flags -> Gauss-point reconstruction (linear inline, troubled passes
//   compacted the same way) -> dense WENO-AO pass] -> gas-kinetic flux per Gauss point
// -> stage update.  dt is reduced, clipped to t_end and applied on the device.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdio>

#include "hgks_internal.h"
#include "hgks_math.cuh"

namespace hgks {

const char* kclass_names[KC_COUNT] = {"ghost", "dt", "raw_normal_flags", "normal_recon", "normal_weno_ao",
                                      "raw_tangential_flags", "tangential_recon", "tangential_weno_ao",
                                      "gks_flux", "stage_update", "misc"};

namespace {

constexpr int TPB = 256;

// Global-memory access.  Every load and store of a kernel names the range its pointer must lie
// in (R.lo, R.hi: the solver's device buffers).  The debug build (HGKS_DEBUG_BOUNDS) checks each
// access against that range: an access outside it is skipped (a load returns 0), counted, and
// the address of the first one is kept for hgks_debug_bounds; nothing traps.  The normal build
// accesses memory directly.
#ifdef HGKS_DEBUG_BOUNDS
__device__ unsigned long long g_dbg_count;
__device__ unsigned long long g_dbg_first;
template <class T>
__device__ __forceinline__ bool in_range(const T* p, const char* lo, const char* hi)
{
    const char* c = (const char*)p;
    if (c >= lo && c + sizeof(T) <= hi) return true;
    atomicAdd(&g_dbg_count, 1ull);
    atomicCAS(&g_dbg_first, 0ull, (unsigned long long)(uintptr_t)c);
    return false;
}
template <class T, class R>
__device__ __forceinline__ T ldc(const T* p, const R& r) { return in_range(p, r.lo, r.hi) ? __ldg(p) : T(0); }
template <class T, class R>
__device__ __forceinline__ T rdc(const T* p, const R& r) { return in_range(p, r.lo, r.hi) ? *p : T(0); }
template <class T, class V, class R>
__device__ __forceinline__ void stc(T* p, V v, const R& r) { if (in_range(p, r.lo, r.hi)) *p = (T)v; }
#else
template <class T, class R>
__device__ __forceinline__ T ldc(const T* p, const R&) { return __ldg(p); }
template <class T, class R>
__device__ __forceinline__ T rdc(const T* p, const R&) { return *p; }
template <class T, class V, class R>
__device__ __forceinline__ void stc(T* p, V v, const R&) { *p = (T)v; }
#endif

// ---------------------------------------------------------------- ghost cells
// x ghosts on interior rows, then y ghosts over the padded width (fills corners).
// Non-reflecting: zero-gradient copy; reflect / symmetry: mirror, normal momentum negated;
// no-slip adiabatic: mirror, both momenta negated.  Prescribed states (Sec. 3.5): inflow,
// the wall that starts at x = shock_x0, and the boundary that follows the oblique shock line
// x = shock_x0 + shock_cot (y + shock_speed t), all evaluated at the ghost cell's centre at the
// stage time (t^n, or t^n + dt/2 in the second stage).  The centre and line positions are
// computed in one fixed IEEE order (no contraction) so that the side of the line a ghost cell
// falls on is the same in every implementation that follows this order.
__device__ __forceinline__ double stage_time(const Ctrl* ctrl, int stage)
{
    return stage == 0 ? ctrl->t : (ex(ctrl->t) + ex(0.5) * ex(ctrl->dt)).v;
}

__device__ __forceinline__ double cell_centre(double origin, int i, double h)
{
    return (ex(origin) + (ex((double)i) + ex(0.5)) * ex(h)).v;
}

// The first thread of a stage's x-ghost launch also empties the stage's work lists (no kernel
// of the stage reads them before the ghost fills are complete).
__device__ __forceinline__ void b_ghost_x(const Params& P, double* __restrict__ W, Ctrl* __restrict__ ctrl, long long id)
{
    if (ctrl->done) return;
    if (id == 0) ctrl->cnt[0][0] = ctrl->cnt[0][1] = ctrl->cnt[1][0] = ctrl->cnt[1][1] = 0;
    const GridGeom& g = P.g;
    int rowsI = g.dim == 2 ? g.ny : 1;
    long long total = (long long)g.nv * rowsI * NG * 2;
    if (id >= total) return;
    int side = (int)(id % 2); id /= 2;
    int l = (int)(id % NG) + 1; id /= NG;
    int j = (int)(id % rowsI);
    int k = (int)(id / rowsI);
    int bc = P.bc[side];
    int dst = side == 0 ? -l : g.nx - 1 + l;
    double* base = W + g.origin + (long long)k * g.plane + (long long)j * g.pitch;
    if (bc == HGKS_BC_INFLOW) { stc(base + dst, P.bc_state[side][k], g); return; }
    int src;
    bool mirror = bc == HGKS_BC_REFLECT || bc == HGKS_BC_SYMMETRY || bc == HGKS_BC_NOSLIP;
    if (bc == HGKS_BC_PERIODIC) src = side == 0 ? g.nx - l : l - 1;
    else if (bc == HGKS_BC_EXTRAP) src = side == 0 ? 0 : g.nx - 1;
    else src = side == 0 ? l - 1 : g.nx - l;
    double v = rdc(base + src, g);
    if (mirror) {
        if (k == 1) v = -v;
        if (bc == HGKS_BC_NOSLIP && g.dim == 2 && k == 2) v = -v;
    }
    stc(base + dst, v, g);
}

__global__ void k_ghost_x(Params P, double* __restrict__ W, Ctrl* __restrict__ ctrl)
{
    b_ghost_x(P, W, ctrl, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}


__device__ __forceinline__ void b_ghost_y(const Params& P, double* __restrict__ W, const Ctrl* __restrict__ ctrl, int stage, long long id)
{
    if (ctrl->done) return;
    const GridGeom& g = P.g;
    int width = g.nx + 2 * NG;
    long long total = (long long)g.nv * width * NG * 2;
    if (id >= total) return;
    int i = (int)(id % width) - NG; id /= width;
    int side = (int)(id % 2); id /= 2;
    int l = (int)(id % NG) + 1;
    int k = (int)(id / NG);
    int bc = P.bc[2 + side];
    int dst = side == 0 ? -l : g.ny - 1 + l;
    double* base = W + g.origin + (long long)k * g.plane + i;
    if (bc == HGKS_BC_INFLOW) { stc(base + (long long)dst * g.pitch, P.bc_state[2 + side][k], g); return; }
    if (bc == HGKS_BC_SHOCK_TRACK) {
        const double xc = cell_centre(P.x0, i, g.dx), yc = cell_centre(P.y0, dst, g.dy);
        const double t = stage_time(ctrl, stage);
        const double xs = (ex(P.shock_x0) + ex(P.shock_cot) * (ex(yc) + ex(P.shock_speed) * ex(t))).v;
        stc(base + (long long)dst * g.pitch, xc < xs ? P.bc_state[2 + side][k] : P.shock_pre[k], g);
        return;
    }
    if (bc == HGKS_BC_SHOCK_WALL && cell_centre(P.x0, i, g.dx) < P.shock_x0) {
        stc(base + (long long)dst * g.pitch, P.bc_state[2 + side][k], g);
        return;
    }
    int src;
    bool mirror = bc == HGKS_BC_REFLECT || bc == HGKS_BC_SYMMETRY || bc == HGKS_BC_NOSLIP || bc == HGKS_BC_SHOCK_WALL;
    if (bc == HGKS_BC_PERIODIC) src = side == 0 ? g.ny - l : l - 1;
    else if (bc == HGKS_BC_EXTRAP) src = side == 0 ? 0 : g.ny - 1;
    else src = side == 0 ? l - 1 : g.ny - l;
    double v = rdc(base + (long long)src * g.pitch, g);
    if (mirror) {
        if (k == 2) v = -v;
        if (bc == HGKS_BC_NOSLIP && k == 1) v = -v;
    }
    stc(base + (long long)dst * g.pitch, v, g);
}

__global__ void k_ghost_y(Params P, double* __restrict__ W, const Ctrl* __restrict__ ctrl, int stage)
{
    b_ghost_y(P, W, ctrl, stage, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}


// ---------------------------------------------------------------- time step
__global__ void k_begin_step(Ctrl* ctrl)
{
    ctrl->dtmin_bits = 0x7FF0000000000000ull;   // +inf
    ctrl->cnt[0][0] = ctrl->cnt[0][1] = ctrl->cnt[1][0] = ctrl->cnt[1][1] = 0;
}


// Sec. 3 preamble: dt = CFL min(h/(|U|+a), h^2/(4 nu)), h = min(dx, dy), nu = mu/rho;
// same evaluation order as the CPU reference so that dt is reproduced exactly.
__device__ __forceinline__ void b_dt(const Params& P, const double* __restrict__ W, Ctrl* ctrl, double h, long long start, long long stride)
{
    const GridGeom& g = P.g;
    int rowsI = g.dim == 2 ? g.ny : 1;
    long long n = (long long)rowsI * g.nx;
    unsigned long long best = 0x7FF0000000000000ull;
    for (long long id = start; id < n; id += stride) {
        int i = (int)(id % g.nx), j = (int)(id / g.nx);
        const double* c = W + g.origin + (long long)j * g.pitch + i;
        ex rho(rdc(c, g));
        ex ri = ex(1.0) / rho;
        ex U = ex(rdc(c + g.plane, g)) * ri;
        ex V = g.dim == 2 ? ex(rdc(c + 2 * g.plane, g)) * ri : ex(0.0);
        ex q2 = U * U + V * V;
        ex p = (ex(P.gamma) - ex(1.0)) * (ex(rdc(c + (g.nv - 1) * g.plane, g)) - (ex(0.5) * rho) * q2);
        ex a = xsqrt((ex(P.gamma) * p) * ri);
        ex d = ex(h) / (xsqrt(q2) + a);
        if (P.viscous) {
            ex nu = ex(P.mu) * ri;
            ex dv = (ex(h) * ex(h)) / (ex(4.0) * nu);
            if (dv.v < d.v) d = dv;
        }
        unsigned long long bits = (unsigned long long)__double_as_longlong(d.v);
        if (!(d.v > 0.0)) bits = 0x7FF8000000000000ull;   // non-physical cells are caught by the update
        best = bits < best ? bits : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(&ctrl->dtmin_bits, best);
}

__global__ void k_dt(Params P, const double* __restrict__ W, Ctrl* ctrl, double h)
{
    b_dt(P, W, ctrl, h, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}


__global__ void k_dt_final(Ctrl* ctrl, double cfl, double fixed_dt, double t_end, double tol)
{
    double dt = fixed_dt > 0.0 ? fixed_dt : cfl * __longlong_as_double((long long)ctrl->dtmin_bits);
    int done = ctrl->status != 0 || !(t_end - ctrl->t > tol);
    if (!done && ctrl->t + dt > t_end) dt = t_end - ctrl->t;
    if (!done && !(dt > 0.0 && dt < 1e300)) { ctrl->status = HGKS_ENONPHYSICAL; done = 1; }
    ctrl->dt = dt;
    ctrl->done = done;
}

__global__ void k_end_step(Ctrl* ctrl)
{
    if (ctrl->done) return;
    ctrl->t += ctrl->dt;
    ctrl->last_dt = ctrl->dt;
    ctrl->steps += 1;
}

__global__ void k_set_time(Ctrl* ctrl, double t0)
{
    ctrl->t = t0;
    ctrl->dt = 0.0;
    ctrl->last_dt = 0.0;
    ctrl->steps = 0;
    ctrl->status = 0;
    ctrl->done = 0;
    for (int a = 0; a < 2; a++) for (int b = 0; b < 2; b++) for (int c = 0; c < 2; c++) {
        ctrl->troubled[a][b][c] = 0; ctrl->examined[a][b][c] = 0;
    }
}

// warp-aggregated counter add
__device__ __forceinline__ void warp_count(unsigned long long* dst, unsigned int v)
{
    unsigned int tot = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(dst, (unsigned long long)tot);
}

// warp-aggregated append of one item per set predicate; returns nothing, writes list
template <class R>
__device__ __forceinline__ void warp_push(unsigned int* cnt, uint32_t* list, bool pred, uint32_t item, const R& rg)
{
    unsigned int mask = __ballot_sync(0xffffffffu, pred);
    if (!mask) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    unsigned int base = 0;
    if (lane == leader) base = atomicAdd(cnt, (unsigned int)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) stc(list + base + __popc(mask & ((1u << lane) - 1u)), item, rg);
}

// ---------------------------------------------------------------- normal pass
// local state access: component k of cell n on line t
__device__ __forceinline__ const double* cellp(const Params& P, const Sweep& S, const double* W, int t, int n)
{
    return W + P.g.origin + (long long)t * S.sT + (long long)n * S.sN;
}

template <int NV>
__device__ __forceinline__ void b_raw_nflags(const Params& P, const Sweep& S, const double* __restrict__ W, const Ctrl* __restrict__ ctrl, long long id)
{
    if (ctrl->done) return;
    int width = S.nn + 4;
    long long total = (long long)S.nlines * width;
    if (id >= total) return;
    int c = (int)(id % width), L = (int)(id / width);
    int t = L + S.tlo, n = c - 2;
    int tr = 0;
    if (P.recon_mode == HGKS_RECON_HYBRID) {
        const double* base = cellp(P, S, W, t, n - 2);
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double q[5];
            const double* b = base + (long long)S.perm[k] * P.g.plane;
#pragma unroll
            for (int s = 0; s < 5; s++) q[s] = ldc(b + (long long)s * S.sN, S);
            tr |= indicator_raw(q, S.Z1n);
        }
    }
    stc(S.rawN + id, tr, S);
}

// A solver's own sweep kernels run the two sweeps of a 2D stage in one launch (they share no
// buffer and no result until the update): blocks [0, nb0) work on the x sweep, the others on the
// y sweep; 1D launches give every block to the x sweep.  `id` is the thread's index within its
// sweep's blocks, `lanes` the number of threads on that sweep.
struct SweepBlock { int dir; long long id, lanes; };

__device__ __forceinline__ SweepBlock sweep_block(int nb0)
{
    SweepBlock r;
    r.dir = (int)blockIdx.x >= nb0 ? 1 : 0;
    const long long first = r.dir ? nb0 : 0;
    const long long nb = r.dir ? (long long)gridDim.x - nb0 : (long long)nb0;
    r.id = ((long long)blockIdx.x - first) * blockDim.x + threadIdx.x;
    r.lanes = nb * blockDim.x;
    return r;
}

template <int NV>
__global__ void k_raw_nflags(const SolveDesc* __restrict__ D, int nb0, int stage)
{
    const SweepBlock b = sweep_block(nb0);
    const SolveDesc& d = *D;
    b_raw_nflags<NV>(d.P, d.sw[b.dir], stage == 0 ? d.W : d.Ws, d.ctrl, b.id);
}


template <int NV>
__device__ __forceinline__ void store_line(const Params& P, const Sweep& S, int L, int m, int side, const double* val, const double* der)
{
    long long plane = (long long)S.nlines * S.nm;
    long long o = (long long)L * S.nm + m;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        stc(S.line + (long long)(side * NV + k) * plane + o, val[k], S);
        stc(S.line + (long long)((2 + side) * NV + k) * plane + o, der[k], S);
    }
}

template <int NV>
__device__ __forceinline__ void b_normal(const Params& P, const Sweep& S, const double* __restrict__ W, Ctrl* ctrl, int stage, long long id)
{
    if (ctrl->done) return;
    long long total = (long long)S.nlines * S.nm;
    bool active = id < total;
    int L = 0, m = 0;
    if (active) { m = (int)(id % S.nm); L = (int)(id / S.nm); }
    int t = L + S.tlo;
    int fl[2] = {0, 0};
    if (active) {
        const uint8_t* raw = S.rawN + (long long)L * (S.nn + 4);
#pragma unroll
        for (int side = 0; side < 2; side++) {
            int c = m - 1 + side;     // cell index; raw index of cell c is c + 2
            int f;
            if (P.recon_mode == HGKS_RECON_LINEAR) f = 0;
            else if (P.recon_mode == HGKS_RECON_WENOAO) f = 1;
            else f = rdc(raw + c + 1, S) | rdc(raw + c + 2, S) | rdc(raw + c + 3, S);   // Step 4
            fl[side] = f;
        }
        uint8_t* fo = S.flagN + (long long)L * (S.nn + 2);
        stc(fo + m + 1, fl[1], S);
        if (m == 0) stc(fo, fl[0], S);
    }
    bool counted = active && t >= 0 && t < S.nt && m < S.nn;
    warp_count(&ctrl->troubled[stage][S.dir][0], counted && fl[1] ? 1u : 0u);
    warp_count(&ctrl->examined[stage][S.dir][0], counted ? 1u : 0u);
#pragma unroll
    for (int side = 0; side < 2; side++) {
        bool push = active && fl[side];
        warp_push(&ctrl->cnt[S.dir][0], S.itemsN, push, (uint32_t)((((long long)L * S.nm + m) << 1) | side), S);
        if (!active || fl[side]) continue;
        int c = m - 1 + side;
        double val[NV], der[NV];
        const double* base = cellp(P, S, W, t, c - 2);
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double q[5];
            const double* b = base + (long long)S.perm[k] * P.g.plane;
#pragma unroll
            for (int s = 0; s < 5; s++) q[s] = ldc(b + (long long)s * S.sN, S);
            if (side == 0) linear_left(q, S.inv12hn, val[k], der[k]);
            else linear_right(q, S.inv12hn, val[k], der[k]);
        }
        if (nonphysical<NV>(P.gamma, val)) {
            const double* cc = cellp(P, S, W, t, c);
#pragma unroll
            for (int k = 0; k < NV; k++) { val[k] = ldc(cc + (long long)S.perm[k] * P.g.plane, S); der[k] = 0.0; }
        }
        store_line<NV>(P, S, L, m, side, val, der);
    }
}

template <int NV>
__global__ void k_normal(const SolveDesc* __restrict__ D, int nb0, int stage)
{
    const SweepBlock b = sweep_block(nb0);
    const SolveDesc& d = *D;
    b_normal<NV>(d.P, d.sw[b.dir], stage == 0 ? d.W : d.Ws, d.ctrl, stage, b.id);
}


// Troubled items of one compacted WENO-AO pass at or above which every item gets one lane, below
// which an aligned group of 4 lanes (one characteristic field per lane).  The lane-group form
// repeats the eigenvector work in each of its lanes (about 1.9 times the FP64 instructions per
// item) and pays only while the items leave the schedulers short of warps; measured on this part
// (512^2 and 1024^2 four-quadrant steps, 200x100 tube, thresholds 8192 / 32768 / 131072) the
// crossover lies near 32768 items.  A constant, not a function of the launch, so that a solve
// takes the same form in its own kernels and in batched ones.
constexpr unsigned int kAoOneLaneMin = 32768;

// The window (cells i-2..i+2 across the face, all components) and the face average of the
// troubled side `it` of the normal pass.
template <int NV>
__device__ __forceinline__ void normal_ao_item(const Params& P, const Sweep& S, const double* __restrict__ W, uint32_t it,
                                               double (*Qw)[NV], double* Qs, int& side, int& L, int& m)
{
    side = it & 1;
    const long long lm = it >> 1;
    m = (int)(lm % S.nm); L = (int)(lm / S.nm);
    const int t = L + S.tlo;
    const int c = m - 1 + side;
    const double* base = cellp(P, S, W, t, c - 2);
#pragma unroll
    for (int s = 0; s < 5; s++)
#pragma unroll
        for (int k = 0; k < NV; k++) Qw[s][k] = ldc(base + (long long)s * S.sN + (long long)S.perm[k] * P.g.plane, S);
    const double* cl = cellp(P, S, W, t, m - 1);
    const double* cr = cellp(P, S, W, t, m);
#pragma unroll
    for (int k = 0; k < NV; k++) {
        long long o = (long long)S.perm[k] * P.g.plane;
        Qs[k] = ((ex(ldc(cl + o, S)) + ex(ldc(cr + o, S))) * ex(0.5)).v;
    }
}

// The troubled sides of the normal pass: one per lane (weno_ao_face) from kAoOneLaneMin items
// on, else one per aligned group of 4 lanes (weno_ao_face_x4: lane q carries characteristic
// field q and stores component q).  Both forms give the same bits.  `lane`, `lanes`: this
// thread's index among, and the number of, the lanes working on the pass.
template <int NV>
__device__ __forceinline__ void b_normal_ao(const Params& P, const Sweep& S, const double* __restrict__ W, const Ctrl* __restrict__ ctrl, long long lane, long long lanes)
{
    if (ctrl->done) return;
    unsigned int n = ctrl->cnt[S.dir][0];
    AOConst ak;
    for (int j = 0; j < 4; j++) ak.g[j] = P.g_ao[j];
    ak.g3inv = P.g3inv; ak.gr[0] = P.gr[0]; ak.gr[1] = P.gr[1]; ak.gr[2] = P.gr[2]; ak.eps = P.eps;
    const long long plane = (long long)S.nlines * S.nm;
    if (n >= kAoOneLaneMin) {
        for (unsigned int i = (unsigned int)lane; i < n; i += (unsigned int)lanes) {
            double Qw[5][NV], Qs[NV], val[NV], d[NV];
            int side, L, m;
            normal_ao_item<NV>(P, S, W, rdc(S.itemsN + i, S), Qw, Qs, side, L, m);
            weno_ao_face<NV>(P.gamma, ak, Qw, Qs, side == 0 ? +1 : -1, val, d);
            const bool bad = nonphysical<NV>(P.gamma, val);
            const long long o = (long long)L * S.nm + m;
#pragma unroll
            for (int k = 0; k < NV; k++) {
                stc(S.line + (long long)(side * NV + k) * plane + o, bad ? Qw[2][k] : val[k], S);
                stc(S.line + (long long)((2 + side) * NV + k) * plane + o, bad ? 0.0 : (ex(d[k]) * ex(S.inv_hn)).v, S);
            }
        }
        return;
    }
    const int q = threadIdx.x & 3;
    const unsigned gmask = 0xFu << (threadIdx.x & 28);
    for (unsigned int i = (unsigned int)(lane >> 2); i < n; i += (unsigned int)(lanes >> 2)) {
        double Qw[5][NV], Qs[NV], val[NV], dq;
        int side, L, m;
        normal_ao_item<NV>(P, S, W, rdc(S.itemsN + i, S), Qw, Qs, side, L, m);
        weno_ao_face_x4<NV>(P.gamma, ak, Qw, Qs, side == 0 ? +1 : -1, gmask, val, dq);
        double vq = 0.0;
        if (nonphysical<NV>(P.gamma, val)) {
            vq = Qw[2][q < NV ? q : 0];
            dq = 0.0;
        } else {
#pragma unroll
            for (int k = 0; k < NV; k++)
                if (k == q) vq = val[k];
            dq = (ex(dq) * ex(S.inv_hn)).v;
        }
        if (q < NV) {
            long long o = (long long)L * S.nm + m;
            stc(S.line + (long long)(side * NV + q) * plane + o, vq, S);
            stc(S.line + (long long)((2 + side) * NV + q) * plane + o, dq, S);
        }
    }
}

template <int NV>
__global__ void k_normal_ao(const SolveDesc* __restrict__ D, int nb0, int stage)
{
    const SweepBlock b = sweep_block(nb0);
    const SolveDesc& d = *D;
    b_normal_ao<NV>(d.P, d.sw[b.dir], stage == 0 ? d.W : d.Ws, d.ctrl, b.id, b.lanes);
}


// ---------------------------------------------------------------- tangential passes (2D)
__device__ __forceinline__ double lineval(const Sweep& S, int X, int k, int t, int m)
{
    long long plane = (long long)S.nlines * S.nm;
    return ldc(S.line + (long long)(X * 4 + k) * plane + (long long)(t - S.tlo) * S.nm + m, S);
}

// Raw tangential flags, one segment per aligned group of 4 lanes: lane q runs the indicator of
// every pass X on component q, the 4 components' bits are OR-ed with shuffles (a cell is smooth
// only if every component is), and lane 0 stores them.  `id` counts lanes.
__device__ __forceinline__ void b_raw_tflags_x4(const Params& P, const Sweep& S, const Ctrl* __restrict__ ctrl, long long id)
{
    if (ctrl->done) return;
    long long total = (long long)(S.nt + 2) * S.nm;
    const long long seg = id >> 2;
    if (seg >= total) return;                       // the same for the 4 lanes of a group
    const int q = (int)(id & 3);
    const unsigned gmask = 0xFu << (threadIdx.x & 28);
    int m = (int)(seg % S.nm);
    int t = (int)(seg / S.nm) - 1;
    unsigned int bits = 0;
    if (P.recon_mode == HGKS_RECON_HYBRID) {
#pragma unroll
        for (int X = 0; X < 4; X++) {
            double qv[5];
#pragma unroll
            for (int s = 0; s < 5; s++) qv[s] = lineval(S, X, q, t - 2 + s, m);
            bits |= (unsigned)indicator_raw(qv, S.Z1t) << X;
        }
        bits |= __shfl_xor_sync(gmask, bits, 1);
        bits |= __shfl_xor_sync(gmask, bits, 2);
    }
    if (q == 0) stc(S.rawT + seg, bits, S);
}

__device__ __forceinline__ void b_raw_tflags_x1(const Params& P, const Sweep& S, const Ctrl* __restrict__ ctrl, long long id)
{
    if (ctrl->done) return;
    long long total = (long long)(S.nt + 2) * S.nm;
    if (id >= total) return;
    int m = (int)(id % S.nm);
    int t = (int)(id / S.nm) - 1;
    uint8_t bits = 0;
    if (P.recon_mode == HGKS_RECON_HYBRID) {
#pragma unroll
        for (int X = 0; X < 4; X++) {
            int tr = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                double q[5];
#pragma unroll
                for (int s = 0; s < 5; s++) q[s] = lineval(S, X, k, t - 2 + s, m);
                tr |= indicator_raw(q, S.Z1t);
            }
            bits |= (uint8_t)(tr << X);
        }
    }
    stc(S.rawT + id, bits, S);
}

// Small sweeps (fewer segments than a few warps per scheduler) spread a segment over 4 lanes,
// which shortens the chain of FP64 instructions per thread; large sweeps keep one segment per
// thread.  The arithmetic, and so every result, is the same either way.
__device__ __forceinline__ void b_raw_tflags(const Params& P, const Sweep& S, const Ctrl* __restrict__ ctrl, long long id)
{
    if (S.tlanes == 4) b_raw_tflags_x4(P, S, ctrl, id);
    else b_raw_tflags_x1(P, S, ctrl, id);
}

__global__ void k_raw_tflags(const SolveDesc* __restrict__ D, int nb0)
{
    const SweepBlock b = sweep_block(nb0);
    const SolveDesc& d = *D;
    b_raw_tflags(d.P, d.sw[b.dir], d.ctrl, b.id);
}


__device__ __forceinline__ void gp_positivity(const Params& P, const Sweep& S, int t, int m, int X, double (*v)[2], double (*d)[2])
{
    if (X > 1) return;
#pragma unroll
    for (int g = 0; g < 2; g++) {
        double Q[4] = {v[0][g], v[1][g], v[2][g], v[3][g]};
        if (nonphysical<4>(P.gamma, Q)) {
#pragma unroll
            for (int k = 0; k < 4; k++) { v[k][g] = lineval(S, X, k, t, m); d[k][g] = 0.0; }
        }
    }
}

// Gauss-point reconstruction of the smooth passes, one segment per aligned group of 4 lanes, lane q
// carrying component q: the Step-4 spread flags of the segment (the same in every lane; lane 0
// stores them, counts them and appends the troubled passes to the WENO-AO work list), then for
// every smooth pass the quartic of component q at both Gauss points; the positivity test of the
// Q^l, Q^r passes gathers the 4 components with shuffles.  `id` counts lanes.  Every lane of the
// warp reaches the warp-wide counts and appends.
__device__ __forceinline__ void b_tang_x4(const Params& P, const Sweep& S, Ctrl* ctrl, int stage, long long id)
{
    if (ctrl->done) return;
    long long total = (long long)S.nt * S.nm;
    const long long seg = id >> 2;
    const int q = (int)(id & 3);
    const int lane0 = threadIdx.x & 28;
    const unsigned gmask = 0xFu << lane0;
    bool active = seg < total;                      // the same for the 4 lanes of a group
    int m = 0, t = 0;
    unsigned int bits = 0;
    if (active) {
        m = (int)(seg % S.nm); t = (int)(seg / S.nm);
        if (P.recon_mode == HGKS_RECON_LINEAR) bits = 0;
        else if (P.recon_mode == HGKS_RECON_WENOAO) bits = 0xF;
        else bits = rdc(S.rawT + (long long)t * S.nm + m, S) | rdc(S.rawT + (long long)(t + 1) * S.nm + m, S)
                    | rdc(S.rawT + (long long)(t + 2) * S.nm + m, S);
        if (q == 0) stc(S.flagT + seg, bits, S);
    }
    const bool lead = active && q == 0;
    warp_count(&ctrl->troubled[stage][S.dir][1], lead ? (unsigned)__popc(bits) : 0u);
    warp_count(&ctrl->examined[stage][S.dir][1], lead ? 4u : 0u);
    const long long plane = (long long)S.nt * S.nm;
    const long long o = (long long)t * S.nm + m;
#pragma unroll
    for (int X = 0; X < 4; X++) {
        bool f = active && ((bits >> X) & 1);
        warp_push(&ctrl->cnt[S.dir][1], S.itemsT, f && q == 0, (uint32_t)((seg << 2) | X), S);
        if (!active || f) continue;                 // the same for the 4 lanes of a group
        double qv[5], v[2], d[2];
#pragma unroll
        for (int s = 0; s < 5; s++) qv[s] = lineval(S, X, q, t - 2 + s, m);
        gauss_linear(qv, v, d);
        if (X <= 1) {
            // Reading: a reconstructed state with rho <= 0 or p <= 0 falls back to first order
#pragma unroll
            for (int g = 0; g < 2; g++) {
                double Q[4];
#pragma unroll
                for (int c = 0; c < 4; c++) Q[c] = __shfl_sync(gmask, v[g], lane0 + c);
                if (nonphysical<4>(P.gamma, Q)) { v[g] = lineval(S, X, q, t, m); d[g] = 0.0; }
            }
        }
        // Q index: 0 Wl, 1 Wlx, 2 Wly, 3 Wr, 4 Wrx, 5 Wry
        constexpr int qx[4] = {0, 3, 1, 4};
#pragma unroll
        for (int g = 0; g < 2; g++) {
            stc(S.gp + (long long)((g * 6 + qx[X]) * 4 + q) * plane + o, v[g], S);
            if (X <= 1) stc(S.gp + (long long)((g * 6 + qx[X] + 2) * 4 + q) * plane + o, d[g] * S.inv_ht, S);
        }
    }
}

// Large sweeps: the Step-4 spread flags of a segment (stored, counted, troubled passes appended
// to the WENO-AO work list); the smooth passes are reconstructed inside the flux kernel
// (b_flux, gp_linear_at), so their Gauss-point states never go to memory.
__device__ __forceinline__ void b_tflags_x1(const Params& P, const Sweep& S, Ctrl* ctrl, int stage, long long id)
{
    if (ctrl->done) return;
    long long total = (long long)S.nt * S.nm;
    bool active = id < total;
    int m = 0, t = 0;
    unsigned int bits = 0;
    if (active) {
        m = (int)(id % S.nm); t = (int)(id / S.nm);
        if (P.recon_mode == HGKS_RECON_LINEAR) bits = 0;
        else if (P.recon_mode == HGKS_RECON_WENOAO) bits = 0xF;
        else bits = rdc(S.rawT + (long long)t * S.nm + m, S) | rdc(S.rawT + (long long)(t + 1) * S.nm + m, S)
                    | rdc(S.rawT + (long long)(t + 2) * S.nm + m, S);
        stc(S.flagT + id, bits, S);
    }
    warp_count(&ctrl->troubled[stage][S.dir][1], active ? (unsigned)__popc(bits) : 0u);
    warp_count(&ctrl->examined[stage][S.dir][1], active ? 4u : 0u);
#pragma unroll
    for (int X = 0; X < 4; X++) {
        bool f = active && ((bits >> X) & 1);
        warp_push(&ctrl->cnt[S.dir][1], S.itemsT, f, (uint32_t)((((long long)t * S.nm + m) << 2) | X), S);
    }
}

// Gauss-point state of the smooth pass X of segment (t, m) at Gauss point g (0: -xi_g, 1: +xi_g):
// the quartic of each component (the FMA chain of gauss_linear, so the same bits), the
// first-order fallback of the Q^l, Q^r passes, the tangential derivative in 1/h_t units.
__device__ __forceinline__ void gp_linear_at(const Params& P, const Sweep& S, int X, int t, int m, int g,
                                             double* v, double* d)
{
    const double* cv = g == 0 ? c_gauss.VM[3] : c_gauss.VP[3];
    const double* cd = g == 0 ? c_gauss.DM[3] : c_gauss.DP[3];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        double q[5];
#pragma unroll
        for (int j = 0; j < 5; j++) q[j] = lineval(S, X, k, t - 2 + j, m);
        double a = cv[2] * q[2], e = cd[2] * q[2];
#pragma unroll
        for (int j = 0; j < 5; j++) {
            if (j == 2) continue;
            a = fma(cv[j], q[j], a);
            e = fma(cd[j], q[j], e);
        }
        v[k] = a; d[k] = e;
    }
    if (X <= 1 && nonphysical<4>(P.gamma, v)) {
#pragma unroll
        for (int k = 0; k < 4; k++) { v[k] = lineval(S, X, k, t, m); d[k] = 0.0; }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) d[k] = d[k] * S.inv_ht;
}

__device__ __forceinline__ void b_tang(const Params& P, const Sweep& S, Ctrl* ctrl, int stage, long long id)
{
    if (S.tlanes == 4) b_tang_x4(P, S, ctrl, stage, id);
    else b_tflags_x1(P, S, ctrl, stage, id);
}

__global__ void k_tang(const SolveDesc* __restrict__ D, int nb0, int stage)
{
    const SweepBlock b = sweep_block(nb0);
    const SolveDesc& d = *D;
    b_tang(d.P, d.sw[b.dir], d.ctrl, stage, b.id);
}


// The troubled tangential pass `it`: its pass X, segment (t, m), the eigenvectors at the face
// average (tangential direction) and the pass's 5 line values.
__device__ __forceinline__ void tang_ao_item(const Params& P, const Sweep& S, const double* __restrict__ W, uint32_t it,
                                             int& X, int& t, int& m, fx (*Lm)[4], fx (*Rm)[4], fx (*x)[4])
{
    X = it & 3;
    const long long tm = it >> 2;
    m = (int)(tm % S.nm); t = (int)(tm / S.nm);
    fx qs[4];
    const double* cl = cellp(P, S, W, t, m - 1);
    const double* cr = cellp(P, S, W, t, m);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        long long o = (long long)S.perm[k] * P.g.plane;
        qs[k] = (fx(ldc(cl + o, S)) + fx(ldc(cr + o, S))) * fx(0.5);
    }
    eigvec<4>(P.gamma, qs, 0.0, 1.0, Lm, Rm);
#pragma unroll
    for (int s = 0; s < 5; s++)
#pragma unroll
        for (int k = 0; k < 4; k++) x[s][k] = fx(lineval(S, X, k, t - 2 + s, m));
}

// The troubled tangential passes: one per lane (tang_ao) from kAoOneLaneMin items on, else one
// per aligned group of 4 lanes (tang_ao_x4, lane q computes and stores component q).  Free-order
// arithmetic (the outputs only feed the flux).  `lane`, `lanes`: this thread's index among, and
// the number of, the lanes working on the pass.
__device__ __forceinline__ void b_tang_ao(const Params& P, const Sweep& S, const double* __restrict__ W, const Ctrl* __restrict__ ctrl, long long lane, long long lanes)
{
    if (ctrl->done) return;
    unsigned int n = ctrl->cnt[S.dir][1];
    AOConst ak;
    for (int j = 0; j < 4; j++) ak.g[j] = P.g_ao[j];
    ak.g3inv = P.g3inv; ak.gr[0] = P.gr[0]; ak.gr[1] = P.gr[1]; ak.gr[2] = P.gr[2]; ak.eps = P.eps;
    // Gauss-point buffer: Q index 0 Wl, 1 Wlx, 2 Wly, 3 Wr, 4 Wrx, 5 Wry; pass X writes its values
    // to qv and (X = 0, 1) its tangential derivatives to qv + 2
    const long long plane = (long long)S.nt * S.nm;
    if (n >= kAoOneLaneMin) {
        for (unsigned int i = (unsigned int)lane; i < n; i += (unsigned int)lanes) {
            int X, t, m;
            fx Lm[4][4], Rm[4][4], x[5][4];
            tang_ao_item(P, S, W, rdc(S.itemsT + i, S), X, t, m, Lm, Rm, x);
            double v[4][2], d[4][2];
            tang_ao(Lm, Rm, x, ak, v, d);
            gp_positivity(P, S, t, m, X, v, d);
            const long long o = (long long)t * S.nm + m;
            const int qv = X == 0 ? 0 : (X == 1 ? 3 : (X == 2 ? 1 : 4));
#pragma unroll
            for (int k = 0; k < 4; k++)
#pragma unroll
                for (int g = 0; g < 2; g++) {
                    stc(S.gp + (long long)((g * 6 + qv) * 4 + k) * plane + o, v[k][g], S);
                    if (X <= 1) stc(S.gp + (long long)((g * 6 + qv + 2) * 4 + k) * plane + o, d[k][g] * S.inv_ht, S);
                }
        }
        return;
    }
    const int q = threadIdx.x & 3;
    const int lane0 = threadIdx.x & 28;
    const unsigned gmask = 0xFu << lane0;
    for (unsigned int i = (unsigned int)(lane >> 2); i < n; i += (unsigned int)(lanes >> 2)) {
        int X, t, m;
        fx Lm[4][4], Rm[4][4], x[5][4];
        tang_ao_item(P, S, W, rdc(S.itemsT + i, S), X, t, m, Lm, Rm, x);
        double vq[2], dq[2];
        tang_ao_x4(Lm, Rm, x, ak, gmask, vq, dq);
        if (X <= 1) {
            // positivity of the reconstructed Q^l, Q^r states (gp_positivity), on the gathered components
#pragma unroll
            for (int g = 0; g < 2; g++) {
                double Q[4];
#pragma unroll
                for (int k = 0; k < 4; k++) Q[k] = __shfl_sync(gmask, vq[g], lane0 + k);
                if (nonphysical<4>(P.gamma, Q)) { vq[g] = lineval(S, X, q, t, m); dq[g] = 0.0; }
            }
        }
        const long long o = (long long)t * S.nm + m;
        const int qv = X == 0 ? 0 : (X == 1 ? 3 : (X == 2 ? 1 : 4));
#pragma unroll
        for (int g = 0; g < 2; g++) {
            stc(S.gp + (long long)((g * 6 + qv) * 4 + q) * plane + o, vq[g], S);
            if (X <= 1) stc(S.gp + (long long)((g * 6 + qv + 2) * 4 + q) * plane + o, dq[g] * S.inv_ht, S);
        }
    }
}

// The tangential WENO-AO pass and the flux contain products that the compiler may fuse into FMAs
// (free-order arithmetic).  They are compiled once, as non-inlined functions on a solver
// descriptor in device memory, and called by both a solver's own kernels and the batched
// kernels: the same machine code, so batched and solo results are bit-identical by construction.
__device__ __noinline__ void tang_ao_nl(const SolveDesc& d, int dir, int stage, long long lane, long long lanes)
{
    b_tang_ao(d.P, d.sw[dir], stage == 0 ? d.W : d.Ws, d.ctrl, lane, lanes);
}

__global__ void k_tang_ao(const SolveDesc* __restrict__ D, int nb0, int stage)
{
    const SweepBlock b = sweep_block(nb0);
    tang_ao_nl(*D, b.dir, stage, b.id, b.lanes);
}


// ---------------------------------------------------------------- flux and update
constexpr int kFluxMaxBlock = 256;          // largest block of a flux launch (solo 64, batched up to 256)

template <int DIM, int STAGE, bool PRFIX>
__device__ __forceinline__ void b_flux(const Params& P, const Sweep& S, Ctrl* ctrl, long long id)
{
    if (ctrl->done) return;                   // the same for every thread of a block
    constexpr int NV = DIM + 2;
    const long long per = (long long)S.nt * S.nm;
    // 2D: warps in pairs, warp 2w on Gauss point 0 and warp 2w + 1 on Gauss point 1 of the same
    // 32 segments, so that the pair shares its stencil reads in cache and sums the segment flux
    int g = 0;
    long long o = id;
    if constexpr (DIM == 2) {
        const long long warp = id >> 5;
        g = (int)(warp & 1);
        o = ((warp >> 1) << 5) + (id & 31);
    }
    const bool valid = o < per;
    double o0[NV], o1[NV];
    if (valid) {
    double Wq[6][NV];
    if constexpr (DIM == 2) {
        if (S.tlanes == 4) {
            // small sweeps: every pass was reconstructed by k_tang / k_tang_ao
#pragma unroll
            for (int q = 0; q < 6; q++)
#pragma unroll
                for (int k = 0; k < NV; k++) Wq[q][k] = ldc(S.gp + (long long)((g * 6 + q) * 4 + k) * per + o, S);
        } else {
            // large sweeps: troubled passes from k_tang_ao, smooth ones reconstructed here
            const int t = (int)(o / S.nm), m = (int)(o % S.nm);
            const unsigned bits = rdc(S.flagT + o, S);
            constexpr int qx[4] = {0, 3, 1, 4};      // Q index: 0 Wl, 1 Wlx, 2 Wly, 3 Wr, 4 Wrx, 5 Wry
#pragma unroll
            for (int X = 0; X < 4; X++) {
                if ((bits >> X) & 1) {
#pragma unroll
                    for (int k = 0; k < NV; k++) {
                        Wq[qx[X]][k] = ldc(S.gp + (long long)((g * 6 + qx[X]) * 4 + k) * per + o, S);
                        if (X <= 1) Wq[qx[X] + 2][k] = ldc(S.gp + (long long)((g * 6 + qx[X] + 2) * 4 + k) * per + o, S);
                    }
                } else {
                    double v[4], d[4];
                    gp_linear_at(P, S, X, t, m, g, v, d);
#pragma unroll
                    for (int k = 0; k < NV; k++) {
                        Wq[qx[X]][k] = v[k];
                        if (X <= 1) Wq[qx[X] + 2][k] = d[k];
                    }
                }
            }
        }
    } else {
        long long plane = (long long)S.nlines * S.nm;
#pragma unroll
        for (int k = 0; k < NV; k++) {
            Wq[0][k] = ldc(S.line + (long long)(0 * NV + k) * plane + o, S);
            Wq[1][k] = ldc(S.line + (long long)(2 * NV + k) * plane + o, S);
            Wq[3][k] = ldc(S.line + (long long)(1 * NV + k) * plane + o, S);
            Wq[4][k] = ldc(S.line + (long long)(3 * NV + k) * plane + o, S);
            Wq[2][k] = 0.0; Wq[5][k] = 0.0;
        }
    }
    FluxConst fc;
    fc.gamma = P.gamma; fc.gm1 = P.gamma - 1.0; fc.K = P.K;
    fc.Kq = P.K + (double)DIM; fc.cslope = 4.0 / fc.Kq;
    fc.mu = P.mu; fc.c1 = P.c1; fc.c2 = P.c2; fc.viscous = P.viscous; fc.tau_zero = P.tau_zero;
    fc.prfix = P.prfix;
    if (!gks_flux<DIM, STAGE, PRFIX>(fc, Wq[0], Wq[1], Wq[2], Wq[3], Wq[4], Wq[5], ctrl->dt, o0, o1)) {
        // a non-physical state: the status is latched and the flux is a NaN, so that what the
        // failed step leaves behind does not depend on anything but the solve itself
        ctrl->status = HGKS_ENONPHYSICAL;
        const double nan = __longlong_as_double(0x7FF8000000000000LL);
#pragma unroll
        for (int k = 0; k < NV; k++) { o0[k] = nan; o1[k] = nan; }
    }
    }
    // the segment flux (Gauss weights 1/2): the Gauss point 1 warp hands its fluxes to its partner
    // through shared memory; stored per segment as [output][component][segment]
    constexpr int NO = STAGE == 0 ? 2 : 1;
    if constexpr (DIM == 2) {
        __shared__ double pair[kFluxMaxBlock / 2][2 * 4];
        const int slot = ((threadIdx.x >> 6) << 5) + (threadIdx.x & 31);
        if (g == 1 && valid) {
#pragma unroll
            for (int k = 0; k < NV; k++) {
                pair[slot][k] = o0[k];
                if (STAGE == 0) pair[slot][NV + k] = o1[k];
            }
        }
        __syncthreads();
        if (g == 1 || !valid) return;
#pragma unroll
        for (int k = 0; k < NV; k++) {
            o0[k] = fma(0.5, o0[k], 0.5 * pair[slot][k]);
            if (STAGE == 0) o1[k] = fma(0.5, o1[k], 0.5 * pair[slot][NV + k]);
        }
    } else {
        if (!valid) return;
    }
#pragma unroll
    for (int k = 0; k < NV; k++) {
        const int gk = S.perm[k];
        stc(S.flux + (long long)(0 * NV + gk) * per + o, o0[k], S);
        if (NO == 2) stc(S.flux + (long long)(1 * NV + gk) * per + o, o1[k], S);
    }
}

// Threads of a 2D flux launch for a sweep of `per` segments: two Gauss points per segment, the
// segments padded to whole warps (see b_flux).
inline long long flux_threads(int dim, long long per) { return dim == 2 ? 2 * ((per + 31) / 32) * 32 : per; }


template <int DIM, int STAGE, bool PRFIX>
__device__ __noinline__ void flux_nl(const SolveDesc& d, int dir, long long id)
{
    b_flux<DIM, STAGE, PRFIX>(d.P, d.sw[dir], d.ctrl, id);
}

// 64-thread blocks, at least 4 per SM: the register budget this leaves (up to 256 per thread at
// 8 warps per SM) lets the flux keep its working set in registers (measured 3.5 % faster than
// under a 128-thread bound at the same occupancy)
template <int DIM, int STAGE, bool PRFIX>
__global__ void __launch_bounds__(64, 4) k_flux(const SolveDesc* __restrict__ D, int nb0)
{
    const SweepBlock b = sweep_block(nb0);
    flux_nl<DIM, STAGE, PRFIX>(*D, b.dir, b.id);
}

// Stage 0: W* = W^n - dF(dt/2)/dx - dG(dt/2)/dy (Eq. (19)), Acc = W^n - d(dt F^n + dt^2/6 dF^n)/dx - ...
// Stage 1: W^{n+1} = Acc - d(dt^2/3 dF*)/dx - ... (Eqs. (20)-(22))
template <int DIM, int STAGE>
__device__ __forceinline__ void b_update(const Params& P, const Sweep& Sx, const Sweep& Sy, const double* __restrict__ Win, double* __restrict__ Wout, double* __restrict__ Acc, Ctrl* ctrl, long long id)
{
    if (ctrl->done) return;
    constexpr int NV = DIM + 2;
    const GridGeom& g = P.g;
    int rowsI = DIM == 2 ? g.ny : 1;
    long long n = (long long)rowsI * g.nx;
    if (id >= n) return;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    long long cell = g.origin + (long long)j * g.pitch + i;
    const double inv_dx = Sx.inv_hn, inv_dy = DIM == 2 ? Sy.inv_hn : 0.0;   // 1/dx, 1/dy (host-divided)
    long long perx = (long long)Sx.nt * Sx.nm, pery = DIM == 2 ? (long long)Sy.nt * Sy.nm : 0;
    long long ox = (long long)j * Sx.nm + i, oy = (long long)i * (DIM == 2 ? Sy.nm : 0) + j;
    double out[NV], acc[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double fx0[2], fx1[2], fy0[2] = {0, 0}, fy1[2] = {0, 0};
        // segment fluxes [output][component][segment] of the interfaces on either side
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const double* fb = Sx.flux;
            fx0[s] = ldc(fb + (long long)(0 * NV + k) * perx + ox + s, g);
            fx1[s] = STAGE == 0 ? ldc(fb + (long long)(1 * NV + k) * perx + ox + s, g) : 0.0;
            if constexpr (DIM == 2) {
                const double* gb = Sy.flux;
                fy0[s] = ldc(gb + (long long)(0 * NV + k) * pery + oy + s, g);
                fy1[s] = STAGE == 0 ? ldc(gb + (long long)(1 * NV + k) * pery + oy + s, g) : 0.0;
            }
        }
        if (STAGE == 0) {
            double w = ldc(Win + cell + (long long)k * g.plane, g);
            double ws = fma(-(fx0[1] - fx0[0]), inv_dx, w);
            double wa = fma(-(fx1[1] - fx1[0]), inv_dx, w);
            if (DIM == 2) { ws = fma(-(fy0[1] - fy0[0]), inv_dy, ws); wa = fma(-(fy1[1] - fy1[0]), inv_dy, wa); }
            out[k] = ws; acc[k] = wa;
        } else {
            double a = ldc(Acc + cell + (long long)k * g.plane, g);
            double wn = fma(-(fx0[1] - fx0[0]), inv_dx, a);
            if (DIM == 2) wn = fma(-(fy0[1] - fy0[0]), inv_dy, wn);
            out[k] = wn;
        }
    }
#pragma unroll
    for (int k = 0; k < NV; k++) {
        stc(Wout + cell + (long long)k * g.plane, out[k], g);
        if (STAGE == 0) stc(Acc + cell + (long long)k * g.plane, acc[k], g);
    }
    // rho > 0 and p > 0, the latter as rho E - |m|^2/2 > 0 (no division)
    double ke = DIM == 2 ? 0.5 * fma(out[1], out[1], out[2] * out[2]) : 0.5 * out[1] * out[1];
    double pr = fma(out[NV - 1], out[0], -ke);
    if (!(out[0] > 0.0) || !(pr > 0.0) || !isfinite(out[0]) || !isfinite(pr)) ctrl->status = HGKS_ENONPHYSICAL;
}

template <int DIM, int STAGE>
__global__ void k_update(Params P, Sweep Sx, Sweep Sy, const double* __restrict__ Win, double* __restrict__ Wout,
                         double* __restrict__ Acc, Ctrl* ctrl)
{
    b_update<DIM, STAGE>(P, Sx, Sy, Win, Wout, Acc, ctrl, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}


// ---------------------------------------------------------------- batched kernels
// One launch per kernel class covers the blocks of every solver of a batch: block b belongs
// to solver s with boff[s] <= b < boff[s+1] and runs that solver's kernel body on its local
// block index.  No block mixes solvers, so every result is bit-identical to stepping alone.
__device__ __forceinline__ int find_solve(const int* __restrict__ boff, int n, int b)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (boff[mid] <= b) lo = mid; else hi = mid;
    }
    return lo;
}

#define HGKS_BATCH_BLOCK()                                                              \
    const int s_ = find_solve(boff, n, (int)blockIdx.x);                                 \
    const SolveDesc& d = D[s_];                                                          \
    const long long lblk_ = (long long)blockIdx.x - boff[s_];                            \
    const long long nblk_ = (long long)(boff[s_ + 1] - boff[s_]);                         \
    const long long id = lblk_ * blockDim.x + threadIdx.x;                               \
    (void)nblk_; (void)id;

// sweep classes: the units are (solver, sweep) pairs, unit u = 2 s + dir; n counts solvers
#define HGKS_BATCH_SWEEP_BLOCK()                                                        \
    const int u_ = find_solve(boff, 2 * n, (int)blockIdx.x);                             \
    const SolveDesc& d = D[u_ >> 1];                                                     \
    const int dir = u_ & 1;                                                              \
    const long long lblk_ = (long long)blockIdx.x - boff[u_];                            \
    const long long nblk_ = (long long)(boff[u_ + 1] - boff[u_]);                         \
    const long long id = lblk_ * blockDim.x + threadIdx.x;                               \
    (void)nblk_; (void)id;

__global__ void kb_ctrl(const SolveDesc* __restrict__ D, int n, int what, const double* __restrict__ tend)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    Ctrl* ctrl = D[s].ctrl;
    if (what == 0) {                       // begin step
        ctrl->dtmin_bits = 0x7FF0000000000000ull;
        ctrl->cnt[0][0] = ctrl->cnt[0][1] = ctrl->cnt[1][0] = ctrl->cnt[1][1] = 0;
    } else if (what == 1) {                // dt final (as k_dt_final, t_end per solver)
        const Params& P = D[s].P;
        double t_end = tend[s];
        double tol = 1e-12 * (fabs(t_end) > 1.0 ? fabs(t_end) : 1.0);
        double dt = P.fixed_dt > 0.0 ? P.fixed_dt : P.cfl * __longlong_as_double((long long)ctrl->dtmin_bits);
        int done = ctrl->status != 0 || !(t_end - ctrl->t > tol);
        if (!done && ctrl->t + dt > t_end) dt = t_end - ctrl->t;
        if (!done && !(dt > 0.0 && dt < 1e300)) { ctrl->status = HGKS_ENONPHYSICAL; done = 1; }
        ctrl->dt = dt;
        ctrl->done = done;
    } else {                               // end step
        if (ctrl->done) return;
        ctrl->t += ctrl->dt;
        ctrl->last_dt = ctrl->dt;
        ctrl->steps += 1;
    }
}

__global__ void kb_dt(const SolveDesc* __restrict__ D, const int* __restrict__ boff, int n)
{
    HGKS_BATCH_BLOCK();
    if (d.P.fixed_dt > 0.0) return;
    b_dt(d.P, d.W, d.ctrl, d.h, id, nblk_ * blockDim.x);
}

__global__ void kb_ghost(const SolveDesc* __restrict__ D, const int* __restrict__ boff, int n, int stage, int axis)
{
    HGKS_BATCH_BLOCK();
    double* W = stage == 0 ? d.W : d.Ws;
    if (axis == 0) b_ghost_x(d.P, W, d.ctrl, id);
    else b_ghost_y(d.P, W, d.ctrl, stage, id);
}

template <int NV>
__global__ void kb_raw_nflags(const SolveDesc* __restrict__ D, const int* __restrict__ boff, int n, int stage)
{
    HGKS_BATCH_SWEEP_BLOCK();
    b_raw_nflags<NV>(d.P, d.sw[dir], stage == 0 ? d.W : d.Ws, d.ctrl, id);
}

template <int NV>
__global__ void kb_normal(const SolveDesc* __restrict__ D, const int* __restrict__ boff, int n, int stage)
{
    HGKS_BATCH_SWEEP_BLOCK();
    b_normal<NV>(d.P, d.sw[dir], stage == 0 ? d.W : d.Ws, d.ctrl, stage, id);
}

template <int NV>
__global__ void kb_normal_ao(const SolveDesc* __restrict__ D, const int* __restrict__ boff, int n, int stage)
{
    HGKS_BATCH_SWEEP_BLOCK();
    b_normal_ao<NV>(d.P, d.sw[dir], stage == 0 ? d.W : d.Ws, d.ctrl, id, nblk_ * blockDim.x);
}

__global__ void kb_raw_tflags(const SolveDesc* __restrict__ D, const int* __restrict__ boff, int n)
{
    HGKS_BATCH_SWEEP_BLOCK();
    b_raw_tflags(d.P, d.sw[dir], d.ctrl, id);
}

__global__ void kb_tang(const SolveDesc* __restrict__ D, const int* __restrict__ boff, int n, int stage)
{
    HGKS_BATCH_SWEEP_BLOCK();
    b_tang(d.P, d.sw[dir], d.ctrl, stage, id);
}

__global__ void kb_tang_ao(const SolveDesc* __restrict__ D, const int* __restrict__ boff, int n, int stage)
{
    HGKS_BATCH_SWEEP_BLOCK();
    tang_ao_nl(d, dir, stage, id, nblk_ * blockDim.x);
}

template <int DIM, int STAGE>
__global__ void __launch_bounds__(256) kb_flux(const SolveDesc* __restrict__ D, const int* __restrict__ boff, int n)
{
    HGKS_BATCH_SWEEP_BLOCK();
    if (d.P.prfix != 0.0) flux_nl<DIM, STAGE, true>(d, dir, id);
    else flux_nl<DIM, STAGE, false>(d, dir, id);
}

template <int DIM, int STAGE>
__global__ void kb_update(const SolveDesc* __restrict__ D, const int* __restrict__ boff, int n)
{
    HGKS_BATCH_BLOCK();
    if (STAGE == 0) b_update<DIM, 0>(d.P, d.sw[0], d.sw[1], d.W, d.Ws, d.Acc, d.ctrl, id);
    else b_update<DIM, 1>(d.P, d.sw[0], d.sw[1], d.Ws, d.W, d.Acc, d.ctrl, id);
}

inline unsigned int blocks_for(long long n, int tpb) { return (unsigned int)((n + tpb - 1) / tpb); }

// ---------------------------------------------------------------- FP64 rate probe
// Eight independent DFMA chains per thread: with 8 warps per SM scheduler slot the FP64 pipe
// never waits on a result, so the launch runs at the FMA issue rate of the device.  The sum is
// stored only under a condition the data never meet, which keeps the chains live.
__device__ double g_probe_sink;

__global__ void __launch_bounds__(256) k_dfma_probe(int iters, double seed)
{
    const double m = 0.9999999999, c = 1e-12;
    double a0 = seed + threadIdx.x * 1e-9, a1 = a0 + 1e-3, a2 = a0 + 2e-3, a3 = a0 + 3e-3;
    double a4 = a0 + 4e-3, a5 = a0 + 5e-3, a6 = a0 + 6e-3, a7 = a0 + 7e-3;
    for (int i = 0; i < iters; i++) {
        a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
        a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
    }
    const double s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == -1.0) g_probe_sink = s;
}

}  // namespace

cudaError_t launch_dfma_probe(cudaStream_t st, int blocks, int iters)
{
    k_dfma_probe<<<blocks, 256, 0, st>>>(iters, 1.0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- reciprocal check
// The flux's Newton-refined reciprocal (rcp_nr) against IEEE division, and its reciprocal square
// root (rsqrt_nr) against IEEE division by the IEEE square root, on n arguments spread
// log-uniformly over 1e-8..1e8 (both signs for the reciprocal; splitmix64 hashes of the index);
// the largest differences in units in the last place go to g_rcp_max_ulp[0], [1].
__device__ unsigned long long g_rcp_max_ulp[2];

__global__ void k_rcp_check(long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = (unsigned long long)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);      // [0, 1)
    double x = exp10(16.0 * u - 8.0);
    if (z & 1) x = -x;
    auto ulps = [](double a, double b) {
        const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
        return (unsigned long long)(ia > ib ? ia - ib : ib - ia);
    };
    atomicMax(&g_rcp_max_ulp[0], ulps(rcp_nr(x), 1.0 / x));
    const double ax = fabs(x);
    atomicMax(&g_rcp_max_ulp[1], ulps(rsqrt_nr(ax), 1.0 / sqrt(ax)));
}

cudaError_t rcp_check(long long n, unsigned long long* max_ulp)
{
    const unsigned long long zero[2] = {0, 0};
    cudaError_t e = cudaMemcpyToSymbol(g_rcp_max_ulp, zero, sizeof(zero));
    if (e != cudaSuccess) return e;
    k_rcp_check<<<(unsigned)((n + 255) / 256), 256>>>(n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyFromSymbol(max_ulp, g_rcp_max_ulp, 2 * sizeof(*max_ulp));
}

int debug_bounds_read(unsigned long long* count, unsigned long long* first)
{
#ifdef HGKS_DEBUG_BOUNDS
    cudaError_t e = cudaMemcpyFromSymbol(count, g_dbg_count, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(first, g_dbg_first, sizeof(unsigned long long));
    return e == cudaSuccess ? 1 : -1;
#else
    *count = 0;
    *first = 0;
    return 0;
#endif
}

int device_sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// ---------------------------------------------------------------- host: timing helpers
static cudaEvent_t take_event(hgks_solver* s)
{
    if (!s->event_pool.empty()) { cudaEvent_t e = s->event_pool.back(); s->event_pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// NVTX range around the enqueue of one kernel class (named as in kclass_names), so that a
// timeline tool attributes the launches to their class; free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

template <typename F>
static void timed(hgks_solver* s, int cls, int nkernels, F&& launch)
{
    NvtxRange range(kclass_names[cls]);
    s->launches += nkernels;
    if (!s->timing) { launch(); return; }
    cudaEvent_t a = take_event(s), b = take_event(s);
    cudaEventRecord(a, s->stream);
    launch();
    cudaEventRecord(b, s->stream);
    s->timers.push_back(TimerRec{cls, a, b});
}

// The sweep kernels of one stage, each class one launch over both sweeps (2D): nb[0] blocks for
// the x sweep, then nb[1] for the y sweep.
template <int DIM>
static void enqueue_sweeps(hgks_solver* s, int stage)
{
    const Params& P = s->P;
    cudaStream_t st = s->stream;
    const SolveDesc* D = s->d_self;
    constexpr int NV = DIM + 2;
    const int sms = device_sm_count();
    auto pair = [&](auto blocks, unsigned int* nb) {
        nb[0] = blocks(s->sw[0]);
        nb[1] = DIM == 2 ? blocks(s->sw[1]) : 0u;
        return nb[0] + nb[1];
    };
    // the compacted WENO-AO passes: a grid for 4 lanes per possible item, capped at 8 blocks per SM
    auto ao_blocks = [&](long long maxn) {
        unsigned int b = blocks_for(maxn, 128);
        return b > (unsigned)(sms * 8) ? (unsigned)(sms * 8) : b;
    };
    unsigned int nb[2];
    timed(s, KC_RAWN, 1, [&] {
        unsigned int g = pair([](const Sweep& S) { return blocks_for((long long)S.nlines * (S.nn + 4), TPB); }, nb);
        k_raw_nflags<NV><<<g, TPB, 0, st>>>(D, (int)nb[0], stage);
    });
    timed(s, KC_NORMAL, 1, [&] {
        unsigned int g = pair([](const Sweep& S) { return blocks_for((long long)S.nlines * S.nm, TPB); }, nb);
        k_normal<NV><<<g, TPB, 0, st>>>(D, (int)nb[0], stage);
    });
    timed(s, KC_NORMAL_AO, 1, [&] {
        unsigned int g = pair([&](const Sweep& S) { return ao_blocks((long long)S.nlines * S.nm * 2 * 4); }, nb);
        k_normal_ao<NV><<<g, 128, 0, st>>>(D, (int)nb[0], stage);
    });
    if constexpr (DIM == 2) {
        timed(s, KC_RAWT, 1, [&] {
            unsigned int g = pair([](const Sweep& S) { return blocks_for((long long)(S.nt + 2) * S.nm * S.tlanes, TPB); }, nb);
            k_raw_tflags<<<g, TPB, 0, st>>>(D, (int)nb[0]);
        });
        timed(s, KC_TANG, 1, [&] {
            unsigned int g = pair([](const Sweep& S) { return blocks_for((long long)S.nt * S.nm * S.tlanes, TPB); }, nb);
            k_tang<<<g, TPB, 0, st>>>(D, (int)nb[0], stage);
        });
        timed(s, KC_TANG_AO, 1, [&] {
            unsigned int g = pair([&](const Sweep& S) { return ao_blocks((long long)S.nt * S.nm * 4 * 4); }, nb);
            k_tang_ao<<<g, 128, 0, st>>>(D, (int)nb[0], stage);
        });
    }
    if (s->capture) {
        for (int d = 0; d < DIM; d++) {
            const Sweep& S = s->sw[d];
            size_t nbytes = (size_t)S.nlines * (S.nn + 2);
            cudaMemcpyAsync(s->cap[stage][d][0], S.flagN, nbytes, cudaMemcpyDeviceToDevice, st);
            if (DIM == 2) cudaMemcpyAsync(s->cap[stage][d][1], S.flagT, (size_t)S.nt * S.nm, cudaMemcpyDeviceToDevice, st);
        }
    }
    timed(s, KC_FLUX, 1, [&] {
        unsigned int g = pair([](const Sweep& S) { return blocks_for(flux_threads(DIM, (long long)S.nt * S.nm), 64); }, nb);
        const int n0 = (int)nb[0];
        if (P.prfix != 0.0) {
            if (stage == 0) k_flux<DIM, 0, true><<<g, 64, 0, st>>>(D, n0);
            else k_flux<DIM, 1, true><<<g, 64, 0, st>>>(D, n0);
        } else {
            if (stage == 0) k_flux<DIM, 0, false><<<g, 64, 0, st>>>(D, n0);
            else k_flux<DIM, 1, false><<<g, 64, 0, st>>>(D, n0);
        }
    });
}

template <int DIM>
static void enqueue_stage(hgks_solver* s, int stage)
{
    NvtxRange range(stage == 0 ? "S2O4 stage 1" : "S2O4 stage 2");
    const Params& P = s->P;
    cudaStream_t st = s->stream;
    double* Win = stage == 0 ? s->W : s->Ws;
    timed(s, KC_GHOST, DIM == 2 ? 2 : 1, [&] {
        int rowsI = DIM == 2 ? P.g.ny : 1;
        k_ghost_x<<<blocks_for((long long)P.g.nv * rowsI * NG * 2, TPB), TPB, 0, st>>>(P, Win, s->ctrl);
        if (DIM == 2) k_ghost_y<<<blocks_for((long long)P.g.nv * (P.g.nx + 2 * NG) * NG * 2, TPB), TPB, 0, st>>>(P, Win, s->ctrl, stage);
    });
    enqueue_sweeps<DIM>(s, stage);
    timed(s, KC_UPDATE, 1, [&] {
        long long n = (long long)(DIM == 2 ? P.g.ny : 1) * P.g.nx;
        if (stage == 0) k_update<DIM, 0><<<blocks_for(n, TPB), TPB, 0, st>>>(P, s->sw[0], s->sw[1], s->W, s->Ws, s->Acc, s->ctrl);
        else k_update<DIM, 1><<<blocks_for(n, TPB), TPB, 0, st>>>(P, s->sw[0], s->sw[1], s->Ws, s->W, s->Acc, s->ctrl);
    });
}

cudaError_t launch_step(hgks_solver* s, double t_end)
{
    NvtxRange range("hgks_step");
    const Params& P = s->P;
    cudaStream_t st = s->stream;
    double tol = 1e-12 * (fabs(t_end) > 1.0 ? fabs(t_end) : 1.0);
    double h = P.g.dim == 2 ? (P.g.dx < P.g.dy ? P.g.dx : P.g.dy) : P.g.dx;
    timed(s, KC_DT, P.fixed_dt > 0.0 ? 2 : 3, [&] {
        k_begin_step<<<1, 1, 0, st>>>(s->ctrl);
        if (!(P.fixed_dt > 0.0)) {
            long long n = (long long)(P.g.dim == 2 ? P.g.ny : 1) * P.g.nx;
            unsigned int b = blocks_for(n, TPB);
            unsigned int cap = (unsigned)device_sm_count() * 4;
            if (b > cap) b = cap;
            k_dt<<<b, TPB, 0, st>>>(P, s->W, s->ctrl, h);
        }
        k_dt_final<<<1, 1, 0, st>>>(s->ctrl, P.cfl, P.fixed_dt, t_end, tol);
    });
    if (P.g.dim == 2) { enqueue_stage<2>(s, 0); enqueue_stage<2>(s, 1); }
    else { enqueue_stage<1>(s, 0); enqueue_stage<1>(s, 1); }
    timed(s, KC_MISC, 1, [&] { k_end_step<<<1, 1, 0, st>>>(s->ctrl); });
    return cudaGetLastError();
}

// ---------------------------------------------------------------- host: batched step
const int kBatchTpbDefault[BK_COUNT] = {
    32, 256, 256, 256,        // ctrl, dt, ghost x, ghost y
    256,                      // raw normal flags
    256,                      // normal reconstruction
    128,                      // normal WENO-AO
    256,                      // raw tangential flags
    256,                      // tangential reconstruction
    128,                      // tangential WENO-AO
    128,                      // flux
    256                       // update
};

void batch_fill_desc(const hgks_solver* s, SolveDesc& d)
{
    d.P = s->P;
    d.sw[0] = s->sw[0];
    d.sw[1] = s->sw[1];
    d.W = s->W;
    d.Ws = s->Ws;
    d.Acc = s->Acc;
    d.ctrl = s->ctrl;
    d.h = s->P.g.dim == 2 ? (s->P.g.dx < s->P.g.dy ? s->P.g.dx : s->P.g.dy) : s->P.g.dx;
}

// Blocks of one unit of class c with t threads per block: solver d (sweep dir for the sweep classes).
static long long batch_unit_blocks(const SolveDesc& d, int dim, int c, int dir, int t)
{
    const GridGeom& g = d.P.g;
    const Sweep& S = d.sw[dir];
    const long long cells = (long long)(dim == 2 ? g.ny : 1) * g.nx;
    if (batch_sweep_class(c) && dir >= dim) return 0;          // 1D: no y sweep
    long long b = 0;
    switch (c) {
        case BK_CTRL: return 0;
        case BK_DT: b = (cells + (long long)t * 8 - 1) / ((long long)t * 8); break;
        case BK_GHX: b = blocks_for((long long)g.nv * (dim == 2 ? g.ny : 1) * NG * 2, t); break;
        case BK_GHY: if (dim != 2) return 0; b = blocks_for((long long)g.nv * (g.nx + 2 * NG) * NG * 2, t); break;
        case BK_RAWN: b = blocks_for((long long)S.nlines * (S.nn + 4), t); break;
        case BK_NORMAL: b = blocks_for((long long)S.nlines * S.nm, t); break;
        case BK_NAO: b = blocks_for((long long)S.nlines * S.nm * 2 * 4, t * 8); break;
        case BK_RAWT: if (dim != 2) return 0; b = blocks_for((long long)(S.nt + 2) * S.nm * S.tlanes, t); break;
        case BK_TANG: if (dim != 2) return 0; b = blocks_for((long long)S.nt * S.nm * S.tlanes, t); break;
        case BK_TAO: if (dim != 2) return 0; b = blocks_for((long long)S.nt * S.nm * 4 * 4, t * 8); break;
        case BK_FLUX: b = blocks_for(flux_threads(dim, (long long)S.nt * S.nm), t); break;
        case BK_UPD: b = blocks_for(cells, t); break;
    }
    return b < 1 ? 1 : b;
}

void batch_plan(const std::vector<const SolveDesc*>& descs, int dim, const int* tpb, BatchPlan& plan)
{
    const int n = (int)descs.size();
    const size_t stride = (size_t)2 * n + 1;
    plan.n = n;
    plan.dim = dim;
    for (int c = 0; c < BK_COUNT; c++) plan.tpb[c] = tpb[c];
    plan.boff.assign((size_t)BK_COUNT * stride, 0);
    for (int c = 0; c < BK_COUNT; c++) {
        int* bo = plan.boff.data() + (size_t)c * stride;
        const bool sw = batch_sweep_class(c);
        const int units = sw ? 2 * n : n;
        long long acc = 0;
        for (int u = 0; u < units; u++) {
            bo[u] = (int)acc;
            acc += sw ? batch_unit_blocks(*descs[u >> 1], dim, c, u & 1, tpb[c])
                      : batch_unit_blocks(*descs[u], dim, c, 0, tpb[c]);
        }
        bo[units] = (int)acc;
        plan.nblk[c] = c == BK_CTRL ? (int)blocks_for(n, tpb[c]) : (int)acc;
    }
}

cudaError_t batch_enqueue_step(const BatchPlan& plan, const SolveDesc* dd, const int* dboff, const double* dtend,
                               cudaStream_t st, cudaEvent_t* ev)
{
    NvtxRange range("hgks_batch_step");
    const int n = plan.n;
    const int dim = plan.dim;
    auto bo = [&](int c) { return dboff + (size_t)c * (2 * n + 1); };
    auto mark = [&](int c, int which) { if (ev) cudaEventRecord(ev[2 * c + which], st); };
    auto grid = [&](int c) { return (unsigned int)plan.nblk[c]; };
    auto tp = [&](int c) { return plan.tpb[c]; };
    const int tc = plan.tpb[BK_CTRL];
    kb_ctrl<<<grid(BK_CTRL), tc, 0, st>>>(dd, n, 0, dtend);
    mark(BK_DT, 0);
    if (grid(BK_DT)) kb_dt<<<grid(BK_DT), tp(BK_DT), 0, st>>>(dd, bo(BK_DT), n);
    mark(BK_DT, 1);
    kb_ctrl<<<grid(BK_CTRL), tc, 0, st>>>(dd, n, 1, dtend);
    for (int stage = 0; stage < 2; stage++) {
        mark(BK_GHX, 0);
        kb_ghost<<<grid(BK_GHX), tp(BK_GHX), 0, st>>>(dd, bo(BK_GHX), n, stage, 0);
        mark(BK_GHX, 1);
        if (dim == 2) {
            mark(BK_GHY, 0);
            kb_ghost<<<grid(BK_GHY), tp(BK_GHY), 0, st>>>(dd, bo(BK_GHY), n, stage, 1);
            mark(BK_GHY, 1);
        }
        // every sweep class: one launch over both sweeps of every solver
        mark(BK_RAWN, 0);
        if (dim == 2) kb_raw_nflags<4><<<grid(BK_RAWN), tp(BK_RAWN), 0, st>>>(dd, bo(BK_RAWN), n, stage);
        else kb_raw_nflags<3><<<grid(BK_RAWN), tp(BK_RAWN), 0, st>>>(dd, bo(BK_RAWN), n, stage);
        mark(BK_RAWN, 1);
        mark(BK_NORMAL, 0);
        if (dim == 2) kb_normal<4><<<grid(BK_NORMAL), tp(BK_NORMAL), 0, st>>>(dd, bo(BK_NORMAL), n, stage);
        else kb_normal<3><<<grid(BK_NORMAL), tp(BK_NORMAL), 0, st>>>(dd, bo(BK_NORMAL), n, stage);
        mark(BK_NORMAL, 1);
        mark(BK_NAO, 0);
        if (dim == 2) kb_normal_ao<4><<<grid(BK_NAO), tp(BK_NAO), 0, st>>>(dd, bo(BK_NAO), n, stage);
        else kb_normal_ao<3><<<grid(BK_NAO), tp(BK_NAO), 0, st>>>(dd, bo(BK_NAO), n, stage);
        mark(BK_NAO, 1);
        if (dim == 2) {
            mark(BK_RAWT, 0);
            kb_raw_tflags<<<grid(BK_RAWT), tp(BK_RAWT), 0, st>>>(dd, bo(BK_RAWT), n);
            mark(BK_RAWT, 1);
            mark(BK_TANG, 0);
            kb_tang<<<grid(BK_TANG), tp(BK_TANG), 0, st>>>(dd, bo(BK_TANG), n, stage);
            mark(BK_TANG, 1);
            mark(BK_TAO, 0);
            kb_tang_ao<<<grid(BK_TAO), tp(BK_TAO), 0, st>>>(dd, bo(BK_TAO), n, stage);
            mark(BK_TAO, 1);
        }
        mark(BK_FLUX, 0);
        const int tf = tp(BK_FLUX);
        if (dim == 2) {
            if (stage == 0) kb_flux<2, 0><<<grid(BK_FLUX), tf, 0, st>>>(dd, bo(BK_FLUX), n);
            else kb_flux<2, 1><<<grid(BK_FLUX), tf, 0, st>>>(dd, bo(BK_FLUX), n);
        } else {
            if (stage == 0) kb_flux<1, 0><<<grid(BK_FLUX), tf, 0, st>>>(dd, bo(BK_FLUX), n);
            else kb_flux<1, 1><<<grid(BK_FLUX), tf, 0, st>>>(dd, bo(BK_FLUX), n);
        }
        mark(BK_FLUX, 1);
        mark(BK_UPD, 0);
        const int tu = tp(BK_UPD);
        if (dim == 2) {
            if (stage == 0) kb_update<2, 0><<<grid(BK_UPD), tu, 0, st>>>(dd, bo(BK_UPD), n);
            else kb_update<2, 1><<<grid(BK_UPD), tu, 0, st>>>(dd, bo(BK_UPD), n);
        } else {
            if (stage == 0) kb_update<1, 0><<<grid(BK_UPD), tu, 0, st>>>(dd, bo(BK_UPD), n);
            else kb_update<1, 1><<<grid(BK_UPD), tu, 0, st>>>(dd, bo(BK_UPD), n);
        }
        mark(BK_UPD, 1);
    }
    kb_ctrl<<<grid(BK_CTRL), tc, 0, st>>>(dd, n, 3, dtend);
    return cudaGetLastError();
}

cudaError_t launch_set_time(hgks_solver* s, double t0)
{
    k_set_time<<<1, 1, 0, s->stream>>>(s->ctrl, t0);
    return cudaGetLastError();
}

}  // namespace hgks
