// hgks_api.cu -- the C ABI of the solver (declared in include/hgks.h): configuration
// checks, the device memory pool of a solver, state transfer, the step loop, parity
// hooks (flags), per-kernel timing and batched stepping.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "hgks.h"
#include "hgks_internal.h"

using namespace hgks;

namespace {

thread_local char g_create_err[512] = "";

void set_err(char* buf, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

double zeta1_scaled(int mode, double h)
{
    // Z1 = 17 zeta1 h^2 for the Step-1 test |D| <= Z1 (Sec. 2.3.1, Eq. (24))
    if (mode == HGKS_ZETA1_A) return 5.0 * h * h * h;
    if (mode == HGKS_ZETA1_C) return 5.0;
    return 5.0 * h;
}

double dof_K(int dim, double gam)
{
    // Sec. 2.1: K = (5 - 3 gamma)/(gamma - 1) + 1 in 2D; 1D: (3 - gamma)/(gamma - 1)
    if (dim == 2) return (5.0 - 3.0 * gam) / (gam - 1.0) + 1.0;
    return (3.0 - gam) / (gam - 1.0);
}

int validate(const hgks_config* c, char* err)
{
    if (!c) { set_err(err, "config is NULL"); return HGKS_EINVAL; }
    if (c->dim != 1 && c->dim != 2) { set_err(err, "dim must be 1 or 2 (got %d)", c->dim); return HGKS_EINVAL; }
    if (c->nx < NG) { set_err(err, "nx must be >= %d (got %d)", NG, c->nx); return HGKS_EINVAL; }
    if (c->dim == 1 && c->ny != 1) { set_err(err, "ny must be 1 in 1D"); return HGKS_EINVAL; }
    if (c->dim == 2 && c->ny < NG) { set_err(err, "ny must be >= %d (got %d)", NG, c->ny); return HGKS_EINVAL; }
    if ((long long)c->nx * c->ny > (1LL << 28)) { set_err(err, "grid too large (%d x %d)", c->nx, c->ny); return HGKS_EINVAL; }
    if (!(c->x1 > c->x0) || (c->dim == 2 && !(c->y1 > c->y0))) { set_err(err, "empty domain"); return HGKS_EINVAL; }
    if (!(c->gamma > 1.0) || !std::isfinite(c->gamma)) { set_err(err, "gamma must be > 1"); return HGKS_EINVAL; }
    if (!(c->fixed_dt > 0.0) && !(c->cfl > 0.0)) { set_err(err, "need cfl > 0 or fixed_dt > 0"); return HGKS_EINVAL; }
    if (c->viscous && !(c->mu > 0.0)) { set_err(err, "viscous run needs mu > 0"); return HGKS_EINVAL; }
    if (c->viscous && !(c->prandtl > 0.0 && std::isfinite(c->prandtl))) {
        set_err(err, "the Prandtl number must be > 0 (got %g)", c->prandtl);
        return HGKS_EINVAL;
    }
    if (c->c1 < 0.0 || c->c2 < 0.0) { set_err(err, "c1, c2 must be >= 0"); return HGKS_EINVAL; }
    int nb = c->dim == 2 ? 4 : 2;
    for (int k = 0; k < nb; k++)
        if (c->bc[k] < HGKS_BC_PERIODIC || c->bc[k] > HGKS_BC_SHOCK_TRACK) { set_err(err, "bad boundary type %d", c->bc[k]); return HGKS_EINVAL; }
    for (int k = 0; k < nb; k++) {
        if (c->bc[k] == HGKS_BC_SHOCK_WALL && k != 2) { set_err(err, "HGKS_BC_SHOCK_WALL is a y-lo boundary"); return HGKS_EINVAL; }
        if (c->bc[k] == HGKS_BC_SHOCK_TRACK && k < 2) { set_err(err, "HGKS_BC_SHOCK_TRACK is a y boundary"); return HGKS_EINVAL; }
        if (c->bc[k] >= HGKS_BC_INFLOW) {
            bool ok = c->bc_state[k][0] > 0.0;
            for (int j = 0; j < c->dim + 2; j++) ok = ok && std::isfinite(c->bc_state[k][j]);
            if (c->bc[k] == HGKS_BC_SHOCK_TRACK) {
                ok = ok && c->shock_pre[0] > 0.0 && std::isfinite(c->shock_cot) && std::isfinite(c->shock_speed);
                for (int j = 0; j < c->dim + 2; j++) ok = ok && std::isfinite(c->shock_pre[j]);
            }
            if (c->bc[k] >= HGKS_BC_SHOCK_WALL) ok = ok && std::isfinite(c->shock_x0);
            if (!ok) { set_err(err, "boundary %d needs finite prescribed states with rho > 0 (and shock data)", k); return HGKS_EINVAL; }
        }
    }
    for (int a = 0; a < nb; a += 2)
        if ((c->bc[a] == HGKS_BC_PERIODIC) != (c->bc[a + 1] == HGKS_BC_PERIODIC)) {
            set_err(err, "periodic boundaries must be paired on an axis"); return HGKS_EINVAL;
        }
    if (c->recon_mode < 0 || c->recon_mode > 2) { set_err(err, "bad recon_mode"); return HGKS_EINVAL; }
    if (c->zeta1_mode < 0 || c->zeta1_mode > 2) { set_err(err, "bad zeta1_mode"); return HGKS_EINVAL; }
    if (!(c->gamma_hi > 0.0 && c->gamma_hi < 1.0) || !(c->gamma_lo > 0.0 && c->gamma_lo < 1.0)) {
        set_err(err, "gamma_hi, gamma_lo must lie in (0, 1)"); return HGKS_EINVAL;
    }
    if (!(c->eps > 0.0)) { set_err(err, "eps must be > 0"); return HGKS_EINVAL; }
    return HGKS_OK;
}

struct Layout {
    size_t total;
    size_t off_W, off_Ws, off_Acc, off_ctrl, off_desc;
    size_t off_line[2], off_gp[2];
    size_t off_rawN[2], off_flagN[2], off_rawT[2], off_flagT[2], off_itemsN[2], off_itemsT[2], off_flux[2];
};

void fill_params(const hgks_config* c, Params& P)
{
    memset(&P, 0, sizeof(P));
    GridGeom& g = P.g;
    g.dim = c->dim; g.nx = c->nx; g.ny = c->dim == 2 ? c->ny : 1; g.nv = c->dim + 2;
    g.pitch = (int)align_up((size_t)c->nx + 2 * NG, 4);
    g.rows = c->dim == 2 ? c->ny + 2 * NG : 1;
    g.plane = (long long)g.pitch * g.rows;
    g.origin = (c->dim == 2 ? (long long)NG * g.pitch : 0) + NG;
    g.dx = (c->x1 - c->x0) / c->nx;
    g.dy = c->dim == 2 ? (c->y1 - c->y0) / c->ny : 1.0;
    P.gamma = c->gamma; P.K = dof_K(c->dim, c->gamma); P.mu = c->mu; P.c1 = c->c1; P.c2 = c->c2;
    P.cfl = c->cfl; P.fixed_dt = c->fixed_dt;
    P.viscous = c->viscous; P.tau_zero = c->tau_zero; P.recon_mode = c->recon_mode;
    P.prfix = (c->viscous && c->prandtl != 1.0) ? 1.0 / c->prandtl - 1.0 : 0.0;
    for (int k = 0; k < 4; k++) P.bc[k] = c->bc[k];
    P.x0 = c->x0; P.y0 = c->dim == 2 ? c->y0 : 0.0;
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++) P.bc_state[k][j] = c->bc_state[k][j];
    for (int j = 0; j < 4; j++) P.shock_pre[j] = c->shock_pre[j];
    P.shock_x0 = c->shock_x0; P.shock_cot = c->shock_cot; P.shock_speed = c->shock_speed;
    double ghi = c->gamma_hi, glo = c->gamma_lo;
    P.g_ao[3] = ghi;
    P.g_ao[0] = ((1.0 - ghi) * (1.0 - glo)) * 0.5;
    P.g_ao[2] = P.g_ao[0];
    P.g_ao[1] = (1.0 - ghi) * glo;
    P.g3inv = 1.0 / ghi;
    for (int j = 0; j < 3; j++) P.gr[j] = P.g_ao[j] / ghi;
    P.eps = c->eps;
}

void fill_sweeps(const hgks_config* c, const Params& P, Sweep* sw)
{
    const GridGeom& g = P.g;
    for (int d = 0; d < 2; d++) {
        Sweep& S = sw[d];
        memset(&S, 0, sizeof(S));
        if (d == 1 && c->dim == 1) continue;
        S.dir = d;
        S.nn = d == 0 ? g.nx : g.ny;
        S.nt = c->dim == 2 ? (d == 0 ? g.ny : g.nx) : 1;
        S.nm = S.nn + 1;
        S.nlines = c->dim == 2 ? S.nt + 6 : 1;
        // below ~4 warps per scheduler of segments, spread a segment over 4 lanes (shorter FP64
        // chains per thread); the results do not depend on the choice
        S.tlanes = (long long)S.nt * S.nm < 65536 ? 4 : 1;
        S.tlo = c->dim == 2 ? -3 : 0;
        S.sN = d == 0 ? 1 : g.pitch;
        S.sT = d == 0 ? g.pitch : 1;
        S.perm[0] = 0; S.perm[1] = d == 0 ? 1 : 2; S.perm[2] = d == 0 ? 2 : 1; S.perm[3] = 3;
        if (c->dim == 1) { S.perm[2] = 2; }
        double hn = d == 0 ? g.dx : g.dy, ht = d == 0 ? g.dy : g.dx;
        S.inv12hn = 1.0 / (12.0 * hn);
        S.inv_hn = 1.0 / hn;
        S.inv_ht = 1.0 / ht;
        S.Z1n = zeta1_scaled(c->zeta1_mode, hn);
        S.Z1t = zeta1_scaled(c->zeta1_mode, ht);
    }
}

Layout plan(const hgks_config* c, const Params& P, const Sweep* sw)
{
    Layout L;
    memset(&L, 0, sizeof(L));
    const size_t A = 256;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, A); return o; };
    size_t st = (size_t)P.g.nv * P.g.plane * sizeof(double);
    L.off_W = take(st); L.off_Ws = take(st); L.off_Acc = take(st);
    L.off_ctrl = take(sizeof(Ctrl));
    L.off_desc = take(sizeof(SolveDesc));
    int nd = c->dim;
    // every buffer a sweep writes is its own: the two sweeps of a stage run in the same launches
    for (int d = 0; d < nd; d++) {
        const Sweep& S = sw[d];
        L.off_line[d] = take((size_t)4 * P.g.nv * S.nlines * S.nm * sizeof(double));
        L.off_gp[d] = c->dim == 2 ? take((size_t)2 * 6 * 4 * S.nt * S.nm * sizeof(double)) : 0;
        L.off_rawN[d] = take((size_t)S.nlines * (S.nn + 4));
        L.off_flagN[d] = take((size_t)S.nlines * (S.nn + 2));
        L.off_itemsN[d] = take((size_t)S.nlines * S.nm * 2 * sizeof(uint32_t));
        if (c->dim == 2) {
            L.off_rawT[d] = take((size_t)(S.nt + 2) * S.nm);
            L.off_flagT[d] = take((size_t)S.nt * S.nm);
            L.off_itemsT[d] = take((size_t)S.nt * S.nm * 4 * sizeof(uint32_t));
        }
        // segment fluxes (the Gauss points already combined): [2 outputs][nv][nt][nn+1]
        L.off_flux[d] = take((size_t)2 * P.g.nv * S.nt * S.nm * sizeof(double));
    }
    L.total = off;
    return L;
}

#define CUDA_TRY(s, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            set_err((s)->err, "%s failed: %s", #call, cudaGetErrorString(e_));           \
            return HGKS_ECUDA;                                                             \
        }                                                                                  \
    } while (0)

int sync_ctrl(hgks_solver* s)
{
    CUDA_TRY(s, cudaMemcpyAsync(s->ctrl_host, s->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    return HGKS_OK;
}

}  // namespace

extern "C" int hgks_config_default(hgks_config* c)
{
    if (!c) return HGKS_EINVAL;
    memset(c, 0, sizeof(*c));
    c->dim = 2; c->nx = 64; c->ny = 64;
    c->x0 = 0.0; c->x1 = 1.0; c->y0 = 0.0; c->y1 = 1.0;
    c->gamma = 1.4; c->viscous = 0; c->mu = 0.0; c->prandtl = 1.0;
    c->c1 = 0.01; c->c2 = 1.0; c->cfl = 0.5; c->fixed_dt = 0.0; c->tau_zero = 0;
    for (int k = 0; k < 4; k++) c->bc[k] = HGKS_BC_PERIODIC;
    c->recon_mode = HGKS_RECON_HYBRID; c->zeta1_mode = HGKS_ZETA1_B;
    c->gamma_hi = 0.85; c->gamma_lo = 0.85; c->eps = 1e-8;
    return HGKS_OK;
}

extern "C" size_t hgks_footprint_bytes(const hgks_config* cfg)
{
    char err[512];
    if (validate(cfg, err) != HGKS_OK) return 0;
    Params P; Sweep sw[2];
    fill_params(cfg, P);
    fill_sweeps(cfg, P, sw);
    return plan(cfg, P, sw).total;
}

extern "C" int hgks_create_solver(const hgks_config* cfg, void* stream, hgks_solver** out)
{
    if (!out) { set_err(g_create_err, "out is NULL"); return HGKS_EINVAL; }
    *out = nullptr;
    int st = validate(cfg, g_create_err);
    if (st != HGKS_OK) return st;
    hgks_solver* s = new (std::nothrow) hgks_solver();
    if (!s) { set_err(g_create_err, "host allocation failed"); return HGKS_ENOMEM; }
    s->cfg = *cfg;
    s->stream = (cudaStream_t)stream;
    s->err[0] = 0;
    cudaGetDevice(&s->device);
    fill_params(cfg, s->P);
    fill_sweeps(cfg, s->P, s->sw);
    Layout L = plan(cfg, s->P, s->sw);
    cudaError_t e = cudaMalloc(&s->pool, L.total);
    if (e != cudaSuccess) {
        set_err(g_create_err, "cudaMalloc(%zu) failed: %s", L.total, cudaGetErrorString(e));
        delete s;
        return e == cudaErrorMemoryAllocation ? HGKS_ENOMEM : HGKS_ECUDA;
    }
    s->pool_bytes = L.total;
    e = cudaMallocHost(&s->ctrl_host, sizeof(Ctrl));
    if (e != cudaSuccess) {
        set_err(g_create_err, "cudaMallocHost failed: %s", cudaGetErrorString(e));
        cudaFree(s->pool); delete s; return HGKS_ENOMEM;
    }
    char* base = (char*)s->pool;
    s->P.g.lo = base;
    s->P.g.hi = base + L.total;
    s->W = (double*)(base + L.off_W);
    s->Ws = (double*)(base + L.off_Ws);
    s->Acc = (double*)(base + L.off_Acc);
    s->ctrl = (Ctrl*)(base + L.off_ctrl);
    for (int d = 0; d < cfg->dim; d++) {
        Sweep& S = s->sw[d];
        S.line = (double*)(base + L.off_line[d]);
        S.gp = cfg->dim == 2 ? (double*)(base + L.off_gp[d]) : nullptr;
        S.rawN = (uint8_t*)(base + L.off_rawN[d]);
        S.flagN = (uint8_t*)(base + L.off_flagN[d]);
        S.itemsN = (uint32_t*)(base + L.off_itemsN[d]);
        if (cfg->dim == 2) {
            S.rawT = (uint8_t*)(base + L.off_rawT[d]);
            S.flagT = (uint8_t*)(base + L.off_flagT[d]);
            S.itemsT = (uint32_t*)(base + L.off_itemsT[d]);
        }
        S.flux = (double*)(base + L.off_flux[d]);
        S.lo = base;
        S.hi = base + L.total;
    }
    memset(s->cap, 0, sizeof(s->cap));
    s->capture = 0;
    s->launches = 0;
    s->timing = 0;
    s->timer_ms.assign(KC_COUNT, 0.0);
    s->timer_calls.assign(KC_COUNT, 0);
    s->d_self = (SolveDesc*)(base + L.off_desc);
    SolveDesc self;
    batch_fill_desc(s, self);
    e = cudaMemsetAsync(s->pool, 0, L.total, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_self, &self, sizeof(SolveDesc), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = launch_set_time(s, 0.0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        set_err(g_create_err, "initialisation failed: %s", cudaGetErrorString(e));
        cudaFreeHost(s->ctrl_host); cudaFree(s->pool); delete s;
        return HGKS_ECUDA;
    }
    *out = s;
    return HGKS_OK;
}

extern "C" void hgks_destroy_solver(hgks_solver* s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    for (auto& r : s->timers) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : s->event_pool) cudaEventDestroy(e);
    for (int a = 0; a < 2; a++) for (int b = 0; b < 2; b++) for (int c = 0; c < 2; c++)
        if (s->cap[a][b][c]) cudaFree(s->cap[a][b][c]);
    cudaFreeHost(s->ctrl_host);
    cudaFree(s->pool);
    delete s;
}

extern "C" const char* hgks_last_error(const hgks_solver* s)
{
    return s ? s->err : g_create_err;
}

extern "C" int hgks_set_state(hgks_solver* s, const double* W, int on_device, double t0)
{
    if (!s || !W) return HGKS_EINVAL;
    const GridGeom& g = s->P.g;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int k = 0; k < g.nv; k++) {
        CUDA_TRY(s, cudaMemcpy2DAsync(s->W + g.origin + (long long)k * g.plane, (size_t)g.pitch * sizeof(double),
                                      W + (size_t)k * g.nx * g.ny, (size_t)g.nx * sizeof(double),
                                      (size_t)g.nx * sizeof(double), (size_t)g.ny, kind, s->stream));
    }
    CUDA_TRY(s, launch_set_time(s, t0));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    s->launches = 0;
    return HGKS_OK;
}

extern "C" int hgks_get_state(hgks_solver* s, double* W, int on_device)
{
    if (!s || !W) return HGKS_EINVAL;
    const GridGeom& g = s->P.g;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int k = 0; k < g.nv; k++) {
        CUDA_TRY(s, cudaMemcpy2DAsync(W + (size_t)k * g.nx * g.ny, (size_t)g.nx * sizeof(double),
                                      s->W + g.origin + (long long)k * g.plane, (size_t)g.pitch * sizeof(double),
                                      (size_t)g.nx * sizeof(double), (size_t)g.ny, kind, s->stream));
    }
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    return HGKS_OK;
}

extern "C" int hgks_step(hgks_solver* s, double t_end, int max_steps, int* steps_done)
{
    if (!s || max_steps < 0 || !std::isfinite(t_end)) return HGKS_EINVAL;
    if (!steps_done) {
        for (int n = 0; n < max_steps; n++) CUDA_TRY(s, launch_step(s, t_end));
        return HGKS_OK;
    }
    int st = sync_ctrl(s);
    if (st != HGKS_OK) return st;
    long long steps0 = s->ctrl_host->steps;
    int left = max_steps, chunk = 8;
    while (left > 0 && !s->ctrl_host->status) {
        int n = left < chunk ? left : chunk;
        for (int k = 0; k < n; k++) CUDA_TRY(s, launch_step(s, t_end));
        left -= n;
        st = sync_ctrl(s);
        if (st != HGKS_OK) return st;
        if (s->ctrl_host->done) break;
        if (chunk < 512) chunk *= 2;
    }
    *steps_done = (int)(s->ctrl_host->steps - steps0);
    if (s->ctrl_host->status) {
        set_err(s->err, "non-physical state (rho <= 0, p <= 0 or non-finite) detected at t = %.17g", s->ctrl_host->t);
        return s->ctrl_host->status;
    }
    return HGKS_OK;
}

extern "C" int hgks_get_time(hgks_solver* s, double* t)
{
    if (!s || !t) return HGKS_EINVAL;
    int st = sync_ctrl(s);
    if (st != HGKS_OK) return st;
    *t = s->ctrl_host->t;
    return HGKS_OK;
}

extern "C" int hgks_get_stats(hgks_solver* s, hgks_stats* out)
{
    if (!s || !out) return HGKS_EINVAL;
    int st = sync_ctrl(s);
    if (st != HGKS_OK) return st;
    const Ctrl& c = *s->ctrl_host;
    memset(out, 0, sizeof(*out));
    out->steps = c.steps; out->t = c.t; out->last_dt = c.last_dt; out->status = c.status;
    out->launches = s->launches;
    for (int a = 0; a < 2; a++) for (int b = 0; b < 2; b++) for (int k = 0; k < 2; k++) {
        out->troubled[a][b][k] = (long long)c.troubled[a][b][k];
        out->examined[a][b][k] = (long long)c.examined[a][b][k];
    }
    return HGKS_OK;
}

extern "C" size_t hgks_flags_size(const hgks_solver* s, int sweep, int kind)
{
    if (!s || sweep < 0 || sweep >= s->cfg.dim || kind < 0 || kind > 1) return 0;
    const Sweep& S = s->sw[sweep];
    if (kind == 0) return (size_t)S.nlines * (S.nn + 2);
    if (s->cfg.dim == 1) return 0;
    return (size_t)S.nt * S.nm;
}

extern "C" int hgks_set_flag_capture(hgks_solver* s, int enable)
{
    if (!s) return HGKS_EINVAL;
    if (enable) {
        for (int a = 0; a < 2; a++) for (int d = 0; d < s->cfg.dim; d++) for (int k = 0; k < 2; k++) {
            size_t n = hgks_flags_size(s, d, k);
            if (n && !s->cap[a][d][k]) {
                CUDA_TRY(s, cudaMalloc(&s->cap[a][d][k], n));
                CUDA_TRY(s, cudaMemsetAsync(s->cap[a][d][k], 0, n, s->stream));
            }
        }
    }
    s->capture = enable ? 1 : 0;
    return HGKS_OK;
}

extern "C" int hgks_get_flags(hgks_solver* s, int stage, int sweep, int kind, uint8_t* out)
{
    if (!s || !out || stage < 0 || stage > 1) return HGKS_EINVAL;
    size_t n = hgks_flags_size(s, sweep, kind);
    if (!n || !s->cap[stage][sweep][kind]) { set_err(s->err, "flags not captured (enable capture first)"); return HGKS_EINVAL; }
    CUDA_TRY(s, cudaMemcpyAsync(out, s->cap[stage][sweep][kind], n, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    return HGKS_OK;
}

extern "C" int hgks_set_timing(hgks_solver* s, int enable)
{
    if (!s) return HGKS_EINVAL;
    s->timing = enable ? 1 : 0;
    return HGKS_OK;
}

extern "C" int hgks_get_timing(hgks_solver* s, int cap, const char** names, double* ms, long long* calls)
{
    if (!s) return HGKS_EINVAL;
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    for (auto& r : s->timers) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            s->timer_ms[r.cls] += t;
            s->timer_calls[r.cls] += 1;
        }
        s->event_pool.push_back(r.a);
        s->event_pool.push_back(r.b);
    }
    s->timers.clear();
    int n = 0;
    for (int k = 0; k < KC_COUNT && n < cap; k++) {
        if (names) names[n] = kclass_names[k];
        if (ms) ms[n] = s->timer_ms[k];
        if (calls) calls[n] = s->timer_calls[k];
        n++;
    }
    return n;
}

// ---------------------------------------------------------------------------
// Batched execution: one launch per kernel class for all solvers of a batch.
struct hgks_batch {
    int n = 0, dim = 0, device = 0;
    cudaStream_t stream = nullptr;
    std::vector<hgks_solver*> solvers;
    SolveDesc* d_desc = nullptr;
    int* d_boff = nullptr;
    double* d_tend = nullptr;
    double* h_tend = nullptr;
    BatchPlan plan;
    int tuned = 0;
    cudaEvent_t ev[2 * BK_COUNT];
    cudaEvent_t tend_ev = nullptr;   // marks the last copy out of h_tend
    std::vector<cudaStream_t> others;   // the solvers' own streams other than the batch stream
    std::vector<cudaEvent_t> other_ev;  // one per entry of others: work enqueued there before a step
    cudaEvent_t done_ev = nullptr;      // the batch stream after the last enqueued step
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_stale = 0;                // the plan changed since the capture: recapture, update exec
    int cap = 0;                        // solvers the device arrays hold
    long long steps_enqueued = 0;
    char err[512];
};

namespace {

int batch_upload_plan(hgks_batch* b, const int* tpb)
{
    std::vector<SolveDesc> h(b->n);
    std::vector<const SolveDesc*> ptrs(b->n);
    for (int i = 0; i < b->n; i++) { batch_fill_desc(b->solvers[i], h[i]); ptrs[i] = &h[i]; }
    batch_plan(ptrs, b->dim, tpb, b->plan);
    cudaError_t e = cudaMemcpyAsync(b->d_boff, b->plan.boff.data(), b->plan.boff.size() * sizeof(int),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) { set_err(b->err, "plan upload failed: %s", cudaGetErrorString(e)); return HGKS_ECUDA; }
    if (b->exec) b->graph_stale = 1;    // the next graph step recaptures and updates the executable graph
    return HGKS_OK;
}

// (Re)build the per-stream ordering events for the solvers' own streams.
int batch_set_streams(hgks_batch* b)
{
    for (cudaEvent_t ev : b->other_ev) cudaEventDestroy(ev);
    b->others.clear();
    b->other_ev.clear();
    for (int i = 0; i < b->n; i++) {
        cudaStream_t st = b->solvers[i]->stream;
        bool seen = st == b->stream;
        for (cudaStream_t o : b->others) seen = seen || o == st;
        if (seen) continue;
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) { set_err(b->err, "event creation failed: %s", cudaGetErrorString(e)); return HGKS_ECUDA; }
        b->others.push_back(st);
        b->other_ev.push_back(ev);
    }
    return HGKS_OK;
}

// Device arrays for at least n solvers (grown by doubling; contents not kept).
int batch_reserve(hgks_batch* b, int n)
{
    if (n <= b->cap) return HGKS_OK;
    int cap = b->cap * 2 > n ? b->cap * 2 : n;
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_boff) cudaFree(b->d_boff);
    if (b->d_tend) cudaFree(b->d_tend);
    if (b->h_tend) cudaFreeHost(b->h_tend);
    b->d_desc = nullptr; b->d_boff = nullptr; b->d_tend = nullptr; b->h_tend = nullptr; b->cap = 0;
    cudaError_t e = cudaMalloc(&b->d_desc, sizeof(SolveDesc) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_boff, sizeof(int) * (size_t)BK_COUNT * (2 * (size_t)cap + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tend, sizeof(double) * cap);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_tend, sizeof(double) * cap);
    if (e != cudaSuccess) { set_err(b->err, "batch allocation failed: %s", cudaGetErrorString(e)); return HGKS_ENOMEM; }
    b->cap = cap;
    return HGKS_OK;
}

// Upload the descriptors of the current solvers, zero end times and the plan with block sizes tpb.
int batch_upload_members(hgks_batch* b, const int* tpb)
{
    std::vector<SolveDesc> h(b->n);
    for (int i = 0; i < b->n; i++) { batch_fill_desc(b->solvers[i], h[i]); b->h_tend[i] = 0.0; }
    cudaError_t e = cudaMemcpyAsync(b->d_desc, h.data(), sizeof(SolveDesc) * b->n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_tend, b->h_tend, sizeof(double) * b->n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->tend_ev, b->stream);
    if (e != cudaSuccess) { set_err(b->err, "batch upload failed: %s", cudaGetErrorString(e)); return HGKS_ECUDA; }
    return batch_upload_plan(b, tpb);
}

}  // namespace

extern "C" int hgks_batch_create(hgks_solver* const* solvers, int n, void* stream, hgks_batch** out)
{
    if (!out || n < 1 || !solvers) { set_err(g_create_err, "need at least one solver"); return HGKS_EINVAL; }
    *out = nullptr;
    int dev = -1;
    cudaGetDevice(&dev);
    int dim = 0;
    for (int i = 0; i < n; i++) {
        if (!solvers[i]) { set_err(g_create_err, "solver %d is NULL", i); return HGKS_EINVAL; }
        if (i == 0) dim = solvers[i]->cfg.dim;
        if (solvers[i]->cfg.dim != dim) { set_err(g_create_err, "all solvers of a batch must have the same dimension"); return HGKS_EINVAL; }
        if (solvers[i]->device != dev) { set_err(g_create_err, "solver %d lives on another device", i); return HGKS_EINVAL; }
    }
    hgks_batch* b = new (std::nothrow) hgks_batch();
    if (!b) return HGKS_ENOMEM;
    b->n = n; b->dim = dim; b->device = dev; b->stream = (cudaStream_t)stream;
    b->solvers.assign(solvers, solvers + n);
    b->err[0] = 0;
    for (int i = 0; i < n; i++) cudaStreamSynchronize(solvers[i]->stream);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 * BK_COUNT && e == cudaSuccess; k++) e = cudaEventCreate(&b->ev[k]);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->tend_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        set_err(g_create_err, "batch event creation failed: %s", cudaGetErrorString(e));
        hgks_batch_destroy(b);
        return HGKS_ECUDA;
    }
    int st = batch_reserve(b, n);
    if (st == HGKS_OK) st = batch_set_streams(b);
    if (st == HGKS_OK) st = batch_upload_members(b, kBatchTpbDefault);
    if (st != HGKS_OK) { set_err(g_create_err, "%s", b->err); hgks_batch_destroy(b); return st; }
    *out = b;
    return HGKS_OK;
}

extern "C" int hgks_batch_update(hgks_batch* b, hgks_solver* const* solvers, int n)
{
    if (!b || n < 1 || !solvers) { if (b) set_err(b->err, "need at least one solver"); return HGKS_EINVAL; }
    for (int i = 0; i < n; i++) {
        if (!solvers[i]) { set_err(b->err, "solver %d is NULL", i); return HGKS_EINVAL; }
        if (solvers[i]->cfg.dim != b->dim) { set_err(b->err, "all solvers of a batch must have the same dimension"); return HGKS_EINVAL; }
        if (solvers[i]->device != b->device) { set_err(b->err, "solver %d lives on another device", i); return HGKS_EINVAL; }
    }
    // the batch's earlier steps read the old descriptors: let them finish first
    CUDA_TRY(b, cudaStreamSynchronize(b->stream));
    for (int i = 0; i < n; i++) CUDA_TRY(b, cudaStreamSynchronize(solvers[i]->stream));
    int st = batch_reserve(b, n);
    if (st != HGKS_OK) return st;
    b->n = n;
    b->solvers.assign(solvers, solvers + n);
    st = batch_set_streams(b);
    if (st != HGKS_OK) return st;
    return batch_upload_members(b, b->plan.tpb);
}

extern "C" void hgks_batch_destroy(hgks_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (int k = 0; k < 2 * BK_COUNT; k++) if (b->ev[k]) cudaEventDestroy(b->ev[k]);
    if (b->tend_ev) cudaEventDestroy(b->tend_ev);
    if (b->done_ev) cudaEventDestroy(b->done_ev);
    for (cudaEvent_t ev : b->other_ev) cudaEventDestroy(ev);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_boff) cudaFree(b->d_boff);
    if (b->d_tend) cudaFree(b->d_tend);
    if (b->h_tend) cudaFreeHost(b->h_tend);
    delete b;
}

extern "C" int hgks_batch_step(hgks_batch* b, const double* t_end, int nsteps, int flags)
{
    if (!b || nsteps < 0) return HGKS_EINVAL;
    // work already enqueued on the solvers' own streams (set_state, ...) runs first
    for (size_t i = 0; i < b->others.size(); i++) {
        CUDA_TRY(b, cudaEventRecord(b->other_ev[i], b->others[i]));
        CUDA_TRY(b, cudaStreamWaitEvent(b->stream, b->other_ev[i], 0));
    }
    if (t_end) {
        for (int i = 0; i < b->n; i++)
            if (!std::isfinite(t_end[i])) { set_err(b->err, "t_end[%d] is not finite", i); return HGKS_EINVAL; }
        // the pinned staging array may still be read by the previous call's copy: wait for it
        CUDA_TRY(b, cudaEventSynchronize(b->tend_ev));
        for (int i = 0; i < b->n; i++) b->h_tend[i] = t_end[i];
        CUDA_TRY(b, cudaMemcpyAsync(b->d_tend, b->h_tend, sizeof(double) * b->n, cudaMemcpyHostToDevice, b->stream));
        CUDA_TRY(b, cudaEventRecord(b->tend_ev, b->stream));
    }
    int left = nsteps;
    if ((flags & HGKS_BATCH_AUTOTUNE) && !b->tuned && left > 0) {
        // try three block sizes per kernel class on live steps (the per-item arithmetic does not
        // depend on the block size), then keep the fastest size of each class.  One untimed step
        // with the default sizes first loads every batched kernel.
        CUDA_TRY(b, batch_enqueue_step(b->plan, b->d_desc, b->d_boff, b->d_tend, b->stream, nullptr));
        b->steps_enqueued++;
        left--;
        static const int cand_small[3] = {64, 128, 256};
        static const int cand_big[3] = {128, 256, 512};
        double best_ms[BK_COUNT];
        int best_tpb[BK_COUNT];
        for (int c = 0; c < BK_COUNT; c++) { best_ms[c] = 1e300; best_tpb[c] = kBatchTpbDefault[c]; }
        for (int k = 0; k < 3 && left > 0; k++) {
            int tpb[BK_COUNT];
            for (int c = 0; c < BK_COUNT; c++) {
                bool heavy_regs = c == BK_FLUX || c == BK_NAO || c == BK_TAO;
                tpb[c] = c == BK_CTRL ? 32 : (heavy_regs ? cand_small[k] : cand_big[k]);
            }
            int st = batch_upload_plan(b, tpb);
            if (st != HGKS_OK) return st;
            CUDA_TRY(b, batch_enqueue_step(b->plan, b->d_desc, b->d_boff, b->d_tend, b->stream, b->ev));
            CUDA_TRY(b, cudaStreamSynchronize(b->stream));
            b->steps_enqueued++;
            left--;
            for (int c = 0; c < BK_COUNT; c++) {
                // classes without launches in this dimension (and the control kernels) carry no events
                if (c == BK_CTRL || b->plan.nblk[c] == 0) continue;
                float ms = 0.0f;
                cudaError_t qe = cudaEventElapsedTime(&ms, b->ev[2 * c], b->ev[2 * c + 1]);
                if (qe != cudaSuccess) { (void)cudaGetLastError(); continue; }
                if (ms < best_ms[c]) {
                    best_ms[c] = ms;
                    best_tpb[c] = tpb[c];
                }
            }
        }
        int st = batch_upload_plan(b, best_tpb);
        if (st != HGKS_OK) return st;
        b->tuned = 1;
    }
    const bool use_graph = (flags & HGKS_BATCH_GRAPH) && b->stream != nullptr;
    for (int k = 0; k < left; k++) {
        if (use_graph) {
            if (!b->exec || b->graph_stale) {
                cudaGraph_t g = nullptr;
                CUDA_TRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = batch_enqueue_step(b->plan, b->d_desc, b->d_boff, b->d_tend, b->stream, nullptr);
                cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
                if (e != cudaSuccess || e2 != cudaSuccess) {
                    set_err(b->err, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
                    return HGKS_ECUDA;
                }
                // the same kernels in the same order with new grids and arguments: update the
                // executable graph in place when the driver accepts it, else instantiate anew
                bool updated = false;
                if (b->exec) {
                    cudaGraphExecUpdateResultInfo info;
                    updated = cudaGraphExecUpdate(b->exec, g, &info) == cudaSuccess;
                    if (!updated) {
                        (void)cudaGetLastError();
                        cudaGraphExecDestroy(b->exec);
                        b->exec = nullptr;
                    }
                }
                if (b->graph) cudaGraphDestroy(b->graph);
                b->graph = g;
                b->graph_stale = 0;
                if (!updated) CUDA_TRY(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
            }
            CUDA_TRY(b, cudaGraphLaunch(b->exec, b->stream));
        } else {
            CUDA_TRY(b, batch_enqueue_step(b->plan, b->d_desc, b->d_boff, b->d_tend, b->stream, nullptr));
        }
        b->steps_enqueued++;
    }
    // and work enqueued on them later (get_state, ...) runs after the batched steps
    if (!b->others.empty()) {
        CUDA_TRY(b, cudaEventRecord(b->done_ev, b->stream));
        for (cudaStream_t o : b->others) CUDA_TRY(b, cudaStreamWaitEvent(o, b->done_ev, 0));
    }
    return HGKS_OK;
}

extern "C" int hgks_batch_sync(hgks_batch* b, int* n_active, int* n_failed)
{
    if (!b) return HGKS_EINVAL;
    for (int i = 0; i < b->n; i++)
        CUDA_TRY(b, cudaMemcpyAsync(b->solvers[i]->ctrl_host, b->solvers[i]->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(b, cudaStreamSynchronize(b->stream));
    int active = 0, failed = 0;
    for (int i = 0; i < b->n; i++) {
        const Ctrl& c = *b->solvers[i]->ctrl_host;
        double te = b->h_tend[i];
        double tol = 1e-12 * (fabs(te) > 1.0 ? fabs(te) : 1.0);
        if (c.status) failed++;
        else if (te - c.t > tol) active++;
    }
    if (n_active) *n_active = active;
    if (n_failed) *n_failed = failed;
    return HGKS_OK;
}

extern "C" int hgks_batch_status(const hgks_batch* b, double* t, int* status, long long* steps)
{
    if (!b) return HGKS_EINVAL;
    for (int i = 0; i < b->n; i++) {
        const Ctrl& c = *b->solvers[i]->ctrl_host;
        if (t) t[i] = c.t;
        if (status) status[i] = c.status;
        if (steps) steps[i] = c.steps;
    }
    return HGKS_OK;
}

extern "C" int hgks_batch_info(const hgks_batch* b, int* tpb, int cap, long long* steps_enqueued)
{
    if (!b) return HGKS_EINVAL;
    int m = cap < (int)BK_COUNT ? cap : (int)BK_COUNT;
    for (int c = 0; c < m && tpb; c++) tpb[c] = b->plan.tpb[c];
    if (steps_enqueued) *steps_enqueued = b->steps_enqueued;
    return (int)BK_COUNT;
}

extern "C" const char* hgks_batch_last_error(const hgks_batch* b) { return b ? b->err : g_create_err; }

// ---------------------------------------------------------------------------
// Debug build: out-of-range accesses the kernels skipped.
extern "C" int hgks_debug_bounds(unsigned long long* count, unsigned long long* first_address)
{
    if (!count || !first_address) return HGKS_EINVAL;
    int r = debug_bounds_read(count, first_address);
    if (r < 0) { set_err(g_create_err, "hgks_debug_bounds: reading the counters failed"); return HGKS_ECUDA; }
    return r;
}

// ---------------------------------------------------------------------------
// FP64 rate of the current device (the denominator of the benchmark's roofline).
extern "C" int hgks_probe_fp64(void* stream, double* tflops, double* ms, int* sms)
{
    if (!tflops) return HGKS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int nsm = device_sm_count();
    const int blocks = nsm * 8, iters = 16384;     // 8 blocks of 256 threads per SM: 64 warps, ~0.3 s
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = launch_dfma_probe(st, blocks, 64);     // loads the kernel
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    for (int r = 0; r < 4 && e == cudaSuccess; r++) e = launch_dfma_probe(st, blocks, iters);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) {
        set_err(g_create_err, "hgks_probe_fp64: %s", cudaGetErrorString(e));
        return HGKS_ECUDA;
    }
    const double flop = 4.0 * blocks * 256.0 * iters * 8.0 * 2.0;
    *tflops = flop / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    if (sms) *sms = nsm;
    return HGKS_OK;
}

extern "C" int hgks_check_reciprocal(long long n, unsigned long long* max_ulp)
{
    if (n < 1 || !max_ulp) return HGKS_EINVAL;
    cudaError_t e = rcp_check(n, max_ulp);
    if (e != cudaSuccess) {
        set_err(g_create_err, "hgks_check_reciprocal: %s", cudaGetErrorString(e));
        return HGKS_ECUDA;
    }
    return HGKS_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free single step (hgks_step_noalloc): the same S2O4 step as a solver
// performs, with every intermediate buffer carved out of one file-scope device
// array instead of a cudaMalloc'd pool.  The array is part of the library image,
// so every GPU that loads the library keeps HGKS_NOALLOC_SCRATCH_BYTES of it
// until the process exits.
#include <mutex>

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[HGKS_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
void* g_noalloc_addr[kNoallocMaxDevices];   // device address of the array, per device (host stand-in is not usable)
std::mutex g_noalloc_mutex;

}  // namespace

extern "C" int hgks_step_noalloc(const hgks_config* cfg, const double* W_in, double* W_out, int* status, void* stream)
{
    int st = validate(cfg, g_create_err);
    if (st != HGKS_OK) return st;
    if (!W_in || !W_out) { set_err(g_create_err, "W_in and W_out must be device pointers"); return HGKS_EINVAL; }
    Params P;
    Sweep sw[2];
    fill_params(cfg, P);
    fill_sweeps(cfg, P, sw);
    Layout L = plan(cfg, P, sw);
    if (L.total > (size_t)HGKS_NOALLOC_SCRATCH_BYTES) {
        set_err(g_create_err, "grid needs %zu bytes of scratch; the static scratch of hgks_step_noalloc holds %zu",
                L.total, (size_t)HGKS_NOALLOC_SCRATCH_BYTES);
        return HGKS_EINVAL;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
        set_err(g_create_err, "no usable current CUDA device (%s)", cudaGetErrorString(e));
        return HGKS_ECUDA;
    }
    void* base = nullptr;
    {
        // one-time set-up per device, with that device current: the address of the array
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                set_err(g_create_err, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
                return HGKS_ECUDA;
            }
            g_noalloc_addr[dev] = p;
        }
        base = g_noalloc_addr[dev];
    }
    // a solver object on the stack whose buffers all live in the static array
    hgks_solver s;
    s.cfg = *cfg;
    s.P = P;
    s.sw[0] = sw[0];
    s.sw[1] = sw[1];
    s.stream = (cudaStream_t)stream;
    s.device = dev;
    s.pool = base;
    s.pool_bytes = L.total;
    s.ctrl_host = nullptr;
    memset(s.cap, 0, sizeof(s.cap));
    s.capture = 0;
    s.launches = 0;
    s.timing = 0;
    s.err[0] = 0;
    char* b = (char*)base;
    s.P.g.lo = b;
    s.P.g.hi = b + L.total;
    s.W = (double*)(b + L.off_W);
    s.Ws = (double*)(b + L.off_Ws);
    s.Acc = (double*)(b + L.off_Acc);
    s.ctrl = (Ctrl*)(b + L.off_ctrl);
    for (int d = 0; d < cfg->dim; d++) {
        Sweep& S = s.sw[d];
        S.line = (double*)(b + L.off_line[d]);
        S.gp = cfg->dim == 2 ? (double*)(b + L.off_gp[d]) : nullptr;
        S.rawN = (uint8_t*)(b + L.off_rawN[d]);
        S.flagN = (uint8_t*)(b + L.off_flagN[d]);
        S.itemsN = (uint32_t*)(b + L.off_itemsN[d]);
        if (cfg->dim == 2) {
            S.rawT = (uint8_t*)(b + L.off_rawT[d]);
            S.flagT = (uint8_t*)(b + L.off_flagT[d]);
            S.itemsT = (uint32_t*)(b + L.off_itemsT[d]);
        }
        S.flux = (double*)(b + L.off_flux[d]);
        S.lo = b;
        S.hi = b + L.total;
    }
    const GridGeom& g = s.P.g;
    s.d_self = (SolveDesc*)(b + L.off_desc);
    SolveDesc self;
    batch_fill_desc(&s, self);
    // the array keeps the previous call's contents: start every call from zero
    e = cudaMemsetAsync(base, 0, L.total, s.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.d_self, &self, sizeof(SolveDesc), cudaMemcpyHostToDevice, s.stream);
    for (int k = 0; k < g.nv && e == cudaSuccess; k++)
        e = cudaMemcpy2DAsync(s.W + g.origin + (long long)k * g.plane, (size_t)g.pitch * sizeof(double),
                              W_in + (size_t)k * g.nx * g.ny, (size_t)g.nx * sizeof(double),
                              (size_t)g.nx * sizeof(double), (size_t)g.ny, cudaMemcpyDeviceToDevice, s.stream);
    if (e == cudaSuccess) e = launch_set_time(&s, 0.0);
    if (e == cudaSuccess) e = launch_step(&s, 1e300);
    for (int k = 0; k < g.nv && e == cudaSuccess; k++)
        e = cudaMemcpy2DAsync(W_out + (size_t)k * g.nx * g.ny, (size_t)g.nx * sizeof(double),
                              s.W + g.origin + (long long)k * g.plane, (size_t)g.pitch * sizeof(double),
                              (size_t)g.nx * sizeof(double), (size_t)g.ny, cudaMemcpyDeviceToDevice, s.stream);
    // the status the step latched on the device (0 or HGKS_ENONPHYSICAL), for the caller to read
    // once the stream has passed this point; no host wait here
    if (status && e == cudaSuccess)
        e = cudaMemcpyAsync(status, &s.ctrl->status, sizeof(int), cudaMemcpyDefault, s.stream);
    if (e != cudaSuccess) {
        set_err(g_create_err, "hgks_step_noalloc: %s", cudaGetErrorString(e));
        return HGKS_ECUDA;
    }
    return HGKS_OK;
}
