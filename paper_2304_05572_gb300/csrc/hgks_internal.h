// hgks_internal.h -- private declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hgks.h"

namespace hgks {

constexpr int NG = 4;            // ghost layers: the widest stencil (a Step-4 spread of 5-cell tests) reaches 4 cells
constexpr int MAXNV = 4;

// Device control block of one solver: time, dt, status and counters.  All
// step logic that would otherwise need a host round trip lives here.
struct Ctrl {
    double t;
    double dt;
    double last_dt;
    unsigned long long dtmin_bits;   // atomicMin over positive doubles as ordered integers
    int done;                        // 1: the current step does nothing (t reached t_end or error latched)
    int status;                      // 0 or HGKS_ENONPHYSICAL
    long long steps;
    unsigned int cnt[2][2];          // AO work-list lengths [sweep][0 normal, 1 tangential]
    unsigned long long troubled[2][2][2];
    unsigned long long examined[2][2][2];
};

struct GridGeom {
    int dim, nx, ny, nv;
    int pitch;                 // padded row length in doubles (nx + 2 NG rounded up)
    int rows;                  // padded rows (ny + 2 NG in 2D, 1 in 1D)
    long long plane;           // pitch * rows
    long long origin;          // offset of interior cell (0, 0)
    double dx, dy;
    const char* lo;            // the solver's device buffers: [lo, hi) (checked by the debug build)
    const char* hi;
};

// One sweep in its local frame: n = index normal to the interfaces, t = tangential index.
struct Sweep {
    int dir;                   // 0: x-interfaces, 1: y-interfaces
    int nn, nt;                // cells normal / tangential
    int nm;                    // interfaces per line (nn + 1)
    int nlines;                // lines with normal reconstruction (nt + 6 in 2D, 1 in 1D)
    int tlanes;                // lanes per segment of the tangential kernels: 4 for small sweeps, else 1
    int tlo;                   // first line index (-3 in 2D, 0 in 1D)
    long long sN, sT;          // state strides for +1 in n / t
    int perm[4];               // local component -> global component
    double inv12hn, inv_hn, inv_ht, Z1n, Z1t;
    uint8_t* rawN;             // [nlines][nn + 4]   raw normal flags, cells -2..nn+1
    uint8_t* flagN;            // [nlines][nn + 2]   final normal flags, cells -1..nn
    double* line;              // [4][nv][nlines][nm] Q^l, Q^r, Q^l_n, Q^r_n
    uint8_t* rawT;             // [nt + 4][nm]       raw tangential flag bits, lines -2..nt+1
    uint8_t* flagT;            // [nt][nm]           final tangential flag bits
    double* gp;                // [2][6][nv][nt][nm] Gauss-point states
    double* flux;              // [2][nv][nt][nm] segment fluxes (Gauss points combined; global component order)
    uint32_t* itemsN;          // AO work list, normal pass
    uint32_t* itemsT;          // AO work list, tangential passes
    const char* lo;            // the solver's device buffers: [lo, hi) (checked by the debug build)
    const char* hi;
};

struct Params {
    GridGeom g;
    double gamma, K, mu, c1, c2, cfl, fixed_dt;
    double prfix;                  // 1/Pr - 1 (viscous runs with Pr != 1), else 0
    int viscous, tau_zero, recon_mode;
    int bc[4];
    double g_ao[4], g3inv, gr[3], eps;
    double x0, y0;                 // domain origin (ghost-cell centres of the prescribed boundaries)
    double bc_state[4][4];         // prescribed boundary states [side][global component]
    double shock_pre[4];
    double shock_x0, shock_cot, shock_speed;
};

struct TimerRec { int cls; cudaEvent_t a, b; };

// One solver as seen by the batched kernels (device array, one entry per solver).
struct SolveDesc {
    Params P;
    Sweep sw[2];
    double* W;
    double* Ws;
    double* Acc;
    Ctrl* ctrl;
    double h;          // min(dx, dy): the CFL length
};

// Kernel classes of a batched step, one launch each per stage.  The sweep classes (BK_RAWN to
// BK_FLUX) cover both sweeps of every solver: their units are (solver s, sweep d), unit 2 s + d.
enum BatchClass {
    BK_CTRL = 0, BK_DT, BK_GHX, BK_GHY,
    BK_RAWN, BK_NORMAL, BK_NAO, BK_RAWT, BK_TANG, BK_TAO, BK_FLUX,
    BK_UPD, BK_COUNT
};

inline bool batch_sweep_class(int c) { return c >= BK_RAWN && c <= BK_FLUX; }

struct BatchPlan {
    int n = 0, dim = 0;
    int tpb[BK_COUNT];
    int nblk[BK_COUNT];            // total blocks of each class
    std::vector<int> boff;         // [BK_COUNT][2 n + 1] block offsets per unit (a solver, or a
                                   // solver's sweep for the sweep classes)
};

}  // namespace hgks

struct hgks_solver {
    hgks_config cfg;
    hgks::Params P;
    cudaStream_t stream;
    int device;
    hgks::Sweep sw[2];
    double* W;       // padded state W^n (and W^{n+1})
    double* Ws;      // padded W*
    double* Acc;     // padded accumulator of stage 1
    hgks::Ctrl* ctrl;        // device
    hgks::Ctrl* ctrl_host;   // pinned mirror
    hgks::SolveDesc* d_self; // device copy of this solver's descriptor (the kernels shared with batches read it)
    void* pool;              // single device allocation holding all buffers
    size_t pool_bytes;
    uint8_t* cap[2][2][2];   // captured flags [stage][sweep][kind]
    int capture;
    long long launches;      // kernels enqueued since set_state (host count)
    int timing;
    std::vector<hgks::TimerRec> timers;
    std::vector<cudaEvent_t> event_pool;
    std::vector<double> timer_ms;
    std::vector<long long> timer_calls;
    char err[512];
};

namespace hgks {

// kernel classes for timing
enum KClass { KC_GHOST = 0, KC_DT, KC_RAWN, KC_NORMAL, KC_NORMAL_AO, KC_RAWT, KC_TANG, KC_TANG_AO, KC_FLUX, KC_UPDATE, KC_MISC, KC_COUNT };
extern const char* kclass_names[KC_COUNT];

// host-side launchers (hgks_kernels.cu); all enqueue on s->stream
cudaError_t launch_step(hgks_solver* s, double t_end);
cudaError_t launch_set_time(hgks_solver* s, double t0);
int device_sm_count();
// the debug build's count of out-of-range accesses and the first such address (returns 1), or 0
// without the checks compiled in, -1 if the device read failed
int debug_bounds_read(unsigned long long* count, unsigned long long* first);
// FP64 rate probe: `blocks` blocks of 256 threads, 8 DFMA chains of `iters` steps per thread
cudaError_t launch_dfma_probe(cudaStream_t st, int blocks, int iters);
cudaError_t rcp_check(long long n, unsigned long long* max_ulp);

// batched execution (hgks_kernels.cu)
void batch_fill_desc(const hgks_solver* s, SolveDesc& d);
void batch_plan(const std::vector<const SolveDesc*>& descs, int dim, const int* tpb, BatchPlan& plan);
// enqueue one batched step; ev (optional, 2 * BK_COUNT events) records each class for timing
cudaError_t batch_enqueue_step(const BatchPlan& plan, const SolveDesc* d_desc, const int* d_boff,
                               const double* d_tend, cudaStream_t st, cudaEvent_t* ev);
extern const int kBatchTpbDefault[BK_COUNT];

}  // namespace hgks
