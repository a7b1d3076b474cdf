#!/usr/bin/env python3
"""Throughput benchmark of the hybrid WENO-AO gas-kinetic S2O4 step on GB300.

Workload: the four-quadrant 2D Riemann problem on [0,1]^2 at 1024^2 cells with
seeded quadrant states (rho, p ~ U[0.1, 2], u, v ~ U[-1, 1], numpy PCG64 seed
20230411), hybrid WENO-AO reconstruction, c1 = 0.01, c2 = 1, CFL 0.5,
non-reflecting boundaries, FP64.  One "step" is one S2O4 step (two stages) over
the whole grid; the unit is interior cells x stages.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N > 1 (launched under torchrun) every rank advances its own
independent replica (the solves do not exchange data) and the value is the
aggregate over ranks divided by the maximum time over ranks.

The default line also carries
  "served":  the served configuration's size ranges (1D shock tubes up to 8192 cells, 2D
             Riemann / vortex up to 1024^2, 2D Navier-Stokes shock tubes up to 2048 x 1024,
             150 GB budget; 20 seeded requests) through the continuous-batching server against
             the same requests one at a time: capacities on the seeded burst, p50 / p99
             latency on the same arrivals stretched to 70 % of the plain capacity measured in
             the same run, bitwise equality of every result (--no-served skips it);
  "batched": the 256-solve batched configuration against one solve per launch set, with 5
             timed steps per solve (--batched-steps; --no-batched skips it).
Other workloads (--workload batched | served | recon_cost | ns_tube | vortex) print
their own line.

The roofline is FP64-ALU bound: the numerator counts the algorithmic FP64 work (fixed
counts, see FLUX_ALG_FLOP_PER_GP); the peak is the device's SM count x 4 FP64 flop per
clock x the SM clock sampled during the timed region, with the DFMA-chain probe
(hgks_probe_fp64) reported beside it.

--impl reference times the CPU oracle (the plain FP64 restatement of the
paper's method) on the host cores, on the same 1024^2 problem.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Mcell-stage updates/s, 2D GKS FP64, served vs plain launch; p50/p99 solve latency"
UNIT = "Mcell-stage/s"
N_SIDE = 1024
WORKLOAD = "four-quadrant 2D Riemann problem, 1024^2 cells, hybrid WENO-AO HGKS, S2O4"

# Algorithmic FP64 work of the step (add / sub, mul, div, sqrt, exp and erfc count one each, fma
# two), kept fixed here so that the yardstick does not move when a kernel changes:
# * the flux per Gauss point: the closed form of the flux kernel (2D Euler, tau > 0), counted on
#   the host by paper_2304_05572_gb300/flopcount.py: 1433 operations in the first stage (F(dt/2)
#   and the F^n + dt/6 dF^n combination), 1389 in the second; on sweeps of 65 536 segments or
#   more the kernel also reconstructs its Gauss point's smooth tangential passes
#   (FLUX_KERNEL_TANG_FLOP_PER_GP); one launch covers both sweeps of a stage;
# * the rest of the step per cell-stage (indicator, reconstruction, update, time step), counted on
#   the oracle by oracle/opcount.py on the first step of the 1024^2 problem (the oracle evaluates
#   these formulas as the paper prints them): every cell smooth 2721.3, every cell troubled
#   19486.7, the hybrid step 3525.5 at its troubled fraction 0.41 %; a run at another troubled
#   fraction f moves the hybrid figure along the troubled-minus-smooth slope.  (The oracle's own
#   flux integrates every moment literally, ORACLE_FLUX_FLOP_PER_GP operations, five times the
#   closed form: a roofline on that count would exceed the peak, so the flux enters with its
#   closed-form count.)
FLUX_ALG_FLOP_PER_GP = (1433.0 + 1389.0) / 2
ORACLE_FLUX_FLOP_PER_GP = 7025.0
# On large sweeps the flux kernel also reconstructs its Gauss point's smooth tangential passes
# (the quartic of Sec. 2.3.3 at the Gauss point): 16 values and 8 tangential derivatives of 5
# terms each (1 mul + 4 fma = 9 operations), 2 positivity tests (6) and 8 derivative scalings:
# 236 operations per Gauss point, counted by hand from the formulas.
FLUX_KERNEL_TANG_FLOP_PER_GP = 16 * 9 + 8 * 9 + 2 * 6 + 8
NONFLUX_FLOP_PER_CELL_STAGE = {"linear": 2721.3, "wenoao": 19486.7, "hybrid": 3525.5,
                               "hybrid_troubled_fraction": 0.004106}
# DRAM bytes (read + write) per flux launch (both sweeps), one ncu pass over a whole 1024^2 step
# with the caches carried from kernel to kernel (--cache-control none), as the step runs: first
# stage 275.5 MB read + 118.6 MB written, second stage 275.6 + 61.5 MB; per Gauss point of the
# launch (4 * 1024 * 1025 of them).
FLUX_DRAM_BYTES_PER_GP = (275.49e6 + 118.56e6 + 275.58e6 + 61.50e6) / 2 / (4 * 1024 * 1025)


def algorithmic_flop_per_cell_stage(n, troubled_fraction):
    """Algorithmic FP64 work per cell-stage of the n^2 hybrid step at the given troubled
    fraction: the oracle's count of everything but the flux, plus the closed-form flux of the
    2 sweeps x 2 Gauss points of every interface."""
    t = NONFLUX_FLOP_PER_CELL_STAGE
    rest = t["hybrid"] + (troubled_fraction - t["hybrid_troubled_fraction"]) * (t["wenoao"] - t["linear"])
    return rest + 4.0 * (n + 1) / n * FLUX_ALG_FLOP_PER_GP


def max_over_ranks(x, dist=None, device="cpu"):
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, cells, steps, seconds):
    """Whole-job Mcell-stage/s of `world` independent replicas, each advancing `cells` cells
    by `steps` two-stage steps, timed by the slowest rank (`seconds`)."""
    return world * cells * 2 * steps / seconds / 1e6


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1])); smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=len(sm))
        return out


def cpu_oracle_rate(n_side, steps, threads=0, problem=None):
    """Time the oracle (as it stands) on `steps` S2O4 steps of the n_side^2 workload (the
    initial state is built outside the timed region)."""
    import oracle
    from paper_2304_05572_gb300 import problems as P
    oracle.build()
    cfg, W, _ = problem if problem is not None else P.riemann4_2d(n_side)
    t0 = time.perf_counter()
    _, _, n, _ = oracle.run(cfg, W, 1e9, max_steps=steps, threads=threads)
    dt = time.perf_counter() - t0
    return n_side * n_side * 2 * n / dt / 1e6, dt, oracle.threads_used(threads)


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on the host cores (rank 0 only), on the benchmark's own
    1024^2 problem: every (warm-up or timed) step is one S2O4 step of the oracle from the
    initial state."""
    if rank != 0:
        return 0
    from paper_2304_05572_gb300 import problems as P
    n_side = args.ref_side
    problem = P.riemann4_2d(n_side)
    cores = None
    for _ in range(args.warmup):
        cpu_oracle_rate(n_side, 1, problem=problem)
    secs = 0.0
    for _ in range(args.steps):
        _, dt, cores = cpu_oracle_rate(n_side, 1, problem=problem)
        secs += dt
    value = n_side * n_side * 2 * args.steps / secs / 1e6
    sample = "%d S2O4 steps (each from the initial state) of the %d^2 problem, OpenMP on all host cores" % (
        args.steps, n_side)
    workload = WORKLOAD if n_side == N_SIDE else WORKLOAD.replace("1024^2", "%d^2" % n_side)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "grid": [n_side, n_side], "stages_per_step": 2},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batched(torch, hgks, P, n_solves, steps, warmup):
    """Independent four-quadrant Riemann solves (sides log-uniform in [64, 1024]): one
    launch set per solve (serial on one stream) against shared batched launches (CUDA
    graph replay, autotuned block sizes).  Both forms advance every solve by the same
    steps from the same state and must give the same bits.  A solve whose state turns
    non-physical (the scheme has no positivity limiter) stops in both forms at the same
    step; the work counted is the cell-stages actually advanced.  Returns the figures."""
    cases = P.batched_workload(n_solves)
    stream = torch.cuda.Stream()
    solvers = [hgks.Solver(cfg, stream=stream) for cfg, _ in cases]
    ncell = [int(np.prod(W.shape[1:])) for _, W in cases]
    warm = max(warmup, 4)          # the autotuner takes 4 steps

    def reset():
        for s, (cfg, W) in zip(solvers, cases):
            s.hgks_set_state(np.ascontiguousarray(W))

    def steps_now():
        return [int(s.hgks_get_stats()["steps"]) for s in solvers]

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b) * 1e-3

    # one solve per launch set
    reset()
    for s in solvers:
        s.hgks_step(1e9, warm, wait=False)
    s0 = steps_now()
    t_plain = timed(lambda: [s.hgks_step(1e9, steps, wait=False) for s in solvers])
    s1 = steps_now()
    plain_final = [s.hgks_get_state() for s in solvers]
    work_plain = sum(c * 2 * (b - a) for c, a, b in zip(ncell, s0, s1))
    # batched
    reset()
    batch = hgks.Batch(solvers, stream=stream)
    te = [1e9] * len(solvers)
    batch.hgks_batch_step(te, nsteps=warm, graph=True, autotune=True)
    batch.hgks_batch_sync()
    b0 = steps_now()
    t_batch = timed(lambda: batch.hgks_batch_step(te, nsteps=steps, graph=True))
    _, failed = batch.hgks_batch_sync()
    b1 = steps_now()
    work_batch = sum(c * 2 * (b - a) for c, a, b in zip(ncell, b0, b1))
    tpb, _ = batch.hgks_batch_info()
    same = b1 == s1 and all(np.array_equal(s.hgks_get_state(), ref, equal_nan=True)
                            for s, ref in zip(solvers, plain_final))
    batch.hgks_batch_destroy()
    for s in solvers:
        s.hgks_destroy_solver()
    return {"workload": "batched: %d four-quadrant Riemann solves, sides log-uniform 64..1024 "
            "(PCG64 seed %d), %d cells in all, %d timed S2O4 steps each after %d untimed"
            % (len(cases), P.BATCH_SEED, sum(ncell), steps, warm),
            "unit": UNIT, "value": work_batch / t_batch / 1e6, "plain_value": work_plain / t_plain / 1e6,
            "speedup_vs_plain": (work_batch / t_batch) / (work_plain / t_plain),
            "batched_ms_per_step": t_batch / steps * 1e3, "plain_ms_per_step": t_plain / steps * 1e3,
            "cell_stages_timed": work_batch, "failed_solves": failed, "bitwise_equal_to_plain": bool(same),
            "autotuned_block_sizes": tpb, "l2": "working set (%.1f GB of state) far above L2" % (
                sum(ncell) * 4 * 8 * 3 / 1e9)}


def bench_batched(args, torch, hgks, P):
    """The batched workload as its own JSON line."""
    d = run_batched(torch, hgks, P, args.solves, args.steps, args.warmup)
    line = {"metric": METRIC, **d, "dtype": "f64", "data": "synthetic", "higher_is_better": True}
    print(json.dumps(line), flush=True)


def _fifo_latencies(trace, dur):
    """Latency of each request when the requests are served one at a time in arrival order
    (FIFO), each taking its measured solo duration."""
    clock, lat = 0.0, {}
    for r in sorted(trace, key=lambda r: r["arrival"]):
        clock = max(clock, r["arrival"]) + dur[r["id"]]
        lat[r["id"]] = clock - r["arrival"]
    return lat


def run_served(torch, P, requests, rate, max_1d, max_2d, max_ns, budget_gb, steps_per_iter, load=0.7):
    """A seeded Poisson stream of mixed solves (1D shock tubes, 2D Riemann / vortex, 2D
    Navier-Stokes shock tubes) through the continuous-batching server against the same
    requests served one at a time (FIFO, each solve alone on the GPU).

    1. Plain arm: every request alone, in order; its solo duration and result are kept.
    2. Burst: the seeded arrivals at `rate` (every request queued within a second) through the
       server: the served and plain throughputs (work / wall) are the two capacities.
    3. Load-scaled: the same arrivals stretched so that the offered load is `load` times the
       plain capacity measured in step 1 (rate = load x requests / total solo time); the
       served latencies against the FIFO latencies of the plain arm on the same arrivals.
    Every served result must equal the request solved alone, bit for bit."""
    from paper_2304_05572_gb300 import server
    trace = P.served_trace(n_requests=requests, rate=rate, max_1d=max_1d, max_2d=max_2d, max_ns=max_ns)
    stream = torch.cuda.Stream()
    dur, alone, work = {}, {}, {}
    for r in trace:
        w0 = time.perf_counter()
        out, st = server.run_alone(r, stream=stream)
        dur[r["id"]] = time.perf_counter() - w0
        alone[r["id"]] = out
        work[r["id"]] = int(np.prod(np.shape(r["W"])[1:])) * 2 * int(st["steps"])
    total_work, total_dur = float(sum(work.values())), float(sum(dur.values()))

    def serve(tr):
        srv = server.Server(budget_bytes=budget_gb * 1e9, stream=stream, steps_per_iter=steps_per_iter,
                            autotune=False)
        res = srv.run(tr)
        lat = np.array([res[r["id"]]["latency"] for r in tr])
        same = all(np.array_equal(res[r["id"]]["W"], alone[r["id"]]) for r in tr)
        return srv, lat, same

    srv_b, lat_b, same_b = serve(trace)
    plain_b = np.array([v for v in _fifo_latencies(trace, dur).values()])
    lam = load * len(trace) / total_dur
    scaled = [dict(r, arrival=r["arrival"] * rate / lam) for r in trace]
    srv_l, lat_l, same_l = serve(scaled)
    plain_l = np.array([v for v in _fifo_latencies(scaled, dur).values()])
    pct = lambda a, q: float(np.percentile(a, q))
    return {"workload": "served: %d requests (PCG64 seed %d), mix of 1D shock tubes 256..%d cells, 2D Riemann/vortex "
            "64..%d^2, 2D NS shock tubes 128x64..%dx%d (Re ~ U[200, 2000]), t_end ~ U[0.05, 0.3], budget %.0f GB"
            % (len(trace), P.SERVE_SEED, max_1d, max_2d, max_ns, max_ns // 2, budget_gb),
            "unit": UNIT, "cell_stages": total_work,
            # burst: capacities
            "value": total_work / srv_b.wall / 1e6, "plain_value": total_work / total_dur / 1e6,
            "burst": {"rate_per_s": rate, "served_wall_s": srv_b.wall, "plain_wall_s": total_dur,
                      "p50_latency_s": pct(lat_b, 50), "p99_latency_s": pct(lat_b, 99),
                      "plain_p50_latency_s": pct(plain_b, 50), "plain_p99_latency_s": pct(plain_b, 99),
                      "iterations": srv_b.iterations, "peak_resident_solves": srv_b.peak_resident},
            # load-scaled: latency at the same offered load
            "load_scaled": {"offered_load_of_plain_capacity": load, "rate_per_s": lam,
                            "served_wall_s": srv_l.wall,
                            "p50_latency_s": pct(lat_l, 50), "p99_latency_s": pct(lat_l, 99),
                            "plain_p50_latency_s": pct(plain_l, 50), "plain_p99_latency_s": pct(plain_l, 99),
                            "iterations": srv_l.iterations, "peak_resident_solves": srv_l.peak_resident},
            "p50_latency_s": pct(lat_l, 50), "p99_latency_s": pct(lat_l, 99),
            "plain_p50_latency_s": pct(plain_l, 50), "plain_p99_latency_s": pct(plain_l, 99),
            "results_bitwise_equal_alone": bool(same_b and same_l)}


def bench_served(args, torch, hgks, P):
    """The served workload at the sizes given on the command line, as its own JSON line."""
    d = run_served(torch, P, args.requests, args.rate, args.max_1d, args.max_2d, args.max_ns, args.budget_gb,
                   args.steps_per_iter)
    line = {"metric": METRIC, **d, "dtype": "f64", "data": "synthetic", "higher_is_better": True}
    print(json.dumps(line), flush=True)


def bench_single(args, torch, hgks, P):
    """One solve of another configuration, K timed S2O4 steps on the device:
    ns_tube: 2D Navier-Stokes viscous shock tube in [0,1] x [0,0.5] (Sec. 3.6 set-up) at
             Re = 1000, Pr = 0.73 (energy-flux Prandtl fix), nx x nx/2 cells;
    vortex:  isentropic vortex on the periodic [0,10]^2 (strength 5, tau = 0), nx^2 cells."""
    nx = args.ns_nx if args.workload == "ns_tube" else args.vortex_n
    if args.workload == "ns_tube":
        cfg, W, _ = P.viscous_shock_tube(nx, nx // 2, Re=1000.0, prandtl=0.73)
        label = "2D NS viscous shock tube, %dx%d, Re 1000, Pr 0.73, hybrid, S2O4" % (nx, nx // 2)
    else:
        cfg, W, _ = P.vortex_2d(nx)
        label = "2D isentropic vortex, %d^2, periodic, tau = 0, hybrid, S2O4" % nx
    stream = torch.cuda.Stream()
    s = hgks.Solver(cfg, stream=stream)
    s.hgks_set_state(np.ascontiguousarray(W))
    s.hgks_step(1e9, args.warmup, wait=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    s.hgks_step(1e9, args.steps, wait=False)
    b.record(stream)
    stream.synchronize()
    ms = a.elapsed_time(b)
    st = s.hgks_get_stats()
    # kernel-class shares from further steps with per-class events (outside the timed ones)
    s.hgks_set_timing(True)
    s.hgks_step(1e9, args.steps, wait=True)
    tim = s.hgks_get_timing()
    s.hgks_destroy_solver()
    cells = int(np.prod(W.shape[1:]))
    tot = sum(v[0] for v in tim.values())
    line = {"metric": METRIC, "workload": label,
            "unit": UNIT, "value": cells * 2 * args.steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / args.steps,
            "steps": args.steps, "status": int(st["status"]), "t": st["t"],
            "troubled_fraction": float(st["troubled"].sum()) / max(1, int(st["examined"].sum())),
            "kernel_time_share": {k: round(v[0] / max(1e-9, tot), 4) for k, v in tim.items() if v[1]},
            "dtype": "f64", "data": "synthetic", "higher_is_better": True}
    print(json.dumps(line), flush=True)


def bench_ns_wall(args, torch, hgks, P):
    """The viscous shock tube of Sec. 3.6 as the paper runs it (Re = 200, Pr = 1, 500 x 250 cells,
    CFL 0.3, t = 1): the density along the bottom wall (the cell row next to it) at t = 1, with
    the run's time, steps and wall time."""
    nx = args.ns_nx
    cfg, W, t_end = P.viscous_shock_tube(nx, nx // 2, Re=200.0, prandtl=1.0)
    stream = torch.cuda.Stream()
    s = hgks.Solver(cfg, stream=stream)
    s.hgks_set_state(np.ascontiguousarray(W))
    t0 = time.perf_counter()
    n = s.hgks_step(t_end, 1 << 30)
    wall = time.perf_counter() - t0
    Wf = s.hgks_get_state()
    st = s.hgks_get_stats()
    s.hgks_destroy_solver()
    dx = 1.0 / nx
    line = {"metric": "bottom-wall density of the viscous shock tube (Sec. 3.6)",
            "workload": "2D NS viscous shock tube, %dx%d, Re 200, Pr 1, CFL 0.3, hybrid, S2O4, to t = %g"
                        % (nx, nx // 2, t_end),
            "t": st["t"], "steps": n, "status": int(st["status"]), "wall_s": wall,
            "troubled_fraction": float(st["troubled"].sum()) / max(1, int(st["examined"].sum())),
            "x_first_centre": 0.5 * dx, "dx": dx, "rho_wall": [float(v) for v in Wf[0, 0, :]],
            "dtype": "f64", "data": "synthetic"}
    print(json.dumps(line), flush=True)


RECON_CLASSES = ("raw_normal_flags", "normal_recon", "normal_weno_ao", "raw_tangential_flags", "tangential_recon",
                 "tangential_weno_ao")

# Reconstruction CPU times of the paper (i5-9400, seconds; hybrid, WENO-AO), Tables 3 and 6.
PAPER_RECON_S = {"sod_100": (0.016, 0.049), "shu_osher_400": (0.245, 1.937), "blast_400": (0.773, 3.176),
                 "riemann_config1_500": (706.471, 6100.513), "riemann_config6_500": (5546.881, 9628.309),
                 "double_mach_960x240": (5334.322, 13596.93), "viscous_tube_500x250_Re200": (12148.766, 46394.377)}


def bench_recon_cost(args, torch, hgks, P):
    """Reconstruction cost of the hybrid scheme against WENO-AO everywhere on the paper's
    test problems (Tables 3 and 6): each problem runs to its end time in both modes with
    per-kernel-class CUDA events; the reconstruction time is the sum of the indicator and
    reconstruction classes (normal and tangential), the rest is flux, update, dt, ghosts."""
    cases = [("sod_100", P.sod_1d(100)), ("shu_osher_400", P.shu_osher_1d(400)), ("blast_400", P.blast_1d(400)),
             ("riemann_config1_500", P.riemann_config1(500)), ("riemann_config6_500", P.riemann_config6(500)),
             ("double_mach_960x240", P.double_mach(960, 240)),
             ("viscous_tube_500x250_Re200", P.viscous_shock_tube(500, 250, Re=200.0))]
    if args.recon_cases:
        keep = set(args.recon_cases.split(","))
        cases = [c for c in cases if c[0] in keep]
    stream = torch.cuda.Stream()
    rows = []
    for name, (cfg, W, t_end) in cases:
        res = {}
        for mode in ("hybrid", "wenoao"):
            s = hgks.Solver(dict(cfg, recon_mode=mode), stream=stream)
            s.hgks_set_state(np.ascontiguousarray(W))
            s.hgks_step(t_end, 2, wait=True)           # loads the kernels; not timed
            s.hgks_set_state(np.ascontiguousarray(W))
            s.hgks_set_timing(True)
            steps, status = 0, 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            while True:
                try:
                    n = s.hgks_step(t_end, 200)
                except hgks.HGKSError as e:
                    status = e.code
                    break
                steps += n
                s.hgks_get_timing()                     # recycles the event pairs
                if n < 200:
                    break
            wall = time.perf_counter() - t0
            tim = s.hgks_get_timing()
            st = s.hgks_get_stats()
            s.hgks_destroy_solver()
            recon = sum(tim[c][0] for c in RECON_CLASSES if c in tim)
            total = sum(v[0] for v in tim.values())
            troubled = float(st["troubled"].sum()) / max(1, int(st["examined"].sum()))
            res[mode] = dict(recon_ms=recon, kernel_ms=total, wall_s=wall, steps=int(st["steps"]),
                             t=st["t"], status=int(st["status"]), troubled_fraction=troubled,
                             class_ms={k: round(v[0], 3) for k, v in tim.items() if v[1]})
        paper = PAPER_RECON_S.get(name)
        rows.append(dict(case=name, cells=int(np.prod(W.shape[1:])), hybrid=res["hybrid"], wenoao=res["wenoao"],
                         recon_ratio=res["hybrid"]["recon_ms"] / max(1e-9, res["wenoao"]["recon_ms"]),
                         total_ratio=res["hybrid"]["kernel_ms"] / max(1e-9, res["wenoao"]["kernel_ms"]),
                         paper_recon_ratio=paper[0] / paper[1] if paper else None))
    line = {"metric": "reconstruction time, hybrid WENO-AO / WENO-AO everywhere (GPU kernel time, FP64)",
            "workload": "the paper's test problems to their end times (Tables 3 and 6)", "cases": rows,
            "dtype": "f64", "data": "synthetic", "higher_is_better": False}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-served", action="store_true", help="skip the served-vs-plain part of the default line")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched part of the default line")
    ap.add_argument("--served-requests", type=int, default=20, help="requests of the default line's served part")
    ap.add_argument("--batched-steps", type=int, default=5, help="timed steps of the default line's batched part")
    ap.add_argument("--n", type=int, default=N_SIDE)
    ap.add_argument("--ref-side", type=int, default=N_SIDE, help="grid side of the reference arm's problem")
    ap.add_argument("--workload", default="riemann1024", choices=["riemann1024", "batched", "served", "recon_cost", "ns_tube", "vortex", "ns_wall"])
    ap.add_argument("--ns-nx", type=int, default=1000, help="ns_tube / ns_wall: cells along x (ny = nx/2)")
    ap.add_argument("--vortex-n", type=int, default=800, help="vortex: cells per side")
    ap.add_argument("--recon-cases", default="", help="comma-separated subset of the recon_cost cases")
    ap.add_argument("--solves", type=int, default=256)
    ap.add_argument("--requests", type=int, default=20)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--max-1d", type=int, default=8192)
    ap.add_argument("--max-2d", type=int, default=1024)
    ap.add_argument("--max-ns", type=int, default=2048)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--steps-per-iter", type=int, default=8)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local_rank = _env_int("LOCAL_RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod

    if args.impl == "reference":
        if dist is not None:
            dist.init_process_group("gloo")
        rc = run_reference(args, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return rc

    import torch
    from paper_2304_05572_gb300 import hgks, problems as P

    torch.cuda.set_device(local_rank)
    if args.workload == "batched":
        return bench_batched(args, torch, hgks, P)
    if args.workload == "served":
        return bench_served(args, torch, hgks, P)
    if args.workload == "recon_cost":
        return bench_recon_cost(args, torch, hgks, P)
    if args.workload in ("ns_tube", "vortex"):
        return bench_single(args, torch, hgks, P)
    if args.workload == "ns_wall":
        return bench_ns_wall(args, torch, hgks, P)
    if dist is not None:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)

    n = args.n
    cfg, W0, _ = P.riemann4_2d(n)
    cells = n * n
    solver = hgks.Solver(cfg, stream=stream)
    W0 = np.ascontiguousarray(W0)
    Wd = torch.from_numpy(W0).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # ---- device-resident timing: W steps untimed, then K timed steps (L2 flushed before each)
    solver.hgks_set_state(Wd)
    for _ in range(args.warmup):
        solver.hgks_step(1e9, 1, wait=False)
    torch.cuda.synchronize()
    solver.hgks_set_timing(True)
    solver.hgks_get_timing()              # drop warm-up records (timing starts now)
    launches0 = int(solver.hgks_get_stats()["launches"])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0) as clk:
        t_wall0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.zero_()
                ev[k][0].record(stream)
                solver.hgks_step(1e9, 1, wait=False)
                ev[k][1].record(stream)
        stream.synchronize()
        t_wall = time.perf_counter() - t_wall0
    barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    timing = solver.hgks_get_timing()
    solver.hgks_set_timing(False)
    stats = solver.hgks_get_stats()
    if stats["status"] != 0:
        raise SystemExit("solver reported status %d" % stats["status"])
    ms = max_over_ranks(ms, dist, dev)
    steps_timed = args.steps
    value = replica_throughput(world, cells, steps_timed, ms * 1e-3)
    troubled = stats["troubled"].sum() / max(1, stats["examined"].sum())

    # ---- end-to-end through the C ABI: pinned host state in, one step, pinned host state out
    Wh = torch.from_numpy(W0).pin_memory()
    Wout = torch.empty_like(Wh).pin_memory()
    e2e_steps = max(3, args.steps // 2)
    barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(e2e_steps):
            flush.zero_()                        # L2 flushed as in the device-resident loop (~0.1 ms)
            solver.hgks_set_state(Wh)            # H2D from pinned host memory (waits for the copy)
            solver.hgks_step(1e9, 1, wait=False)
            solver.hgks_get_state(Wout)          # D2H of the result (waits for the stream)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e_value = replica_throughput(world, cells, e2e_steps, e2e_s)
    state_bytes = int(W0.nbytes)

    # ---- FP64 peak of this GPU: the SM count of the device x 4 FP64 flop per clock and SM (two
    # FP64 instruction issues, the unit count behind the nominal 1.25 TFLOP/s) x the median SM clock
    # of the timed region.  The DFMA-chain probe (its clock sampled while it runs) is reported
    # beside it: chains of one FP64 operation reach 84 % of that issue rate, while the flux kernel's
    # instruction mix reaches 90 % (ncu), so the probe is not a ceiling and the unit count is.
    clocks = clk.summary()
    with ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0) as clkp:
        probe_tflops, probe_ms, n_sm = hgks.hgks_probe_fp64(stream)
    probe_mhz = clkp.summary()["sm_mhz"] or clocks["sm_mhz"]
    run_mhz = clocks["sm_mhz"] or probe_mhz or 2070.0
    peak_tflops = n_sm * 4 * run_mhz / 1e6

    # ---- dominant kernel roofline (FP64 ALU) on the algorithmic count
    flux_ms, flux_calls = timing.get("gks_flux", (0.0, 0))
    launches = int(stats.get("launches", 0)) - launches0     # kernels of the timed steps only
    roofline = None
    if flux_calls:
        avg_ms = flux_ms / flux_calls
        gp_per_launch = 2 * 2 * (n + 1) * n      # Gauss points of both sweeps (one launch per stage)
        # the kernel's work per Gauss point: the flux, and on sweeps of 65 536 segments or more the
        # fused reconstruction of the smooth tangential passes
        per_gp = FLUX_ALG_FLOP_PER_GP + (FLUX_KERNEL_TANG_FLOP_PER_GP if n * (n + 1) >= 65536 else 0.0)
        achieved = per_gp * gp_per_launch / (avg_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                    "frac": achieved / peak_tflops,
                    "traffic": FLUX_DRAM_BYTES_PER_GP * gp_per_launch if n == N_SIDE else None,
                    "kernel": "gks_flux", "avg_launch_ms": avg_ms,
                    "flop_per_launch": per_gp * gp_per_launch,
                    "unit_of_work": "Gauss point: %.0f algorithmic FP64 operations = flux %.0f (closed form; the "
                                    "oracle's literal moment integration takes %.0f) + reconstruction of the smooth "
                                    "tangential passes %.0f" % (per_gp, FLUX_ALG_FLOP_PER_GP, ORACLE_FLUX_FLOP_PER_GP,
                                                                 per_gp - FLUX_ALG_FLOP_PER_GP),
                    "peak_note": "derived: %d SMs (device attribute) x 4 FP64 flop/clk/SM x %s MHz (median SM "
                                 "clock of the timed region); the DFMA-chain probe hgks_probe_fp64 gives %.3f "
                                 "TFLOP/s at %s MHz (%.2f flop/clk/SM)"
                                 % (n_sm, run_mhz, probe_tflops, probe_mhz,
                                    probe_tflops * 1e6 / (n_sm * probe_mhz) if probe_mhz else float("nan"))}
    shares = {k: round(v[0] / max(1e-9, sum(x[0] for x in timing.values())), 4) for k, v in timing.items() if v[1]}
    if roofline is not None and NONFLUX_FLOP_PER_CELL_STAGE["hybrid"] is not None:
        fpcs = algorithmic_flop_per_cell_stage(n, float(troubled))
        step_tflops = fpcs * value / world * 1e6 / 1e12
        roofline["whole_step"] = {"flop_per_cell_stage": fpcs, "achieved": step_tflops,
                                  "frac": step_tflops / peak_tflops, "unit": "TFLOP/s",
                                  "troubled_fraction": float(troubled)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps_timed,
        "warmup": args.warmup, "ms_per_step": ms / steps_timed, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if n == N_SIDE else WORKLOAD.replace("1024^2", "%d^2" % n),
                   "grid": [n, n], "stages_per_step": 2, "replicas": world,
                   "l2": "flushed before every timed step (256 MiB write, outside the events)",
                   "troubled_fraction": round(float(troubled), 5)},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                "note": "hgks_set_state(pinned host) + hgks_step(1) + hgks_get_state(pinned host) per step; "
                        "L2 flushed before every step (256 MiB write, inside the wall-clock timed region)"},
        "gpu_launches": launches,
        "roofline": roofline,
        "kernel_time_share": shares,
        # the same throughput with the dt reduction and the ghost fills taken out (the value above
        # is the whole step, those included)
        "value_without_dt_and_ghost": value / max(1e-9, 1.0 - shares.get("dt", 0.0) - shares.get("ghost", 0.0)
                                                  - shares.get("misc", 0.0)),
        "clocks": clocks,
        "wall_s_timed": t_wall,
    }
    if rank == 0 and world == 1 and not args.no_served:
        # the metric's served-vs-plain part on the served configuration's size ranges: capacity
        # (burst) and p50 / p99 latency at 70 % of the plain capacity, results bitwise equal
        try:
            line["served"] = run_served(torch, P, args.served_requests, 200.0, 8192, 1024, 2048, 150.0,
                                        args.steps_per_iter)
        except Exception as e:  # pragma: no cover
            line["served"] = {"failed": str(e)}
    if rank == 0 and world == 1 and not args.no_batched:
        # the batched configuration (256 solves) with a reduced number of timed steps
        try:
            line["batched"] = run_batched(torch, hgks, P, 256, args.batched_steps, 4)
        except Exception as e:  # pragma: no cover
            line["batched"] = {"failed": str(e)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            v, secs, cores = cpu_oracle_rate(N_SIDE, 1)
            v1, secs1, _ = cpu_oracle_rate(256, 1, threads=1)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": "1 S2O4 step of the same 1024^2 problem (%.1f s)" % secs,
                                    "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                                      "sample": "1 S2O4 step of the problem at 256^2 (%.1f s)" % secs1}}
        except Exception as e:  # pragma: no cover
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": "failed: %s" % e}
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.hgks_destroy_solver()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
