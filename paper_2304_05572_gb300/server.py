"""Continuous-batching solve server on one GPU.

Requests (a configuration, an initial state and an end time) arrive over time.
The server admits a request as soon as its arrival time has passed and the
device memory its solver needs (hgks_footprint_bytes) fits in the budget;
admitted solves keep their state resident on the device and advance together:
every iteration issues one batched group of S2O4 steps (hgks_batch_step, CUDA
graph replay) per dimension for all resident solves, the 1D and 2D groups on
their own streams so that they overlap on the device, so newly admitted solves
overlap on the device with the ones already running.  A solve retires at its
end time (or when its state turned non-physical: the scheme has no positivity
limiter, and the status is reported with the result); its state is copied
back, its memory freed and its latency (completion minus arrival, queueing
included) recorded.

Each solve's arithmetic is independent of the others (batched launches never
mix solvers inside a block), so a result is bit-identical alone and in the mix.
All numerical work runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import time

import numpy as np

from . import hgks


class Server:
    def __init__(self, budget_bytes: float, stream=None, steps_per_iter: int = 4, autotune: bool = False):
        import torch
        self.budget = float(budget_bytes)
        # one stream per dimension: the 1D batch (small, latency-bound launches) overlaps on the
        # device with the 2D batch; `stream`, if given, serves the 2D solves
        self.streams = {1: torch.cuda.Stream(), 2: stream if stream is not None else torch.cuda.Stream()}
        self.steps_per_iter = int(steps_per_iter)
        self.autotune = autotune
        self.used = 0.0
        self.active = {}          # id -> dict(req, solver, bytes, t_admit)
        self.results = {}         # id -> dict(W, latency, admitted, completed, steps, t, status, cells)
        self._batches = {}        # dim -> (tuple of ids, Batch)
        self.iterations = 0
        self.peak_resident = 0

    def _admit(self, req, now):
        dim = int(req["cfg"]["dim"])
        s = hgks.Solver(req["cfg"], stream=self.streams[dim])
        s.hgks_set_state(np.ascontiguousarray(req["W"]))
        self.active[req["id"]] = dict(req=req, solver=s, bytes=req["bytes"], t_admit=now)
        self.used += req["bytes"]
        self.peak_resident = max(self.peak_resident, len(self.active))

    def _retire(self, rid, now, t, status, steps):
        a = self.active.pop(rid)
        s = a["solver"]
        self.results[rid] = dict(W=s.hgks_get_state(), latency=now - a["req"]["arrival"], admitted=a["t_admit"],
                                 completed=now, steps=int(steps), t=t, status=int(status),
                                 cells=int(np.prod(a["req"]["W"].shape[1:])))
        s.hgks_destroy_solver()
        self.used -= a["bytes"]

    def _batch_for(self, dim, ids):
        key = tuple(sorted(ids))
        cur = self._batches.get(dim)
        if cur is not None and cur[0] == key:
            return cur[1]
        if cur is not None:
            cur[1].hgks_batch_destroy()
        b = hgks.Batch([self.active[i]["solver"] for i in key], stream=self.streams[dim])
        self._batches[dim] = (key, b)
        return b

    def run(self, trace, time_scale: float = 1.0):
        """Serve a list of requests (dicts with id, arrival [s], cfg, W, t_end) in arrival
        order; arrival times are scaled by time_scale.  Returns the results dict."""
        pending = sorted(({**r, "arrival": r["arrival"] * time_scale,
                           "bytes": float(hgks.hgks_footprint_bytes(r["cfg"]))} for r in trace),
                         key=lambda r: r["arrival"])
        for r in pending:
            if r["bytes"] > self.budget:
                raise ValueError("request %d alone exceeds the memory budget" % r["id"])
        t0 = time.perf_counter()
        qi = 0
        while qi < len(pending) or self.active:
            now = time.perf_counter() - t0
            while qi < len(pending) and pending[qi]["arrival"] <= now and self.used + pending[qi]["bytes"] <= self.budget:
                self._admit(pending[qi], now)
                qi += 1
            if not self.active:
                if qi < len(pending):
                    time.sleep(max(0.0, min(0.01, pending[qi]["arrival"] - now)))
                continue
            by_dim = {}
            for rid, a in self.active.items():
                by_dim.setdefault(int(a["req"]["cfg"]["dim"]), []).append(rid)
            stepped = []
            for dim, ids in by_dim.items():             # enqueue every dimension first (they overlap)
                b = self._batch_for(dim, ids)
                key = self._batches[dim][0]
                b.hgks_batch_step([self.active[i]["req"]["t_end"] for i in key], nsteps=self.steps_per_iter,
                                  graph=True, autotune=self.autotune)
                stepped.append(dim)
            self.iterations += 1
            finished = []
            for dim in stepped:
                key, b = self._batches[dim]
                b.hgks_batch_sync()
                ts, sts, nsteps = b.hgks_batch_status()
                for rid, t, st, n in zip(key, ts, sts, nsteps):
                    te = self.active[rid]["req"]["t_end"]
                    # a solve retires at its end time, or with its error once its state turned non-physical
                    if st != 0 or te - t <= 1e-12 * max(1.0, abs(te)):
                        finished.append((rid, t, st, n))
            now = time.perf_counter() - t0
            for rid, t, st, n in finished:
                self._retire(rid, now, t, st, n)
        for dim, (key, b) in list(self._batches.items()):
            b.hgks_batch_destroy()
        self._batches.clear()
        self.wall = time.perf_counter() - t0
        return self.results


def run_alone(req, stream=None):
    """The same request solved on its own (reference for the served results).  A solve
    whose state turns non-physical stops there, as in the server; its stats carry the status."""
    s = hgks.Solver(req["cfg"], stream=stream)
    s.hgks_set_state(np.ascontiguousarray(req["W"]))
    try:
        s.hgks_step(req["t_end"], 1 << 30)
    except hgks.HGKSError as e:
        if e.code != hgks.HGKS_ENONPHYSICAL:
            raise
    out = s.hgks_get_state()
    st = s.hgks_get_stats()
    s.hgks_destroy_solver()
    return out, st
