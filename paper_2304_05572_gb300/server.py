"""Continuous-batching solve server on one GPU.

Requests (a configuration, an initial state and an end time) arrive over time.
The server admits a request as soon as its arrival time has passed and the
device memory its solver needs (hgks_footprint_bytes) fits in the budget;
admitted solves keep their state resident on the device and advance together:
every iteration issues one group of S2O4 steps (hgks_batch_step, CUDA graph
replay) per batch, all batches on their own streams so that they overlap on the
device: one batch per dimension (optionally the 2D solves spread over a few
batches, a new solve joining the one with the fewest resident cells); the
batch whose step is faster takes more steps, so that all take about the same
device time, and newly admitted solves join the ones already running.  A solve retires at its
end time, when its state turned non-physical (the scheme has no positivity limiter; the status is
reported with the result) or when its request is cancelled; its state is
copied back, its memory freed and its latency (completion minus arrival,
queueing included) recorded.  A request whose configuration the library
rejects, or whose memory alone exceeds the budget, is answered at once with a
"rejected" status and takes no device memory.

Each solve's arithmetic is independent of the others (batched launches never
mix solvers inside a block), so a result is bit-identical alone and in the mix.
All numerical work runs in the CUDA library; this module only schedules, over a
small backend interface (GpuBackend here; the scheduling logic is the same for
any object with its methods).
"""
from __future__ import annotations

import time

import numpy as np

from . import hgks

STATUS_OK = 0
STATUS_NONPHYSICAL = hgks.HGKS_ENONPHYSICAL
STATUS_REJECTED = "rejected"
STATUS_CANCELLED = "cancelled"


class GpuBackend:
    """Solvers on the current CUDA device, advanced by hgks batches: one per dimension for 1D,
    `groups_2d` for 2D, each batch on its own stream.  A batch is addressed by its key, the
    dimension or a (dimension, group) pair."""

    def __init__(self, stream=None, autotune: bool = False, groups_2d: int = 1):
        import torch
        self._torch = torch
        # 1D batches (small, latency-bound launches) overlap on the device with the 2D ones, at a
        # higher priority, so that their few blocks are dispatched as soon as a slot frees instead
        # of queueing behind the 2D grids (their solves take many short steps and would otherwise
        # set the tail).  groups_2d > 1 splits the 2D solves over that many batches on separate
        # streams, so that the latency-bound kernels of one group overlap the others' work; one
        # batch measured faster (a 16-request burst of small solves: 69.4 Mcell-stage/s with one
        # 2D batch, 65.5 with two, 57 with three or four), so it is the default.  `stream`, if
        # given, serves 2D group 0.
        self.groups = {1: 1, 2: max(1, int(groups_2d))}
        self._stream2 = stream
        self.streams = {}
        self.autotune = autotune
        self._batches = {}        # key -> (tuple of handles, Batch)
        self._events = {}         # key -> (start, end, nsteps) of the last enqueued group of steps
        self._ms_per_step = {}    # key -> device time per batched step of the last group

    def stream(self, key):
        """The stream of a batch key (created on first use)."""
        st = self.streams.get(key)
        if st is None:
            dim, group = key if isinstance(key, tuple) else (key, 0)
            if dim == 2 and group == 0 and self._stream2 is not None:
                st = self._stream2
            else:
                st = self._torch.cuda.Stream(priority=-1 if dim == 1 else 0)
            self.streams[key] = st
        return st

    def footprint(self, cfg) -> int:
        """Device bytes of a solver of cfg; 0 if the library rejects the configuration."""
        try:
            return int(hgks.hgks_footprint_bytes(cfg))
        except (KeyError, TypeError, ValueError):
            return 0

    def create(self, cfg, W):
        s = hgks.Solver(cfg, stream=self.stream((int(cfg["dim"]), 0)))
        s.hgks_set_state(np.ascontiguousarray(W))
        return s

    def _batch(self, key, handles):
        """The key's batch over exactly these solvers: created once, then updated in place
        when the resident set changes (no reallocation, graph updated rather than rebuilt)."""
        members = tuple(handles)
        cur = self._batches.get(key)
        if cur is not None and cur[0] == members:
            return cur[1]
        if cur is not None:
            b = cur[1]
            b.hgks_batch_update(list(members))
        else:
            b = hgks.Batch(list(members), stream=self.stream(key))
        self._batches[key] = (members, b)
        return b

    def step(self, key, handles, t_ends, nsteps):
        """Enqueue nsteps batched steps of the given solvers (no wait), timed by CUDA events."""
        b = self._batch(key, handles)
        st = self.stream(key)
        e0, e1 = self._torch.cuda.Event(enable_timing=True), self._torch.cuda.Event(enable_timing=True)
        e0.record(st)
        b.hgks_batch_step(t_ends, nsteps=nsteps, graph=True, autotune=self.autotune)
        e1.record(st)
        self._events[key] = (e0, e1, nsteps)

    def sync(self, key):
        """Wait for the key's batch; (t, status, steps) per solver in step() order."""
        b = self._batches[key][1]
        b.hgks_batch_sync()
        ev = self._events.pop(key, None)
        if ev is not None and ev[2] > 0:
            self._ms_per_step[key] = ev[0].elapsed_time(ev[1]) / ev[2]
        return list(zip(*b.hgks_batch_status()))

    def ms_per_step(self, key):
        """Device time of one batched step of the key's last group of steps (None before the first)."""
        return self._ms_per_step.get(key)

    def fetch(self, handle):
        return handle.hgks_get_state()

    def release(self, handle):
        handle.hgks_destroy_solver()

    def close(self):
        for _, b in self._batches.values():
            b.hgks_batch_destroy()
        self._batches.clear()


class Server:
    def __init__(self, budget_bytes: float, stream=None, steps_per_iter: int = 4, autotune: bool = False,
                 backend=None, clock=time.perf_counter, groups_2d: int = 1):
        self.budget = float(budget_bytes)
        self.backend = backend if backend is not None else GpuBackend(stream, autotune, groups_2d)
        self.steps_per_iter = int(steps_per_iter)
        self.max_steps_factor = 16
        self.clock = clock
        self.used = 0.0
        self.active = {}          # id -> dict(req, handle, bytes, t_admit)
        self.results = {}         # id -> dict(W, latency, admitted, completed, steps, t, status, cells)
        self.iterations = 0
        self.peak_resident = 0

    def _key(self, req):
        """The batch a new solve joins: its dimension, or, where the backend splits a dimension
        over several batches (its `groups`), the (dimension, group) whose resident solves hold
        the fewest cells.  A solve stays in its batch until it retires."""
        dim = int(req["cfg"]["dim"])
        ng = int(getattr(self.backend, "groups", {}).get(dim, 1))
        if ng <= 1:
            return dim
        load = [0] * ng
        for a in self.active.values():
            k = a["key"]
            if isinstance(k, tuple) and k[0] == dim:
                load[k[1]] += int(np.prod(np.shape(a["req"]["W"])[1:]))
        return (dim, int(np.argmin(load)))

    def _admit(self, req, now):
        h = self.backend.create(req["cfg"], req["W"])
        self.active[req["id"]] = dict(req=req, handle=h, bytes=req["bytes"], t_admit=now, key=self._key(req))
        self.used += req["bytes"]
        self.peak_resident = max(self.peak_resident, len(self.active))

    def _answer(self, req, now, status, W=None, t=0.0, steps=0, admitted=None):
        self.results[req["id"]] = dict(W=W, latency=now - req["arrival"], admitted=admitted, completed=now,
                                       steps=int(steps), t=t, status=status,
                                       cells=int(np.prod(np.shape(req["W"])[1:])))

    def _retire(self, rid, now, t, status, steps):
        a = self.active.pop(rid)
        W = self.backend.fetch(a["handle"])
        self.backend.release(a["handle"])
        self.used -= a["bytes"]
        self._answer(a["req"], now, status, W=W, t=t, steps=steps, admitted=a["t_admit"])

    def _steps_per_batch(self, by_dim):
        """Steps of each batch in this iteration: the batch whose step takes longest on the
        device does steps_per_iter steps, the others as many as fit in the same device time (up
        to max_steps_factor times more), so that no batch waits idle for another at the end of
        an iteration.  Without timings (first iterations, or a backend that reports none) every
        batch does steps_per_iter."""
        ms = {d: getattr(self.backend, "ms_per_step", lambda d: None)(d) for d in by_dim}
        known = [v for v in ms.values() if v]
        if len(by_dim) < 2 or len(known) < len(by_dim):
            return {d: self.steps_per_iter for d in by_dim}
        budget = self.steps_per_iter * max(known)
        return {d: max(1, min(self.steps_per_iter * self.max_steps_factor, int(budget / ms[d])))
                for d in by_dim}

    def run(self, trace, time_scale: float = 1.0):
        """Serve a list of requests (dicts with id, arrival [s], cfg, W, t_end and optionally
        cancel_at [s]) in arrival order; times are scaled by time_scale.  Returns the results
        dict, one entry per request."""
        pending = []
        for r in sorted(trace, key=lambda r: r["arrival"]):
            q = dict(r, arrival=r["arrival"] * time_scale)
            if r.get("cancel_at") is not None:
                q["cancel_at"] = r["cancel_at"] * time_scale
            q["bytes"] = float(self.backend.footprint(r["cfg"]))
            pending.append(q)
        t0 = self.clock()
        qi = 0
        while qi < len(pending) or self.active:
            now = self.clock() - t0
            # admission in arrival order (FIFO): a request that cannot fit waits, and so do the ones behind it
            while qi < len(pending) and pending[qi]["arrival"] <= now:
                req = pending[qi]
                if not (req["bytes"] > 0 and req["bytes"] <= self.budget):
                    self._answer(req, now, STATUS_REJECTED)       # invalid, or larger than the whole budget
                    qi += 1
                    continue
                if req.get("cancel_at") is not None and req["cancel_at"] <= now:
                    self._answer(req, now, STATUS_CANCELLED)      # cancelled while queued
                    qi += 1
                    continue
                if self.used + req["bytes"] > self.budget:
                    break
                self._admit(req, now)
                qi += 1
            for rid in [rid for rid, a in self.active.items()
                        if a["req"].get("cancel_at") is not None and a["req"]["cancel_at"] <= now]:
                self._retire(rid, now, None, STATUS_CANCELLED, 0)
            if not self.active:
                if qi < len(pending):
                    wait = pending[qi]["arrival"] - now
                    if wait > 0:
                        time.sleep(min(0.01, wait))
                continue
            by_dim = {}
            for rid, a in self.active.items():
                by_dim.setdefault(a["key"], []).append(rid)
            nsteps = self._steps_per_batch(by_dim)
            for dim, ids in by_dim.items():             # enqueue every batch first (they overlap)
                ids.sort()
                self.backend.step(dim, [self.active[i]["handle"] for i in ids],
                                  [self.active[i]["req"]["t_end"] for i in ids], nsteps[dim])
            self.iterations += 1
            finished = []
            for dim, ids in by_dim.items():
                for rid, (t, st, n) in zip(ids, self.backend.sync(dim)):
                    te = self.active[rid]["req"]["t_end"]
                    # a solve retires at its end time, or with its error once its state turned non-physical
                    if st != 0 or te - t <= 1e-12 * max(1.0, abs(te)):
                        finished.append((rid, t, st, n))
            now = self.clock() - t0
            for rid, t, st, n in finished:
                self._retire(rid, now, t, st, n)
        self.backend.close()
        self.wall = self.clock() - t0
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
