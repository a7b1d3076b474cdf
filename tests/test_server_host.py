"""Scheduling logic of the continuous-batching server on the CPU, with a simulated backend
in place of the GPU library: admission in arrival order under the memory budget, answers to
requests that cannot be served (rejected, cancelled), retirement at the end time or on a
non-physical state, and latency accounting.  Failures are made on the host (a backend that
reports a non-physical state, a config it rejects, a cancellation); nothing touches a GPU."""
import numpy as np
import pytest

from paper_2304_05572_gb300 import server


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """Each solve advances by a fixed dt per step, clipped to its end time; a solve whose cfg
    has fail_after = k latches a non-physical status after k steps.  Every step advances the
    fake clock by 1 ms, so latencies are deterministic."""

    def __init__(self, clock, bad_dim=None):
        self.clock = clock
        self.created, self.released = [], []
        self.pending = {}
        self.bad_dim = bad_dim

    def footprint(self, cfg):
        if cfg.get("invalid"):
            return 0
        return int(cfg["bytes"])

    def create(self, cfg, W):
        h = dict(cfg=cfg, W=np.array(W, copy=True), t=0.0, steps=0, status=0)
        self.created.append(h)
        return h

    def step(self, dim, handles, t_ends, nsteps):
        self.pending[dim] = list(handles)
        for h, te in zip(handles, t_ends):
            for _ in range(nsteps):
                if h["status"] or te - h["t"] <= 1e-12 * max(1.0, abs(te)):
                    break
                dt = min(h["cfg"]["dt"], te - h["t"])
                h["t"] += dt
                h["steps"] += 1
                h["W"] = h["W"] + 1.0
                if h["cfg"].get("fail_after") == h["steps"]:
                    h["status"] = server.STATUS_NONPHYSICAL
        self.clock.t += 1e-3 * nsteps

    def sync(self, dim):
        return [(h["t"], h["status"], h["steps"]) for h in self.pending[dim]]

    def fetch(self, h):
        return h["W"]

    def release(self, h):
        self.released.append(h)

    def close(self):
        pass


def _req(i, arrival, t_end, dt, nbytes, dim=2, **kw):
    return dict(id=i, arrival=arrival, t_end=t_end, W=np.zeros((dim + 2, 2, 2)),
                cfg=dict(dim=dim, dt=dt, bytes=nbytes, **kw))


def test_admission_budget_fifo_and_latency():
    clock = FakeClock()
    be = FakeBackend(clock)
    trace = [_req(0, 0.0, 1.0, 0.25, 60), _req(1, 0.0, 0.5, 0.25, 60), _req(2, 0.0, 0.5, 0.25, 30, dim=1)]
    srv = server.Server(budget_bytes=100, steps_per_iter=1, backend=be, clock=clock)
    res = srv.run(trace)
    assert set(res) == {0, 1, 2}
    # 1 does not fit beside 0 and waits for it to retire; 2 would fit beside 0 but is queued
    # behind 1 (admission is first-in first-out, so a large request is never starved)
    assert res[0]["admitted"] == 0.0
    assert res[1]["admitted"] == res[0]["completed"] and res[2]["admitted"] == res[1]["admitted"]
    assert srv.peak_resident == 2 and srv.used == 0.0
    for r in trace:
        got = res[r["id"]]
        assert got["status"] == server.STATUS_OK and got["t"] == r["t_end"]
        assert got["steps"] == int(np.ceil(r["t_end"] / r["cfg"]["dt"]))
        assert np.all(got["W"] == got["steps"])
        assert got["latency"] == pytest.approx(got["completed"] - r["arrival"])
    assert len(be.released) == len(be.created) == 3


def test_rejected_cancelled_and_failed_requests_do_not_stop_the_others():
    clock = FakeClock()
    be = FakeBackend(clock)
    trace = [_req(0, 0.0, 1.0, 0.1, 10),
             _req(1, 0.0, 1.0, 0.1, 10, invalid=True),        # the library rejects its config
             _req(2, 0.0, 1.0, 0.1, 1000),                    # alone larger than the budget
             _req(3, 0.0, 1.0, 0.1, 10, fail_after=3),        # non-physical after 3 steps
             dict(_req(4, 0.0, 1.0, 0.1, 10), cancel_at=0.004),
             dict(_req(5, 0.001, 1.0, 0.1, 10), cancel_at=0.0005)]
    srv = server.Server(budget_bytes=100, steps_per_iter=2, backend=be, clock=clock)
    res = srv.run(trace)
    assert res[1]["status"] == server.STATUS_REJECTED and res[1]["W"] is None
    assert res[2]["status"] == server.STATUS_REJECTED
    assert res[3]["status"] == server.STATUS_NONPHYSICAL and res[3]["steps"] == 3
    assert res[4]["status"] == server.STATUS_CANCELLED and res[4]["completed"] >= 0.004
    assert res[5]["status"] == server.STATUS_CANCELLED and res[5]["admitted"] is None
    assert res[0]["status"] == server.STATUS_OK and res[0]["steps"] == 10
    assert len(be.created) == 3 and len(be.released) == 3 and srv.used == 0.0


def test_arrivals_in_the_future_wait_for_their_time():
    clock = FakeClock()
    be = FakeBackend(clock)
    # the second request arrives after the first has finished: the server idles until then
    trace = [_req(0, 0.0, 0.2, 0.1, 10), _req(1, 0.0005, 0.2, 0.1, 10)]

    def tick():
        clock.t += 1e-4
        return clock.t
    srv = server.Server(budget_bytes=100, steps_per_iter=1, backend=be, clock=tick)
    res = srv.run(trace)
    assert res[1]["admitted"] >= 0.0005 - 1e-4
    assert all(r["status"] == server.STATUS_OK for r in res.values())


class TimedBackend(FakeBackend):
    """FakeBackend that reports a device time per batched step for each dimension."""

    def __init__(self, clock, ms):
        super().__init__(clock)
        self.ms = ms
        self.requested = []

    def step(self, dim, handles, t_ends, nsteps):
        self.requested.append((dim, nsteps))
        super().step(dim, handles, t_ends, nsteps)

    def ms_per_step(self, dim):
        return self.ms[dim]


def test_faster_dimension_takes_more_steps_per_iteration():
    clock = FakeClock()
    be = TimedBackend(clock, {1: 0.2, 2: 1.6})
    srv = server.Server(budget_bytes=1e9, steps_per_iter=4, backend=be, clock=clock)
    trace = [_req(0, 0.0, 0.5, 0.001, 10, dim=1), _req(1, 0.0, 0.5, 0.01, 10, dim=2)]
    res = srv.run(trace)
    assert all(r["status"] == 0 for r in res.values())
    first = {}
    for dim, n in be.requested:
        first.setdefault(dim, n)
    assert first == {2: 4, 1: 32}            # 1.6 ms per 2D step x 4 steps = 32 1D steps of 0.2 ms
    # with one dimension resident only, the plain steps_per_iter applies
    be2 = TimedBackend(FakeClock(), {1: 0.2, 2: 1.6})
    srv2 = server.Server(budget_bytes=1e9, steps_per_iter=4, backend=be2, clock=be2.clock)
    srv2.run([_req(0, 0.0, 0.2, 0.01, 10, dim=1)])
    assert {n for _, n in be2.requested} == {4}


class GroupedBackend(FakeBackend):
    """FakeBackend that splits the 2D solves over two batches, as the GPU backend does."""
    groups = {1: 1, 2: 2}

    def __init__(self, clock):
        super().__init__(clock)
        self.members = {}

    def step(self, key, handles, t_ends, nsteps):
        self.members.setdefault(key, set()).update(id(h) for h in handles)
        super().step(key, handles, t_ends, nsteps)


def test_2d_solves_join_the_least_loaded_batch():
    clock = FakeClock()
    be = GroupedBackend(clock)
    srv = server.Server(budget_bytes=1e9, steps_per_iter=2, backend=be, clock=clock)
    big = dict(_req(0, 0.0, 1.0, 0.125, 10), W=np.zeros((4, 40, 40)))
    small = [dict(_req(k, 0.0, 0.5, 0.125, 10), W=np.zeros((4, 10, 10))) for k in (1, 2, 3)]
    trace = [big] + small + [_req(4, 0.0, 0.25, 0.125, 10, dim=1)]
    res = srv.run(trace)
    for r in trace:
        got = res[r["id"]]
        assert got["status"] == server.STATUS_OK and got["t"] == r["t_end"]
        assert got["steps"] == int(np.ceil(r["t_end"] / r["cfg"]["dt"]))
        assert np.all(got["W"] == got["steps"])
    # the 40x40 solve holds batch (2, 0) alone; the three 10x10 ones go to (2, 1), the lighter
    # batch at each admission; the 1D solve keeps its dimension's single batch
    assert set(be.members) == {(2, 0), (2, 1), 1}
    assert len(be.members[(2, 0)]) == 1 and len(be.members[(2, 1)]) == 3 and len(be.members[1]) == 1
