"""Batched execution: solvers of uneven size advanced together by shared launches
(hgks_batch_*) must produce exactly the bits each produces when stepped alone,
with or without graph replay and block-size autotuning, and each solver must stop
at its own end time."""
import numpy as np
import pytest

from paper_2304_05572_gb300 import hgks, problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2304_05572_gb300 import _build
    _build.build()


def _cases_2d():
    out = []
    for k, (nx, ny) in enumerate([(16, 16), (37, 29), (64, 64), (23, 71), (48, 20)]):
        cfg, W, _ = P.riemann4_2d(nx, ny=ny, seed=20230412 + k)
        out.append((cfg, W))
    cfg, W, _ = P.vortex_2d(32)
    out.append((cfg, W))
    cfg, W, _ = P.viscous_shock_tube(40, 20, Re=300.0)
    out.append((cfg, W))
    # Navier-Stokes with the Prandtl fix (its own flux variant)
    cfg, W, _ = P.viscous_shock_tube(48, 24, Re=1000.0, prandtl=0.73)
    out.append((cfg, W))
    # WENO-AO everywhere at 128x128: every compacted pass holds 34572 to 66048 items, above the
    # size from which the passes give each item one lane (the others here use lane groups)
    cfg, W, _ = P.random_smooth_2d(128, 128)
    out.append((dict(cfg, recon_mode="wenoao"), W))
    return out


def _alone(cfg, W, t_end, steps):
    s = hgks.Solver(cfg)
    s.hgks_set_state(np.ascontiguousarray(W))
    s.hgks_step(t_end, steps, wait=False)     # a latched non-physical state shows in the stats
    st = s.hgks_get_stats()
    out, t, n = s.hgks_get_state(), st["t"], st["steps"]
    s.hgks_destroy_solver()
    return out, t, n


@pytest.mark.parametrize("graph,autotune", [(False, False), (True, False), (True, True)])
def test_batch_2d_bitwise_equal_to_alone(graph, autotune):
    import torch
    cases = _cases_2d()
    t_end = [0.004 * (1 + k) for k in range(len(cases))]
    steps = 9
    stream = torch.cuda.Stream()
    solvers = []
    for cfg, W in cases:
        s = hgks.Solver(cfg, stream=stream)
        s.hgks_set_state(np.ascontiguousarray(W))
        solvers.append(s)
    b = hgks.Batch(solvers, stream=stream)
    b.hgks_batch_step(t_end, nsteps=steps, graph=graph, autotune=autotune)
    active, failed = b.hgks_batch_sync()
    assert failed == 0
    for k, ((cfg, W), s) in enumerate(zip(cases, solvers)):
        ref, t_ref, n_ref = _alone(cfg, W, t_end[k], steps)
        got = s.hgks_get_state()
        assert np.array_equal(got, ref), k
        assert s.hgks_get_time() == t_ref
        assert s.hgks_get_stats()["steps"] == n_ref
    assert active == sum(1 for k, (cfg, W) in enumerate(cases)
                         if t_end[k] - solvers[k].hgks_get_time() > 1e-12)
    tpb, nst = b.hgks_batch_info()
    assert nst == steps and all(t in (32, 64, 128, 256, 512) for t in tpb)
    b.hgks_batch_destroy()


def test_batch_1d_and_continuation():
    import torch
    cases = [P.sod_1d(n)[:2] for n in (50, 200, 333)] + [P.blast_1d(120)[:2]]
    # WENO-AO everywhere on 20000 cells: 40002 troubled sides per pass, one lane each
    cfg, W, _ = P.sod_1d(20000)
    cases.append((dict(cfg, recon_mode="wenoao"), W))
    stream = torch.cuda.Stream()
    solvers = []
    for cfg, W in cases:
        s = hgks.Solver(cfg, stream=stream)
        s.hgks_set_state(np.ascontiguousarray(W))
        solvers.append(s)
    b = hgks.Batch(solvers, stream=stream)
    t_end = [0.05, 0.02, 0.2, 0.01, 0.002]
    for _ in range(4):                    # several calls continue where the last stopped
        b.hgks_batch_step(t_end, nsteps=5, graph=True)
    b.hgks_batch_sync()
    for k, ((cfg, W), s) in enumerate(zip(cases, solvers)):
        ref, t_ref, n_ref = _alone(cfg, W, t_end[k], 20)
        assert np.array_equal(s.hgks_get_state(), ref), k
        assert s.hgks_get_time() == t_ref
    b.hgks_batch_destroy()


def test_batch_rejects_mixed_dimensions():
    c1, W1, _ = P.sod_1d(40)
    c2, W2, _ = P.riemann4_2d(16)
    s1, s2 = hgks.Solver(c1), hgks.Solver(c2)
    with pytest.raises(hgks.HGKSError) as e:
        hgks.Batch([s1, s2])
    assert e.value.code == hgks.HGKS_EINVAL


def test_failed_solver_stops_alone_and_others_continue():
    """A four-quadrant case whose state turns non-physical within a few steps (the scheme
    has no positivity limiter; the oracle stops on it too) stops at the same step and with
    the same bits in a batch as alone, and does not stop the other solvers."""
    import torch
    bad = P.riemann4_2d(32, seed=P.BATCH_SEED + 1 + 3)[:2]
    good = [P.riemann4_2d(n, seed=P.BATCH_SEED + 1 + k)[:2] for k, n in ((0, 24), (1, 40))]
    # the other two seeds of the batched set that break (at steps 6 and 7)
    bad2 = [P.riemann4_2d(n, seed=P.BATCH_SEED + 1 + k)[:2] for k, n in ((214, 40), (224, 48))]
    cases = [good[0], bad, good[1]] + bad2
    stream = torch.cuda.Stream()
    solvers = []
    for cfg, W in cases:
        s = hgks.Solver(cfg, stream=stream)
        s.hgks_set_state(np.ascontiguousarray(W))
        solvers.append(s)
    b = hgks.Batch(solvers, stream=stream)
    b.hgks_batch_step([1e9] * len(cases), nsteps=12, graph=True)
    active, failed = b.hgks_batch_sync()
    assert failed == 3 and active == 2
    ts, sts, ns = b.hgks_batch_status()
    for s, t, st, n in zip(solvers, ts, sts, ns):
        ref = s.hgks_get_stats()
        assert (t, st, n) == (ref["t"], ref["status"], ref["steps"])
    for (cfg, W), s in zip(cases, solvers):
        ref, t_ref, n_ref = _alone(cfg, W, 1e9, 12)
        st = s.hgks_get_stats()
        assert st["steps"] == n_ref and st["t"] == t_ref
        assert np.array_equal(s.hgks_get_state(), ref, equal_nan=True)
    assert solvers[1].hgks_get_stats()["status"] == hgks.HGKS_ENONPHYSICAL
    assert solvers[1].hgks_get_stats()["steps"] < 12
    assert solvers[0].hgks_get_stats()["steps"] == 12 and solvers[2].hgks_get_stats()["steps"] == 12
    b.hgks_batch_destroy()


def test_solver_streams_are_ordered_with_the_batch_stream():
    """Solvers on their own streams, the batch on a third: a state set on a solver's stream
    just before hgks_batch_step is the one the batch advances, and hgks_get_state on the
    solver's stream right after it (no hgks_batch_sync) sees the advanced state."""
    import torch
    cases = [P.riemann4_2d(n, seed=P.BATCH_SEED + 1 + k)[:2] for k, n in ((0, 40), (1, 56))]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    solvers = [hgks.Solver(cfg, stream=st) for (cfg, _), st in zip(cases, streams)]
    zero = [np.zeros_like(W) + 1.0 for _, W in cases]
    for s, z in zip(solvers, zero):
        s.hgks_set_state(np.ascontiguousarray(z))
    b = hgks.Batch(solvers, stream=torch.cuda.Stream())
    for s, (cfg, W) in zip(solvers, cases):
        s.hgks_set_state(np.ascontiguousarray(W))      # enqueued on the solver's own stream
    b.hgks_batch_step([1e9, 1e9], nsteps=6, graph=True)
    for s, (cfg, W) in zip(solvers, cases):
        ref, t_ref, n_ref = _alone(cfg, W, 1e9, 6)
        assert np.array_equal(s.hgks_get_state(), ref)
        assert s.hgks_get_time() == t_ref
    b.hgks_batch_destroy()


def test_batch_mixes_prandtl_fixed_and_bgk_solvers():
    """Navier-Stokes solvers with Pr = 0.73 (the energy-flux fix) and Pr = 1 in one batch:
    the batched flux launch serves both kinds of blocks, each bit-identical to its solo run."""
    import torch
    cases = [P.viscous_shock_tube(40, 20, Re=500.0, prandtl=0.73)[:2],
             P.viscous_shock_tube(48, 24, Re=300.0)[:2],
             P.viscous_shock_tube(32, 16, Re=800.0, prandtl=0.73)[:2]]
    stream = torch.cuda.Stream()
    solvers = []
    for cfg, W in cases:
        s = hgks.Solver(cfg, stream=stream)
        s.hgks_set_state(np.ascontiguousarray(W))
        solvers.append(s)
    b = hgks.Batch(solvers, stream=stream)
    b.hgks_batch_step([1e9] * 3, nsteps=5, graph=True)
    b.hgks_batch_sync()
    for (cfg, W), s in zip(cases, solvers):
        ref, t_ref, _ = _alone(cfg, W, 1e9, 5)
        assert np.array_equal(s.hgks_get_state(), ref)
        assert s.hgks_get_time() == t_ref
    b.hgks_batch_destroy()


@pytest.mark.parametrize("graph", [True, False])
def test_batch_update_changes_members_and_keeps_bits(graph):
    """hgks_batch_update: a batch of A and B takes 3 steps, is updated in place to B, C, D
    (more members than before: the device arrays grow) and takes 4 more, then to D alone
    (fewer: arrays reused) and takes 2 more.  Every solver's state equals its solo run with
    the same number of steps, with and without the (updated) CUDA graph."""
    import torch
    cases = _cases_2d()[:4]
    stream = torch.cuda.Stream()
    solvers = []
    for cfg, W in cases:
        s = hgks.Solver(cfg, stream=stream)
        s.hgks_set_state(np.ascontiguousarray(W))
        solvers.append(s)
    A, B, C, D = solvers
    b = hgks.Batch([A, B], stream=stream)
    b.hgks_batch_step([1.0, 1.0], nsteps=3, graph=graph)
    b.hgks_batch_sync()
    b.hgks_batch_update([B, C, D])
    b.hgks_batch_step([1.0, 1.0, 1.0], nsteps=4, graph=graph)
    b.hgks_batch_sync()
    b.hgks_batch_update([D])
    b.hgks_batch_step([1.0], nsteps=2, graph=graph)
    b.hgks_batch_sync()
    b.hgks_batch_destroy()
    for (cfg, W), s, n in zip(cases, solvers, (3, 7, 4, 6)):
        ref, _, n_ref = _alone(cfg, W, 1.0, n)
        assert int(s.hgks_get_stats()["steps"]) == n_ref == n
        assert np.array_equal(s.hgks_get_state(), ref)
    for s in solvers:
        s.hgks_destroy_solver()
