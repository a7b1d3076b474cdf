"""The allocation-free entry point hgks_step_noalloc, called through the C ABI.

Some callers cannot allocate device memory themselves (their framework's
allocator owns the GPU, or they cannot afford the synchronisation an
allocation may cause); for them hgks_step_noalloc takes one S2O4 step on
buffers they own, with its intermediates in the library's static device
scratch.  It runs the solver's own kernels, so its result must equal the
regular solver's step (hgks_create_solver / hgks_set_state / hgks_step /
hgks_get_state) bit for bit, on two calls in a row (the second call reuses the
scratch the first one left behind), and a non-physical step must show in its
status word.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2304_05572_gb300 import hgks, problems as P

pytestmark = pytest.mark.gpu


def solver_step(cfg, W):
    s = hgks.Solver(cfg)
    s.hgks_set_state(np.ascontiguousarray(W))
    assert s.hgks_step(1e300, 1) == 1
    out = s.hgks_get_state()
    s.hgks_destroy_solver()
    return out


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2304_05572_gb300 import _build
    _build.build()


def _case(name):
    if name == "riemann2d":
        return P.riemann4_2d(61, ny=47)[:2]
    if name == "sod1d":
        return P.sod_1d(300)[:2]
    if name == "vortex2d":
        return P.vortex_2d(64)[:2]
    # viscous shock tube: Navier-Stokes flux with the Prandtl fix, no-slip and symmetric walls
    return P.viscous_shock_tube(40, 20, Re=1000.0, prandtl=0.73)[:2]


@pytest.mark.parametrize("case", ["riemann2d", "sod1d", "vortex2d", "ns_tube"])
def test_noalloc_step_matches_solver_on_two_calls(case):
    import torch
    cfg, W = _case(case)
    stream = torch.cuda.Stream()
    W_in = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    W_out = torch.empty_like(W_in)
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    # first call, against the solver's step from the same state
    hgks.hgks_step_noalloc(cfg, W_in, W_out, stream, status=status)
    stream.synchronize()
    ref1 = solver_step(cfg, W)
    got1 = W_out.cpu().numpy()
    assert int(status.item()) == 0
    assert np.array_equal(got1, ref1)
    # second call in a row, from the result of the first, in place
    status.fill_(12345)
    hgks.hgks_step_noalloc(cfg, W_out, W_out, stream, status=status)
    stream.synchronize()
    ref2 = solver_step(cfg, ref1)
    got2 = W_out.cpu().numpy()
    assert int(status.item()) == 0
    assert np.array_equal(got2, ref2)
    assert not np.array_equal(got2, got1)


def test_noalloc_reports_a_nonphysical_step():
    """A state with a negative density: the solver's step fails with HGKS_ENONPHYSICAL, and
    the allocation-free step writes that code into the caller's status word (device or host
    memory); the next call on a good state clears it again."""
    import torch
    cfg, W = _case("riemann2d")
    bad = np.ascontiguousarray(W).copy()
    bad[0, 5, 5] = -1.0
    s = hgks.Solver(cfg)
    s.hgks_set_state(bad)
    with pytest.raises(hgks.HGKSError) as e:
        s.hgks_step(1e300, 1)
    assert e.value.code == hgks.HGKS_ENONPHYSICAL
    s.hgks_destroy_solver()
    W_bad = torch.from_numpy(bad).cuda()
    W_out = torch.empty_like(W_bad)
    st_dev = torch.zeros(1, dtype=torch.int32, device="cuda")
    hgks.hgks_step_noalloc(cfg, W_bad, W_out, status=st_dev)
    torch.cuda.synchronize()
    assert int(st_dev.item()) == hgks.HGKS_ENONPHYSICAL
    st_host = np.zeros(1, dtype=np.int32)
    hgks.hgks_step_noalloc(cfg, W_bad, W_out, status=st_host)
    torch.cuda.synchronize()
    assert int(st_host[0]) == hgks.HGKS_ENONPHYSICAL
    W_good = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    hgks.hgks_step_noalloc(cfg, W_good, W_out, status=st_dev)
    torch.cuda.synchronize()
    assert int(st_dev.item()) == 0


def test_noalloc_rejects_a_grid_beyond_the_scratch_and_wrong_buffers():
    import torch
    cfg, W, _ = P.riemann4_2d(128)
    assert hgks.hgks_footprint_bytes(cfg) > 8 * 1024 * 1024
    W_in = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    with pytest.raises(hgks.HGKSError) as e:
        hgks.hgks_step_noalloc(cfg, W_in, torch.empty_like(W_in))
    assert e.value.code == hgks.HGKS_EINVAL and "static scratch" in str(e.value)
    cfg, W = _case("riemann2d")
    W_in = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    with pytest.raises(ValueError):
        hgks.hgks_step_noalloc(cfg, W_in, torch.empty(W_in.numel() - 1, dtype=torch.float64, device="cuda"))
