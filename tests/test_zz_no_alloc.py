"""The allocation-free entry point hgks_step_noalloc, called through the C ABI.

Some callers cannot allocate device memory themselves (their framework's
allocator owns the GPU, or they cannot afford the synchronisation an
allocation may cause); for them hgks_step_noalloc takes one S2O4 step on
buffers they own, with its intermediates in the library's static device
scratch.  Its result must equal the regular solver's step (hgks_create_solver
/ hgks_set_state / hgks_step / hgks_get_state) within the per-step tolerance of
the parity tests, on two calls in a row (the second call reuses the scratch the
first one left behind).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2304_05572_gb300 import hgks, problems as P

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-11


def rel_diff(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    scale = np.abs(b).max(axis=1)
    scale = np.maximum(scale, 1e-3 * scale.max())
    return float(np.max(np.abs(a - b).max(axis=1) / scale))


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


@pytest.mark.parametrize("case", ["riemann2d", "sod1d", "vortex2d"])
def test_noalloc_step_matches_solver_on_two_calls(case):
    import torch
    if case == "riemann2d":
        cfg, W, _ = P.riemann4_2d(61, ny=47)
    elif case == "sod1d":
        cfg, W, _ = P.sod_1d(300)
    else:
        cfg, W, _ = P.vortex_2d(64)
    stream = torch.cuda.Stream()
    W_in = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    W_out = torch.empty_like(W_in)
    # first call, against the solver's step from the same state
    hgks.hgks_step_noalloc(cfg, W_in, W_out, stream)
    stream.synchronize()
    ref1 = solver_step(cfg, W)
    got1 = W_out.cpu().numpy()
    assert rel_diff(got1, ref1) <= STEP_TOL
    # second call in a row, from the result of the first, in place
    hgks.hgks_step_noalloc(cfg, W_out, W_out, stream)
    stream.synchronize()
    ref2 = solver_step(cfg, ref1)
    got2 = W_out.cpu().numpy()
    assert rel_diff(got2, ref2) <= STEP_TOL
    assert not np.array_equal(got2, got1)


def test_noalloc_rejects_a_grid_beyond_the_scratch():
    import torch
    cfg, W, _ = P.riemann4_2d(128)
    assert hgks.hgks_footprint_bytes(cfg) > 8 * 1024 * 1024
    W_in = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    with pytest.raises(hgks.HGKSError) as e:
        hgks.hgks_step_noalloc(cfg, W_in, torch.empty_like(W_in))
    assert e.value.code == hgks.HGKS_EINVAL and "static scratch" in str(e.value)
