"""The continuous-batching server: requests arriving while others run are admitted
as memory frees, advance in shared batched launches, and each result equals the
same request solved alone, bit for bit."""
import numpy as np
import pytest

from paper_2304_05572_gb300 import hgks, problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2304_05572_gb300 import _build
    _build.build()


def _small_trace():
    trace = P.served_trace(n_requests=10, rate=400.0, max_1d=600, max_2d=72, max_ns=96)
    for r in trace:
        r["t_end"] = 0.1 * r["t_end"]          # keep the test short
    return trace


def test_served_results_equal_alone_and_all_complete():
    from paper_2304_05572_gb300 import server
    trace = _small_trace()
    srv = server.Server(budget_bytes=4e9, steps_per_iter=3)
    res = srv.run(trace)
    assert set(res) == {r["id"] for r in trace}
    for r in trace:
        out, st = server.run_alone(r)
        got = res[r["id"]]
        assert got["status"] == st["status"]
        assert got["steps"] == st["steps"] and got["t"] == st["t"]
        assert np.array_equal(got["W"], out), r["kind"]
        assert got["latency"] >= 0.0
    assert srv.peak_resident >= 2            # requests overlapped on the device


def test_budget_limits_residency():
    from paper_2304_05572_gb300 import server
    trace = _small_trace()
    need = max(hgks.hgks_footprint_bytes(r["cfg"]) for r in trace)
    srv = server.Server(budget_bytes=need * 1.5, steps_per_iter=3)
    res = srv.run(trace)
    assert len(res) == len(trace)
    assert srv.peak_resident <= 2 or any(hgks.hgks_footprint_bytes(r["cfg"]) * 2 <= need * 1.5 for r in trace)
    for r in trace[:3]:
        out, _ = server.run_alone(r)
        assert np.array_equal(res[r["id"]]["W"], out)
