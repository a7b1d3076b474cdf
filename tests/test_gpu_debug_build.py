"""The debug build of the library (HGKS_DEBUG_BOUNDS: every global load and store of every
kernel checked against the solver's device buffers, an access outside them skipped and
counted, nothing trapping) runs the same scheme: on a 2D Riemann problem, a 1D Sod tube, a Navier-Stokes tube, a
batch and the allocation-free step its results equal the normal build's to round-off, and
it records no out-of-range access."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2304_05572_gb300 import hgks

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2304_05572_gb300 import hgks, problems as P
out = {}
for name, (cfg, W, _) in [("riemann", P.riemann4_2d(37, ny=29)), ("sod", P.sod_1d(120)),
                          ("ns", P.viscous_shock_tube(40, 20, Re=1000.0, prandtl=0.73))]:
    Wg, t, n = hgks.run(cfg, W, 1.0, max_steps=6)
    out[name] = Wg.tolist()
cases = [P.riemann4_2d(n, seed=s) for n, s in ((20, 3), (33, 5))]
sv = [hgks.Solver(c) for c, W, _ in cases]
for s, (c, W, _) in zip(sv, cases):
    s.hgks_set_state(W)
b = hgks.Batch(sv)
b.hgks_batch_step([1.0, 1.0], nsteps=3, graph=False)
b.hgks_batch_sync()
out["batch"] = [s.hgks_get_state().tolist() for s in sv]
b.hgks_batch_destroy()
import torch
cfg, W, _ = P.riemann4_2d(24, ny=20)
Wd = torch.from_numpy(np.ascontiguousarray(W)).cuda()
Wo = torch.empty_like(Wd)
hgks.hgks_step_noalloc(cfg, Wd, Wo)
torch.cuda.synchronize()
out["noalloc"] = Wo.cpu().numpy().tolist()
out["bounds"] = list(hgks.hgks_debug_bounds())
print(json.dumps(out))
'''


def _run(debug):
    env = dict(os.environ)
    if debug:
        env["HGKS_DEBUG_BOUNDS"] = "1"
    else:
        env.pop("HGKS_DEBUG_BOUNDS", None)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + RUN], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_same_results_and_no_out_of_range_access():
    from paper_2304_05572_gb300 import _build
    _build.build()
    _build.build(debug=True)
    dbg, ref = _run(True), _run(False)
    assert dbg["bounds"][0] is True and ref["bounds"] == [False, 0, 0]
    assert dbg["bounds"][1] == 0, dbg["bounds"]
    # the checks change the compiled code around the loads, so the free-order parts (the flux,
    # the tangential WENO-AO) may contract products into FMAs differently: the builds agree to
    # round-off, within the per-step parity tolerance
    pairs = [(dbg[k], ref[k], k) for k in ("riemann", "sod", "ns", "noalloc")]
    pairs += [(x, y, "batch %d" % i) for i, (x, y) in enumerate(zip(dbg["batch"], ref["batch"]))]
    for x, y, key in pairs:
        a, b = np.array(x), np.array(y)
        assert a.shape == b.shape
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), key
