"""GPU parity at the sizes of the benchmark configurations.

* The 2D Navier-Stokes viscous shock tube (Sec. 3.6 set-up) at Re = 1000, Pr = 0.73:
  the first 20 steps at 250 x 125 and the first 2 steps at 1000 x 500, each step from
  the oracle's state (identical dt and first-stage flags, state within 1e-11); and the
  whole run to t = 1 at 250 x 125 against the oracle's final state stored by
  tests/golden/make_ns_tube_golden.py.
* The isentropic vortex (strength 5, periodic [0,10]^2, tau = 0) at 100^2 and 200^2
  to t = 2 against the oracle within 1e-9 (a smooth case).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2304_05572_gb300 import hgks, problems as P
from test_gpu_parity import FINAL_TOL, check_step, rel_diff

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ns_tube_250x125_t1.txt")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2304_05572_gb300 import _build
    _build.build()
    oracle.build()


def _read_golden(path):
    meta, blocks, cur = {}, {}, None
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] in ("steps", "t"):
                meta[parts[0]] = float(parts[1])
            elif parts[0] in ("sample", "wall", "colsum"):
                cur = parts[0]
                blocks[cur] = ([int(x) for x in parts[1:]], [])
            else:
                blocks[cur][1].extend(float(x) for x in parts)
    return meta, {k: np.array(v).reshape(shape) for k, (shape, v) in blocks.items()}


def test_ns_tube_250x125_first_20_steps():
    cfg, W, _ = P.viscous_shock_tube(250, 125, Re=1000.0, prandtl=0.73)
    worst = 0.0
    for n in range(20):
        W, _, _, err = check_step(cfg, W, "ns 250x125 step %d" % n)
        worst = max(worst, err)
    print("ns 250x125: 20 steps, worst per-step rel diff %.2e" % worst)


def test_ns_tube_1000x500_first_2_steps():
    cfg, W, _ = P.viscous_shock_tube(1000, 500, Re=1000.0, prandtl=0.73)
    for n in range(2):
        W, _, _, _ = check_step(cfg, W, "ns 1000x500 step %d" % n)


def test_ns_tube_250x125_full_run_against_stored_oracle():
    meta, ref = _read_golden(GOLDEN)
    cfg, W, t_end = P.viscous_shock_tube(250, 125, Re=1000.0, prandtl=0.73)
    Wg, tg, ng = hgks.run(cfg, W, t_end)
    assert ng == int(meta["steps"]) and tg == pytest.approx(meta["t"], abs=1e-14)
    got = {"sample": Wg[:, 2::5, 2::5], "wall": Wg[0, 0, :], "colsum": Wg.sum(axis=1)}
    errs = {k: rel_diff(got[k][None] if got[k].ndim == 1 else got[k], ref[k][None] if ref[k].ndim == 1 else ref[k])
            for k in ref}
    print("ns 250x125 to t = 1 (%d steps): rel diff %s" % (ng, errs))
    assert max(errs.values()) <= FINAL_TOL, errs


@pytest.mark.parametrize("n", [100, 200])
def test_vortex_to_t2_matches_oracle(n):
    cfg, W, t_end = P.vortex_2d(n)
    Wg, tg, ng = hgks.run(cfg, W, t_end)
    Wo, to, no, _ = oracle.run(cfg, W, t_end)
    assert ng == no and tg == to == t_end
    err = rel_diff(Wg, Wo)
    print("vortex %d^2 to t = 2: rel diff %.2e" % (n, err))
    assert err <= FINAL_TOL, err
