"""Operation counts of the oracle (TEST INFRASTRUCTURE ONLY, like the oracle).

``oracle/opcount.cpp`` compiles ``hgks_oracle.c`` unchanged as C++ with every
double replaced by a counting stand-in (``opcount.hpp``): add / sub, mul, div,
sqrt, exp and erfc count one each, fma two.  This module builds that library
and counts the FP64 work of an oracle run or of one Gauss-point flux.

The oracle evaluates the reconstruction, the indicator, the update and the time
step from the paper's formulas as printed; its flux integrates every velocity
moment literally (polynomial products) and solves the moment systems as dense
4 x 4 systems, which takes several times the operations of the closed forms.

  python -m oracle.opcount        # the counts of one 1024^2 four-quadrant step
"""
from __future__ import annotations

import ctypes
import json
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libhgks_oracle_opcount.so")
_SRCS = [os.path.join(_HERE, f) for f in ("opcount.cpp", "opcount.hpp", "hgks_oracle.c")]
KINDS = ("add", "mul", "fma", "div", "sqrt", "exp", "erfc")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=gnu++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, os.path.join(_HERE, "opcount.cpp"), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    from . import Config, _DP
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.or_run.argtypes = [ctypes.POINTER(Config), _DP, _DP, ctypes.c_double, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int), _DP]
            L.or_point_flux.argtypes = [ctypes.POINTER(Config), _DP, _DP, _DP, _DP, _DP, _DP,
                                        ctypes.c_double, _DP, _DP]
            L.or_linear_face.argtypes = [_DP, ctypes.c_double, ctypes.c_int, _DP, _DP]
            L.or_indicator.argtypes = [_DP, ctypes.c_double]
            L.opc_read.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
            L.or_gauss_scalar.argtypes = [_DP, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          _DP, _DP]
            _lib = L
    return _lib


def _read() -> dict:
    buf = (ctypes.c_ulonglong * 8)()
    lib().opc_read(buf)
    return dict(zip(KINDS, (int(x) for x in buf[:7])))


def flop(counts: dict) -> int:
    """FP64 operations of a count: every kind once, fma twice."""
    return sum(counts[k] for k in KINDS) + counts["fma"]


def count_run(cfg: dict, W: np.ndarray, steps: int = 1, threads: int = 0) -> dict:
    """Operations of `steps` oracle S2O4 steps of W (counts by kind)."""
    from . import make_config, _dp
    c = make_config(cfg, threads)
    Wc = np.ascontiguousarray(W, dtype=np.float64).copy()
    t, n, ld = ctypes.c_double(0.0), ctypes.c_int(0), ctypes.c_double(0.0)
    lib().opc_reset()
    st = lib().or_run(ctypes.byref(c), _dp(Wc), ctypes.byref(t), 1e300, int(steps), ctypes.byref(n), ctypes.byref(ld))
    if st != 0 or n.value != steps:
        raise RuntimeError("counting run failed (status %d, %d steps)" % (st, n.value))
    return _read()


def count_point_flux(cfg: dict, Wl, Wlx, Wly, Wr, Wrx, Wry, dt: float) -> dict:
    """Operations of one oracle Gauss-point flux (both time integrals of Eq. (12))."""
    from . import make_config, _dp, _arr
    c = make_config(cfg)
    args = [_arr(a, 4) for a in (Wl, Wlx, Wly, Wr, Wrx, Wry)]
    Fd, Fh = np.zeros(4), np.zeros(4)
    lib().opc_reset()
    st = lib().or_point_flux(ctypes.byref(c), *[_dp(a) for a in args], float(dt), _dp(Fd), _dp(Fh))
    if st != 0:
        raise RuntimeError("counting flux failed (status %d)" % st)
    return _read()


def count_linear_face(q5, h: float, side: int) -> dict:
    from . import _dp, _arr
    v, d = ctypes.c_double(), ctypes.c_double()
    lib().opc_reset()
    lib().or_linear_face(_dp(_arr(q5)), 1.0 / (12.0 * h), int(side), ctypes.byref(v), ctypes.byref(d))
    return _read()


def count_gauss_scalar(q5, use_ao: bool = False) -> dict:
    """Operations of one oracle Gauss-point reconstruction of a 5-cell window (values and
    cell-unit derivatives at both Gauss points; linear, or WENO-AO with use_ao)."""
    from . import _dp, _arr
    v, d = np.zeros(2), np.zeros(2)
    lib().opc_reset()
    lib().or_gauss_scalar(_dp(_arr(q5)), int(use_ao), 0.85, 0.85, 1e-8, _dp(v), _dp(d))
    return _read()


def step_table(n: int = 1024, threads: int = 0) -> dict:
    """Per cell-stage operation counts of one oracle step of the n^2 four-quadrant Riemann
    problem in the three reconstruction modes, and of one Gauss-point flux; the flux share
    of each step is counted separately (its count does not depend on the data), so that the
    rest -- indicator, reconstruction, update, time step -- can be combined with another
    flux count."""
    sys.path.insert(0, os.path.dirname(_HERE))
    from . import step_flags
    from paper_2304_05572_gb300 import problems as P
    cfg, W, _ = P.riemann4_2d(n)
    cell_stages = 2 * n * n
    gp = 2 * 2 * 2 * n * (n + 1)                      # 2 stages x 2 sweeps x 2 Gauss points x interfaces
    fl = count_point_flux(cfg, [1.0, 0.1, 0.2, 2.5], [0.1, 0.05, -0.02, 0.3], [-0.05, 0.01, 0.03, -0.1],
                          [0.8, -0.1, 0.05, 2.0], [0.1, 0.05, -0.02, 0.3], [-0.05, 0.01, 0.03, -0.1], 1e-3)
    out = {"problem": "four-quadrant 2D Riemann problem, %d^2, one S2O4 step from t = 0" % n,
           "gauss_points_per_cell_stage": gp / cell_stages, "oracle_flux_flop_per_gp": flop(fl),
           "oracle_flux_counts_per_gp": fl}
    for mode in ("linear", "hybrid", "wenoao"):
        c = count_run(dict(cfg, recon_mode=mode), W, 1, threads)
        tot = flop(c)
        out[mode] = {"flop_per_cell_stage": tot / cell_stages,
                     "non_flux_flop_per_cell_stage": (tot - gp * flop(fl)) / cell_stages,
                     "counts_per_cell_stage": {k: v / cell_stages for k, v in c.items()}}
    # troubled fraction of the hybrid step (all passes), as the library reports it
    _, _, flags = step_flags(cfg, W, threads=threads)
    tr = ex = 0
    for (stage, d, kind), f in flags.items():
        if kind == "normal":
            f = f[3:-3, 1:-1]
            tr += int(f.sum()); ex += f.size
        else:
            tr += sum(bin(int(v)).count("1") for v in f.ravel()); ex += 4 * f.size
    out["hybrid"]["troubled_fraction"] = tr / ex
    return out


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 1024
    print(json.dumps(step_table(n), indent=1))
