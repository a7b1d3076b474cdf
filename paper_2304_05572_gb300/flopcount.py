"""FP64 operation count of the closed-form gas-kinetic flux per Gauss point.

Compiles ``csrc/flux_flopcount.cpp`` (the flux functions of ``csrc/hgks_math.cuh``
on the host, with a counting stand-in for double) with g++ and runs it.  Each
arithmetic operation counts one, fma two, and division, square root, exp and
erfc one each (the device's instruction sequences for them are not counted).
This is the per-Gauss-point work the benchmark's roofline takes for the flux;
the value it uses is recorded there, so that a later change of the kernel does
not change the yardstick.

  python -m paper_2304_05572_gb300.flopcount
"""
from __future__ import annotations

import json
import os
import subprocess
import tempfile

_PKG = os.path.dirname(os.path.abspath(__file__))


_EXE = {}


def _exe() -> str:
    if "path" not in _EXE:
        d = tempfile.mkdtemp(prefix="hgks_flopcount_")
        exe = os.path.join(d, "flux_flopcount")
        subprocess.run(["g++", "-O1", "-std=gnu++17", "-ffp-contract=off", "-I", os.path.join(_PKG, "csrc"),
                        "-o", exe, os.path.join(_PKG, "csrc", "flux_flopcount.cpp")], check=True)
        _EXE["path"] = exe
    return _EXE["path"]


def count_flux() -> dict:
    """{variant: {"flop": ..., "add": ..., ...}} for the flux variants of the kernels."""
    out = subprocess.run([_exe()], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


def flux_values(dim, stage, Wl, Wlx, Wly, Wr, Wrx, Wry, dt, gamma=1.4, mu=0.0, c1=0.01, c2=1.0, prandtl=1.0,
                viscous=False, tau_zero=False):
    """The closed-form flux of the kernels at one Gauss point, evaluated on the host:
    (ok, o0, o1) with o0 = F(dt/2), o1 = (8 F(dt/2) - F(dt))/3 in the first stage and
    o0 = (4/3)(F(dt) - 2 F(dt/2)) in the second (Eq. (12) combined as in Eqs. (17)-(20))."""
    prfix = bool(viscous) and prandtl != 1.0
    w = []
    for v in (Wl, Wlx, Wly, Wr, Wrx, Wry):
        v = list(v) + [0.0] * (4 - len(v))
        w += [float(x) for x in v]
    args = [_exe(), "values", str(dim), str(stage), str(int(bool(viscous))), str(int(bool(tau_zero))),
            str(int(prfix))] + ["%.17g" % x for x in (gamma, mu, c1, c2, prandtl, dt)] + ["%.17g" % x for x in w]
    out = subprocess.run(args, check=True, capture_output=True, text=True).stdout.split()
    nv = dim + 2
    vals = [float(x) for x in out[1:]]
    return out[0] == "1", vals[:nv], vals[nv:2 * nv]


if __name__ == "__main__":
    print(json.dumps(count_flux(), indent=1))
