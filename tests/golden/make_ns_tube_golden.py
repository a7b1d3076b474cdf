"""Writes ns_tube_250x125_t1.txt: the oracle's state at t = 1 of the viscous shock tube
(Sec. 3.6 set-up: [0,1] x [0,0.5], (120, 0, 120/gamma) | (1.2, 0, 1.2/gamma) at x = 0.5,
no-slip adiabatic walls, symmetry on top, CFL 0.3) at Re = 1000, Pr = 0.73 on 250 x 125
cells, for the GPU full-run parity test.  Calls only the oracle.

The file holds, after '#' header lines (steps, final time), three blocks of whitespace-
separated numbers written with 17 significant digits:
  * 'sample': every component at cells i = 2, 7, ..., 247 and j = 2, 7, ..., 122
    ([4][25][50], C order);
  * 'wall': the density of the bottom row j = 0, all 250 cells;
  * 'colsum': the sums over j of every component, [4][250].

  python tests/golden/make_ns_tube_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2304_05572_gb300 import problems as P  # noqa: E402

NX, NY, RE, PR = 250, 125, 1000.0, 0.73
OUT = os.path.join(HERE, "ns_tube_250x125_t1.txt")
SAMPLE = (slice(None), slice(2, NY, 5), slice(2, NX, 5))


def main():
    cfg, W, t_end = P.viscous_shock_tube(NX, NY, Re=RE, prandtl=PR)
    Wo, t, steps, _ = oracle.run(cfg, W, t_end)
    with open(OUT, "w") as f:
        f.write("# oracle state of the viscous shock tube (Sec. 3.6 set-up) at Re = %g, Pr = %g, %d x %d cells\n"
                % (RE, PR, NX, NY))
        f.write("# written by tests/golden/make_ns_tube_golden.py (oracle only)\n")
        f.write("steps %d\n" % steps)
        f.write("t %.17g\n" % t)
        for name, arr in (("sample", Wo[SAMPLE]), ("wall", Wo[0, 0, :]), ("colsum", Wo.sum(axis=1))):
            f.write("%s %s\n" % (name, " ".join(str(d) for d in arr.shape)))
            f.write("\n".join(" ".join("%.17g" % v for v in row) for row in np.reshape(arr, (-1, arr.shape[-1]))))
            f.write("\n")
    print(OUT, steps, t)


if __name__ == "__main__":
    main()
