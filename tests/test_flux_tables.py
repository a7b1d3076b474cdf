"""The committed erfcx table of the flux kernel (csrc/erfcx_table.inc) against an
independent evaluation of exp(y^2) erfc(y) in 30-digit arithmetic (mpmath)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "paper_2304_05572_gb300", "csrc", "erfcx_table.inc")


def _table():
    txt = open(INC).read()
    n = int(re.search(r"HGKS_ERFCX_INTERVALS (\d+)", txt).group(1))
    deg = int(re.search(r"HGKS_ERFCX_DEGREE (\d+)", txt).group(1))
    body = txt.split("HGKS_ERFCX_TABLE {")[1]
    nums = [float(x) for x in re.findall(r"[-+]?\d\.\d+(?:e[-+]\d+)?", body)]
    assert len(nums) == n * (deg + 1)
    return np.array(nums).reshape(n, deg + 1)


def test_erfcx_table_matches_high_precision_erfc():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    a = _table()
    assert a.shape == (32, 12)
    ys = np.concatenate([np.linspace(0.0, 8.0, 3001)[:-1], np.arange(1, 32) / 4.0 - 1e-15, np.arange(1, 32) / 4.0])
    worst = 0.0
    for y in ys:
        # the kernel's interval choice: the nearest centre (k + 1/2)/4
        k = min(31, max(0, int(np.rint(4.0 * y - 0.5))))
        t = y - (k + 0.5) / 4.0
        assert abs(t) <= 0.125 + 1e-15
        p = 0.0
        for c in a[k][::-1]:
            p = p * t + c
        ref = mp.exp(mp.mpf(y) ** 2) * mp.erfc(mp.mpf(y))
        worst = max(worst, float(abs((p - ref) / ref)))
    assert worst <= 3e-16, worst
