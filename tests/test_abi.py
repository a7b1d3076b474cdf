"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
entry point include/hgks.h declares, the ctypes struct layouts agree with C, and
configuration validation rejects bad input before any device work."""
import ctypes
import os
import re

import pytest

from paper_2304_05572_gb300 import _build, hgks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    _build.build()
    return hgks.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "hgks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hgks_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(hgks.EXPORTED) == names


def test_config_default_layout(L):
    c = hgks.hgks_config()
    assert L.hgks_config_default(ctypes.byref(c)) == 0
    assert (c.dim, c.nx, c.ny) == (2, 64, 64)
    assert c.gamma == 1.4 and c.c1 == 0.01 and c.c2 == 1.0 and c.cfl == 0.5
    assert c.gamma_hi == 0.85 and c.gamma_lo == 0.85 and c.eps == 1e-8
    assert list(c.bc) == [0, 0, 0, 0] and c.recon_mode == 0 and c.zeta1_mode == 1
    assert L.hgks_config_default(None) == hgks.HGKS_EINVAL


@pytest.mark.parametrize("bad,msg", [
    (dict(dim=3), "dim"),
    (dict(nx=3), "nx"),
    (dict(ny=2), "ny"),
    (dict(x1=0.0), "domain"),
    (dict(gamma=1.0), "gamma"),
    (dict(cfl=0.0, fixed_dt=0.0), "cfl"),
    (dict(viscous=1, mu=0.0), "mu"),
    (dict(viscous=1, mu=1e-3, prandtl=0.0), "Prandtl"),
    (dict(bc=["periodic", "periodic", "extrap", "shock_wall"]), "SHOCK_WALL"),
    (dict(bc=["shock_track", "extrap", "extrap", "extrap"]), "SHOCK_TRACK"),
    (dict(bc=["inflow", "extrap", "extrap", "extrap"]), "prescribed"),
    (dict(bc=["periodic", "extrap", "extrap", "extrap"]), "periodic"),
    (dict(recon_mode=7), "recon"),
    (dict(gamma_hi=1.0), "gamma_hi"),
    (dict(nx=20000, ny=20000), "too large"),
])
def test_invalid_config_rejected_before_device_work(L, bad, msg):
    cfg = dict(dim=2, nx=16, ny=16, x0=0.0, x1=1.0, y0=0.0, y1=1.0)
    cfg.update(bad)
    with pytest.raises(hgks.HGKSError) as e:
        hgks.Solver(cfg)
    assert e.value.code == hgks.HGKS_EINVAL
    assert msg in str(e.value)


def test_footprint_scales_with_grid(L):
    a = hgks.hgks_footprint_bytes(dict(dim=2, nx=256, ny=256))
    b = hgks.hgks_footprint_bytes(dict(dim=2, nx=512, ny=512))
    assert 3.5 < b / a < 4.5
    assert hgks.hgks_footprint_bytes(dict(dim=2, nx=2, ny=256)) == 0    # invalid -> 0
    one = hgks.hgks_footprint_bytes(dict(dim=1, nx=200))
    assert 0 < one < a


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(hgks, "LIB_PATH", "/nonexistent/libhgks.so")
    monkeypatch.setattr(hgks, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        hgks.lib()


def test_normal_build_reports_no_bounds_checks(L):
    """hgks_debug_bounds needs no device in the normal build: it reports that the checks are
    not compiled in (the debug build is _lib/libhgks_debug.so)."""
    assert hgks.hgks_debug_bounds() == (False, 0, 0)
