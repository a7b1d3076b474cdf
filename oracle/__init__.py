"""CPU oracle of the hybrid WENO-AO gas-kinetic scheme (arXiv 2304.05572).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain FP64 restatement of the
paper's method in C (``hgks_oracle.c``), loaded here through ctypes.  It is the
reference the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA library: the only thing both sides
consume is the seeded initial data of ``paper_2304_05572_gb300.problems``,
which holds no arithmetic of the method.

The library is built with ``-O2 -ffp-contract=off`` so that every ``a*b + c``
in the C source is a rounded multiply followed by a rounded add, unless the
source writes ``fma()``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hgks_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libhgks_oracle.so")
_lock = threading.Lock()
_lib = None

BC = {"periodic": 0, "extrap": 1, "reflect": 2, "symmetry": 3, "noslip": 4, "inflow": 5, "shock_wall": 6,
      "shock_track": 7}
RECON = {"hybrid": 0, "linear": 1, "wenoao": 2}
ZETA1 = {"A": 0, "B": 1, "C": 2, "D": 3}
NG = 4


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libhgks_oracle.so (gcc, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("viscous", ctypes.c_int),
        ("mu", ctypes.c_double), ("prandtl", ctypes.c_double),
        ("c1", ctypes.c_double), ("c2", ctypes.c_double),
        ("cfl", ctypes.c_double), ("fixed_dt", ctypes.c_double),
        ("tau_zero", ctypes.c_int),
        ("bc", ctypes.c_int * 4),
        ("recon_mode", ctypes.c_int),
        ("zeta1_mode", ctypes.c_int),
        ("gamma_hi", ctypes.c_double), ("gamma_lo", ctypes.c_double), ("eps", ctypes.c_double),
        ("threads", ctypes.c_int),
        ("bc_state", (ctypes.c_double * 4) * 4),
        ("shock_pre", ctypes.c_double * 4),
        ("shock_x0", ctypes.c_double), ("shock_cot", ctypes.c_double), ("shock_speed", ctypes.c_double),
    ]


_DP = ctypes.POINTER(ctypes.c_double)
_U8P = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.or_run.argtypes = [ctypes.POINTER(Config), _DP, _DP, ctypes.c_double, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int), _DP]
            L.or_step_flags.argtypes = [ctypes.POINTER(Config), _DP, ctypes.c_double, ctypes.c_double, _DP,
                                        ctypes.POINTER(_U8P), ctypes.POINTER(_DP), _DP]
            L.or_cfl_dt.argtypes = [ctypes.POINTER(Config), _DP]
            L.or_cfl_dt.restype = ctypes.c_double
            L.or_moments.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, _DP, _DP, _DP, _DP, _DP]
            L.or_dof_K.argtypes = [ctypes.c_int, ctypes.c_double]
            L.or_dof_K.restype = ctypes.c_double
            L.or_micro_slope.argtypes = [ctypes.c_int, ctypes.c_double, _DP, _DP, _DP]
            L.or_time_slope.argtypes = [ctypes.c_int, ctypes.c_double, _DP, _DP, _DP, _DP]
            L.or_slope_moment.argtypes = [ctypes.c_int, ctypes.c_double, _DP, _DP, ctypes.c_int, _DP]
            L.or_point_flux.argtypes = [ctypes.POINTER(Config), _DP, _DP, _DP, _DP, _DP, _DP,
                                        ctypes.c_double, _DP, _DP]
            L.or_indicator.argtypes = [_DP, ctypes.c_double]
            L.or_zeta1_scaled.argtypes = [ctypes.c_int, ctypes.c_double]
            L.or_zeta1_scaled.restype = ctypes.c_double
            L.or_linear_face.argtypes = [_DP, ctypes.c_double, ctypes.c_int, _DP, _DP]
            L.or_ao_betas.argtypes = [_DP, _DP]
            L.or_ao_face_scalar.argtypes = [_DP, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, _DP, _DP]
            L.or_gauss_scalar.argtypes = [_DP, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _DP, _DP]
            L.or_eigvec.argtypes = [ctypes.c_int, ctypes.c_double, _DP, ctypes.c_double, ctypes.c_double,
                                    _DP, _DP]
            L.or_weno_ao_face.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _DP, _DP, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, _DP, _DP]
            L.or_fill_ghosts.argtypes = [ctypes.POINTER(Config), _DP, ctypes.c_double, _DP]
            L.or_threads_used.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None and a.size < n:
        a = np.concatenate([a.ravel(), np.zeros(n - a.size)])
    return a


def make_config(cfg: dict, threads: int = 0) -> Config:
    """Build the C config from a problem dict (keys as in the struct)."""
    c = Config()
    c.dim = int(cfg["dim"]); c.nx = int(cfg["nx"]); c.ny = int(cfg.get("ny", 1))
    c.x0, c.x1 = float(cfg["x0"]), float(cfg["x1"])
    c.y0, c.y1 = float(cfg.get("y0", 0.0)), float(cfg.get("y1", 1.0))
    c.gamma = float(cfg.get("gamma", 1.4))
    c.viscous = int(cfg.get("viscous", 0))
    c.mu = float(cfg.get("mu", 0.0)); c.prandtl = float(cfg.get("prandtl", 1.0))
    c.c1 = float(cfg.get("c1", 0.01)); c.c2 = float(cfg.get("c2", 1.0))
    c.cfl = float(cfg.get("cfl", 0.5)); c.fixed_dt = float(cfg.get("fixed_dt", 0.0))
    c.tau_zero = int(cfg.get("tau_zero", 0))
    bc = cfg.get("bc", ["periodic"] * 4)
    for k in range(4):
        c.bc[k] = BC[bc[k]] if isinstance(bc[k], str) else int(bc[k])
    rm = cfg.get("recon_mode", "hybrid")
    c.recon_mode = RECON[rm] if isinstance(rm, str) else int(rm)
    zm = cfg.get("zeta1_mode", "B")
    c.zeta1_mode = ZETA1[zm] if isinstance(zm, str) else int(zm)
    c.gamma_hi = float(cfg.get("gamma_hi", 0.85)); c.gamma_lo = float(cfg.get("gamma_lo", 0.85))
    c.eps = float(cfg.get("eps", 1e-8))
    c.threads = int(threads)
    for k, st in enumerate(cfg.get("bc_state", [None] * 4)):
        if st is not None:
            for j, v in enumerate(st):
                c.bc_state[k][j] = float(v)
    for j, v in enumerate(cfg.get("shock_pre", [])):
        c.shock_pre[j] = float(v)
    c.shock_x0 = float(cfg.get("shock_x0", 0.0))
    c.shock_cot = float(cfg.get("shock_cot", 0.0))
    c.shock_speed = float(cfg.get("shock_speed", 0.0))
    return c


def _check(st: int, what: str):
    if st != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, st))


def run(cfg: dict, W: np.ndarray, t_end: float, max_steps: int = 1 << 30, t0: float = 0.0, threads: int = 0):
    """Advance the conservative state W[nv][ny][nx] to t_end. Returns (W, t, steps, last_dt)."""
    c = make_config(cfg, threads)
    Wc = np.ascontiguousarray(W, dtype=np.float64).copy()
    t = ctypes.c_double(t0)
    n = ctypes.c_int(0)
    ld = ctypes.c_double(0.0)
    st = lib().or_run(ctypes.byref(c), _dp(Wc), ctypes.byref(t), float(t_end), int(max_steps),
                      ctypes.byref(n), ctypes.byref(ld))
    _check(st, "run")
    return Wc, t.value, n.value, ld.value


def flag_shapes(cfg: dict):
    """Shapes of the per-stage flag arrays: {(dir, 'normal'|'tang'): shape}."""
    dim, nx, ny = int(cfg["dim"]), int(cfg["nx"]), int(cfg.get("ny", 1))
    out = {}
    if dim == 1:
        out[(0, "normal")] = (1, nx + 2)
        return out
    out[(0, "normal")] = (ny + 6, nx + 2)
    out[(0, "tang")] = (ny, nx + 1)
    out[(1, "normal")] = (nx + 6, ny + 2)
    out[(1, "tang")] = (nx, ny + 1)
    return out


def step_flags(cfg: dict, W: np.ndarray, dt: float = 0.0, threads: int = 0, margins: bool = False,
               wstar: np.ndarray = None, t0: float = 0.0):
    """One S2O4 step from time t0; returns (W_next, dt_used, flags) with flags[(stage, dir, kind)] arrays,
    and with margins=True also the relative decision margins in the same layout.  If wstar
    (same shape as W) is given it receives the first-stage state W*."""
    c = make_config(cfg, threads)
    Wc = np.ascontiguousarray(W, dtype=np.float64).copy()
    shapes = flag_shapes(cfg)
    bufs, mbufs = {}, {}
    ptrs = (_U8P * 8)()
    mptrs = (_DP * 8)()
    for s in range(2):
        for d in range(2):
            for ki, kind in enumerate(("normal", "tang")):
                if (d, kind) in shapes:
                    a = np.zeros(shapes[(d, kind)], dtype=np.uint8)
                    bufs[(s, d, kind)] = a
                    ptrs[(s * 2 + d) * 2 + ki] = a.ctypes.data_as(_U8P)
                    if margins:
                        mb = np.full(shapes[(d, kind)], np.inf)
                        mbufs[(s, d, kind)] = mb
                        mptrs[(s * 2 + d) * 2 + ki] = mb.ctypes.data_as(_DP)
    dtu = ctypes.c_double(0.0)
    st = lib().or_step_flags(ctypes.byref(c), _dp(Wc), float(t0), float(dt), ctypes.byref(dtu), ptrs,
                             mptrs if margins else None, _dp(wstar) if wstar is not None else None)
    _check(st, "step")
    if margins:
        return Wc, dtu.value, bufs, mbufs
    return Wc, dtu.value, bufs


def cfl_dt(cfg: dict, W: np.ndarray) -> float:
    c = make_config(cfg)
    Wc = np.ascontiguousarray(W, dtype=np.float64)
    return lib().or_cfl_dt(ctypes.byref(c), _dp(Wc))


def threads_used(requested: int = 0) -> int:
    return lib().or_threads_used(int(requested))


# ---- unit-level hooks ----

NMOM = 10


def moments(dim, K, U, V, lam):
    u, up, un, v = (np.zeros(NMOM) for _ in range(4))
    x = np.zeros(4)
    lib().or_moments(dim, K, U, V, lam, _dp(u), _dp(up), _dp(un), _dp(v), _dp(x))
    return u, up, un, v, x


def dof_K(dim, gamma=1.4):
    return lib().or_dof_K(dim, gamma)


def micro_slope(dim, gamma, W, dW):
    W, dW = _arr(W, 4), _arr(dW, 4)
    a = np.zeros(4)
    _check(lib().or_micro_slope(dim, gamma, _dp(W), _dp(dW), _dp(a)), "micro_slope")
    return a[: dim + 2]


def time_slope(dim, gamma, W, a1, a2=None):
    W, a1 = _arr(W, 4), _arr(a1, 4)
    a2 = _arr(a2 if a2 is not None else np.zeros(4), 4)
    A = np.zeros(4)
    _check(lib().or_time_slope(dim, gamma, _dp(W), _dp(a1), _dp(a2), _dp(A)), "time_slope")
    return A[: dim + 2]


def slope_moment(dim, gamma, W, a, half=0):
    W, a = _arr(W, 4), _arr(a, 4)
    out = np.zeros(4)
    lib().or_slope_moment(dim, gamma, _dp(W), _dp(a), int(half), _dp(out))
    return out[: dim + 2]


def point_flux(cfg, Wl, Wlx, Wr, Wrx, dt, Wly=None, Wry=None):
    c = make_config(cfg)
    z = np.zeros(4)
    args = [_arr(Wl, 4), _arr(Wlx, 4), _arr(Wly if Wly is not None else z, 4),
            _arr(Wr, 4), _arr(Wrx, 4), _arr(Wry if Wry is not None else z, 4)]
    Fd, Fh = np.zeros(4), np.zeros(4)
    st = lib().or_point_flux(ctypes.byref(c), *[_dp(a) for a in args], float(dt), _dp(Fd), _dp(Fh))
    _check(st, "point_flux")
    nv = int(cfg["dim"]) + 2
    return Fd[:nv], Fh[:nv]


def indicator(q5, Z1):
    return int(lib().or_indicator(_dp(_arr(q5)), float(Z1)))


def zeta1_scaled(mode, h):
    return lib().or_zeta1_scaled(ZETA1[mode] if isinstance(mode, str) else int(mode), float(h))


def linear_face(q5, h, side):
    v, d = ctypes.c_double(), ctypes.c_double()
    lib().or_linear_face(_dp(_arr(q5)), 1.0 / (12.0 * h), int(side), ctypes.byref(v), ctypes.byref(d))
    return v.value, d.value


def ao_betas(q5):
    b = np.zeros(4)
    lib().or_ao_betas(_dp(_arr(q5)), _dp(b))
    return b


def ao_face_scalar(q5, side, ghi=0.85, glo=0.85, eps=1e-8):
    v, d = ctypes.c_double(), ctypes.c_double()
    lib().or_ao_face_scalar(_dp(_arr(q5)), ghi, glo, eps, int(side), ctypes.byref(v), ctypes.byref(d))
    return v.value, d.value


def gauss_scalar(q5, use_ao=False, ghi=0.85, glo=0.85, eps=1e-8):
    v, d = np.zeros(2), np.zeros(2)
    lib().or_gauss_scalar(_dp(_arr(q5)), int(use_ao), ghi, glo, eps, _dp(v), _dp(d))
    return v, d


def eigvec(dim, gamma, Q, nx=1.0, ny=0.0):
    L, R = np.zeros(16), np.zeros(16)
    lib().or_eigvec(dim, gamma, _dp(_arr(Q, 4)), nx, ny, _dp(L), _dp(R))
    nv = dim + 2
    return L.reshape(4, 4)[:nv, :nv], R.reshape(4, 4)[:nv, :nv]


def weno_ao_face(dim, gamma, Qw, Qs, nx, ny, side, ghi=0.85, glo=0.85, eps=1e-8):
    Qw = np.asarray(Qw, dtype=np.float64)
    Q20 = np.zeros((5, 4)); Q20[:, : Qw.shape[1]] = Qw
    Q20 = np.ascontiguousarray(Q20)
    v, d = np.zeros(4), np.zeros(4)
    lib().or_weno_ao_face(dim, gamma, ghi, glo, eps, _dp(Q20), _dp(_arr(Qs, 4)), nx, ny, int(side), _dp(v), _dp(d))
    return v[: dim + 2], d[: dim + 2]


def fill_ghosts(cfg, W, t=0.0):
    c = make_config(cfg)
    dim, nx, ny = int(cfg["dim"]), int(cfg["nx"]), int(cfg.get("ny", 1))
    nv = dim + 2
    NY = ny + 2 * NG if dim == 2 else 1
    out = np.zeros((nv, NY, nx + 2 * NG))
    Wc = np.ascontiguousarray(W, dtype=np.float64)
    _check(lib().or_fill_ghosts(ctypes.byref(c), _dp(Wc), float(t), _dp(out)), "fill_ghosts")
    return out
