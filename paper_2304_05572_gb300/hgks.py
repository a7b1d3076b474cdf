"""Python binding of the C ABI in include/hgks.h (argument marshalling only).

Every step of the scheme runs in the CUDA library ``_lib/libhgks.so``; this
module only converts arguments.  There is no CPU fallback: if the library is
missing it raises.  PyTorch, when used, only supplies device memory
(``tensor.data_ptr()``) and streams (``torch.cuda.Stream.cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# HGKS_DEBUG_BOUNDS=1 in the environment loads the debug build (every kernel access range-checked)
LIB_PATH = os.path.join(_PKG, "_lib", "libhgks_debug.so" if os.environ.get("HGKS_DEBUG_BOUNDS") == "1"
                        else "libhgks.so")

HGKS_OK = 0
HGKS_EINVAL = -1
HGKS_ENOMEM = -2
HGKS_ENONPHYSICAL = -3
HGKS_ETIMEOUT = -4
HGKS_ECUDA = -5
ERR_NAMES = {-1: "HGKS_EINVAL", -2: "HGKS_ENOMEM", -3: "HGKS_ENONPHYSICAL", -4: "HGKS_ETIMEOUT", -5: "HGKS_ECUDA"}

BC = {"periodic": 0, "extrap": 1, "reflect": 2, "symmetry": 3, "noslip": 4, "inflow": 5, "shock_wall": 6,
      "shock_track": 7}
RECON = {"hybrid": 0, "linear": 1, "wenoao": 2}
ZETA1 = {"A": 0, "B": 1, "C": 2}

EXPORTED = [
    "hgks_config_default", "hgks_create_solver", "hgks_destroy_solver", "hgks_set_state", "hgks_step",
    "hgks_get_state", "hgks_get_time", "hgks_get_stats", "hgks_set_flag_capture", "hgks_flags_size",
    "hgks_get_flags", "hgks_set_timing", "hgks_get_timing", "hgks_last_error", "hgks_footprint_bytes",
    "hgks_batch_create", "hgks_batch_update", "hgks_batch_step", "hgks_batch_sync", "hgks_batch_status",
    "hgks_batch_info",
    "hgks_batch_last_error",
    "hgks_batch_destroy", "hgks_debug_bounds", "hgks_probe_fp64", "hgks_check_reciprocal", "hgks_step_noalloc",
]
HGKS_BATCH_GRAPH = 1
HGKS_BATCH_AUTOTUNE = 2


class hgks_config(ctypes.Structure):
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
        ("recon_mode", ctypes.c_int), ("zeta1_mode", ctypes.c_int),
        ("gamma_hi", ctypes.c_double), ("gamma_lo", ctypes.c_double), ("eps", ctypes.c_double),
        ("bc_state", (ctypes.c_double * 4) * 4),
        ("shock_pre", ctypes.c_double * 4),
        ("shock_x0", ctypes.c_double), ("shock_cot", ctypes.c_double), ("shock_speed", ctypes.c_double),
    ]


class hgks_stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_longlong), ("t", ctypes.c_double), ("last_dt", ctypes.c_double),
        ("status", ctypes.c_int), ("pad_", ctypes.c_int),
        ("troubled", ctypes.c_longlong * 8), ("examined", ctypes.c_longlong * 8),
        ("launches", ctypes.c_longlong),
    ]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libhgks.so (built by __graft_entry__.build() or _build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        L.hgks_config_default.argtypes = [ctypes.POINTER(hgks_config)]
        L.hgks_create_solver.argtypes = [ctypes.POINTER(hgks_config), vp, ctypes.POINTER(vp)]
        L.hgks_destroy_solver.argtypes = [vp]
        L.hgks_destroy_solver.restype = None
        L.hgks_set_state.argtypes = [vp, vp, ctypes.c_int, ctypes.c_double]
        L.hgks_step.argtypes = [vp, ctypes.c_double, ctypes.c_int, ip]
        L.hgks_get_state.argtypes = [vp, vp, ctypes.c_int]
        L.hgks_get_time.argtypes = [vp, dp]
        L.hgks_get_stats.argtypes = [vp, ctypes.POINTER(hgks_stats)]
        L.hgks_set_flag_capture.argtypes = [vp, ctypes.c_int]
        L.hgks_flags_size.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.hgks_flags_size.restype = ctypes.c_size_t
        L.hgks_get_flags.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
        L.hgks_set_timing.argtypes = [vp, ctypes.c_int]
        L.hgks_get_timing.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), dp,
                                      ctypes.POINTER(ctypes.c_longlong)]
        L.hgks_last_error.argtypes = [vp]
        L.hgks_last_error.restype = ctypes.c_char_p
        L.hgks_footprint_bytes.argtypes = [ctypes.POINTER(hgks_config)]
        L.hgks_footprint_bytes.restype = ctypes.c_size_t
        L.hgks_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.hgks_batch_update.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int]
        L.hgks_batch_step.argtypes = [vp, dp, ctypes.c_int, ctypes.c_int]
        L.hgks_batch_sync.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.hgks_batch_status.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]
        L.hgks_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
        L.hgks_batch_last_error.argtypes = [vp]
        L.hgks_batch_last_error.restype = ctypes.c_char_p
        L.hgks_batch_destroy.argtypes = [vp]
        L.hgks_batch_destroy.restype = None
        L.hgks_probe_fp64.argtypes = [vp, dp, dp, ip]
        L.hgks_check_reciprocal.argtypes = [ctypes.c_longlong, ctypes.POINTER(ctypes.c_ulonglong)]
        L.hgks_debug_bounds.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)]
        L.hgks_step_noalloc.argtypes = [ctypes.POINTER(hgks_config), vp, vp, vp, vp]
        _lib = L
        return L


class HGKSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERR_NAMES.get(code, "?"), code, msg))
        self.code = code


def make_config(cfg: dict) -> hgks_config:
    """hgks_config from a problem dict (keys as in the struct; names accepted for enums)."""
    c = hgks_config()
    lib().hgks_config_default(ctypes.byref(c))
    for key in ("dim", "nx", "ny", "viscous", "tau_zero"):
        if key in cfg:
            setattr(c, key, int(cfg[key]))
    for key in ("x0", "x1", "y0", "y1", "gamma", "mu", "prandtl", "c1", "c2", "cfl", "fixed_dt",
                "gamma_hi", "gamma_lo", "eps"):
        if key in cfg:
            setattr(c, key, float(cfg[key]))
    if int(cfg.get("dim", 2)) == 1:
        c.ny = 1
    bc = cfg.get("bc")
    if bc is not None:
        for k in range(4):
            c.bc[k] = BC[bc[k]] if isinstance(bc[k], str) else int(bc[k])
    rm = cfg.get("recon_mode")
    if rm is not None:
        c.recon_mode = RECON[rm] if isinstance(rm, str) else int(rm)
    zm = cfg.get("zeta1_mode")
    if zm is not None:
        c.zeta1_mode = ZETA1[zm] if isinstance(zm, str) else int(zm)
    for k, st in enumerate(cfg.get("bc_state", [None] * 4)):
        if st is not None:
            for j, v in enumerate(st):
                c.bc_state[k][j] = float(v)
    for j, v in enumerate(cfg.get("shock_pre", [])):
        c.shock_pre[j] = float(v)
    for key in ("shock_x0", "shock_cot", "shock_speed"):
        if key in cfg:
            setattr(c, key, float(cfg[key]))
    return c


def hgks_footprint_bytes(cfg: dict) -> int:
    c = make_config(cfg)
    return int(lib().hgks_footprint_bytes(ctypes.byref(c)))


def _ptr(a):
    """(pointer, on_device) for a numpy array or a CUDA torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("state arrays must be C-contiguous float64")
        return ctypes.c_void_p(a.ctypes.data), 0
    # torch tensor (device or host)
    if not a.is_contiguous() or str(a.dtype) != "torch.float64":
        raise ValueError("state tensors must be contiguous float64")
    return ctypes.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0)


class Solver:
    """One solver object (hgks_create_solver .. hgks_destroy_solver)."""

    def __init__(self, cfg: dict, stream=None):
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        self.dim = self._c.dim
        self.nx, self.ny = self._c.nx, self._c.ny
        self.nv = self.dim + 2
        h = ctypes.c_void_p()
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        rc = lib().hgks_create_solver(ctypes.byref(self._c), ctypes.c_void_p(st or 0), ctypes.byref(h))
        if rc != HGKS_OK:
            raise HGKSError(rc, lib().hgks_last_error(None).decode())
        self._h = h

    # -- C names -----------------------------------------------------------
    def _check(self, rc):
        if rc != HGKS_OK:
            raise HGKSError(rc, lib().hgks_last_error(self._h).decode())

    def hgks_set_state(self, W, t0: float = 0.0):
        p, dev = _ptr(W)
        self._check(lib().hgks_set_state(self._h, p, dev, float(t0)))

    def hgks_step(self, t_end: float, max_steps: int, wait: bool = True) -> int:
        n = ctypes.c_int(0)
        self._check(lib().hgks_step(self._h, float(t_end), int(max_steps), ctypes.byref(n) if wait else None))
        return n.value if wait else -1

    def hgks_get_state(self, out=None):
        if out is None:
            out = np.empty((self.nv, self.ny, self.nx), dtype=np.float64)
        p, dev = _ptr(out)
        self._check(lib().hgks_get_state(self._h, p, dev))
        return out

    def hgks_get_time(self) -> float:
        t = ctypes.c_double()
        self._check(lib().hgks_get_time(self._h, ctypes.byref(t)))
        return t.value

    def hgks_get_stats(self) -> dict:
        s = hgks_stats()
        self._check(lib().hgks_get_stats(self._h, ctypes.byref(s)))
        tr = np.array(s.troubled[:], dtype=np.int64).reshape(2, 2, 2)
        ex = np.array(s.examined[:], dtype=np.int64).reshape(2, 2, 2)
        return {"steps": s.steps, "t": s.t, "last_dt": s.last_dt, "status": s.status, "troubled": tr, "examined": ex,
                "launches": s.launches}

    def hgks_set_flag_capture(self, enable: bool = True):
        self._check(lib().hgks_set_flag_capture(self._h, int(bool(enable))))

    def flag_shape(self, sweep: int, kind: int):
        if self.dim == 1:
            return (1, self.nx + 2) if kind == 0 else None
        nn, nt = (self.nx, self.ny) if sweep == 0 else (self.ny, self.nx)
        return (nt + 6, nn + 2) if kind == 0 else (nt, nn + 1)

    def hgks_get_flags(self, stage: int, sweep: int, kind: int):
        n = lib().hgks_flags_size(self._h, sweep, kind)
        out = np.zeros(n, dtype=np.uint8)
        self._check(lib().hgks_get_flags(self._h, stage, sweep, kind, ctypes.c_void_p(out.ctypes.data)))
        return out.reshape(self.flag_shape(sweep, kind))

    def hgks_set_timing(self, enable: bool = True):
        self._check(lib().hgks_set_timing(self._h, int(bool(enable))))

    def hgks_get_timing(self) -> dict:
        cap = 32
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        calls = (ctypes.c_longlong * cap)()
        n = lib().hgks_get_timing(self._h, cap, names, ms, calls)
        if n < 0:
            self._check(n)
        return {names[i].decode(): (ms[i], calls[i]) for i in range(n)}

    def hgks_destroy_solver(self):
        if getattr(self, "_h", None):
            lib().hgks_destroy_solver(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def __del__(self):
        try:
            self.hgks_destroy_solver()
        except Exception:
            pass


class Batch:
    """A group of solvers advanced by shared batched launches (hgks_batch_*)."""

    def __init__(self, solvers, stream=None):
        self.solvers = list(solvers)
        n = len(self.solvers)
        arr = (ctypes.c_void_p * n)(*[sv.handle for sv in self.solvers])
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        h = ctypes.c_void_p()
        rc = lib().hgks_batch_create(arr, n, ctypes.c_void_p(st or 0), ctypes.byref(h))
        if rc != HGKS_OK:
            raise HGKSError(rc, lib().hgks_last_error(None).decode())
        self._h = h

    def _check(self, rc):
        if rc != HGKS_OK:
            raise HGKSError(rc, lib().hgks_batch_last_error(self._h).decode())

    def hgks_batch_update(self, solvers):
        """Replace the batch's solvers (hgks_batch_update); the same stream and block sizes."""
        new = list(solvers)
        arr = (ctypes.c_void_p * len(new))(*[sv.handle for sv in new])
        self._check(lib().hgks_batch_update(self._h, arr, len(new)))
        self.solvers = new

    def hgks_batch_step(self, t_end=None, nsteps=1, graph=True, autotune=False):
        te = None
        if t_end is not None:
            te = (ctypes.c_double * len(self.solvers))(*[float(t) for t in t_end])
        flags = (HGKS_BATCH_GRAPH if graph else 0) | (HGKS_BATCH_AUTOTUNE if autotune else 0)
        self._check(lib().hgks_batch_step(self._h, te, int(nsteps), flags))

    def hgks_batch_sync(self):
        """Wait for the batch; returns (active, failed) solver counts."""
        n, f = ctypes.c_int(0), ctypes.c_int(0)
        self._check(lib().hgks_batch_sync(self._h, ctypes.byref(n), ctypes.byref(f)))
        return n.value, f.value

    def hgks_batch_status(self):
        """(t, status, steps) arrays of the solvers as of the last hgks_batch_sync."""
        n = len(self.solvers)
        t = (ctypes.c_double * n)()
        st = (ctypes.c_int * n)()
        steps = (ctypes.c_longlong * n)()
        self._check(lib().hgks_batch_status(self._h, t, st, steps))
        return list(t), list(st), list(steps)

    def hgks_batch_info(self):
        tpb = (ctypes.c_int * 64)()
        steps = ctypes.c_longlong(0)
        n = lib().hgks_batch_info(self._h, tpb, 64, ctypes.byref(steps))
        return list(tpb[:n]), steps.value

    def hgks_batch_destroy(self):
        if getattr(self, "_h", None):
            lib().hgks_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.hgks_batch_destroy()
        except Exception:
            pass


def run(cfg: dict, W, t_end: float, max_steps: int = 1 << 30, t0: float = 0.0):
    """Convenience: create a solver, advance W to t_end, return (W, t, steps)."""
    s = Solver(cfg)
    try:
        s.hgks_set_state(np.ascontiguousarray(W, dtype=np.float64), t0)
        n = s.hgks_step(t_end, max_steps)
        return s.hgks_get_state(), s.hgks_get_time(), n
    finally:
        s.hgks_destroy_solver()


def hgks_debug_bounds():
    """(checked, count, first_address): whether this library checks every kernel access
    (the debug build), how many out-of-range accesses it skipped, and the first address."""
    n, a = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
    rc = lib().hgks_debug_bounds(ctypes.byref(n), ctypes.byref(a))
    if rc < 0:
        raise HGKSError(rc, lib().hgks_last_error(None).decode())
    return bool(rc), n.value, a.value


def hgks_check_reciprocal(n: int = 1 << 24):
    """(1/x, 1/sqrt(x)): largest distances in ulps of the flux's Newton-refined reciprocal and
    reciprocal square root from their IEEE counterparts over n arguments (see include/hgks.h)."""
    u = (ctypes.c_ulonglong * 2)()
    rc = lib().hgks_check_reciprocal(int(n), u)
    if rc != HGKS_OK:
        raise HGKSError(rc, lib().hgks_last_error(None).decode())
    return u[0], u[1]


def hgks_probe_fp64(stream=None):
    """FP64 FMA rate of the current device: (TFLOP/s, ms of the probe, SM count)."""
    tf, ms, sms = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_int(0)
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    rc = lib().hgks_probe_fp64(ctypes.c_void_p(st or 0), ctypes.byref(tf), ctypes.byref(ms), ctypes.byref(sms))
    if rc != HGKS_OK:
        raise HGKSError(rc, lib().hgks_last_error(None).decode())
    return tf.value, ms.value, sms.value


def hgks_step_noalloc(cfg: dict, W_in, W_out, stream=None, status=None):
    """One S2O4 step W_in -> W_out (CUDA float64 tensors [nv][ny][nx] on the current device)
    without any device allocation: the intermediates live in the library's static scratch
    (see include/hgks.h).  status: None, or a one-element int32 tensor (device or host) /
    numpy array that receives 0 or HGKS_ENONPHYSICAL when the stream reaches the end of
    the step."""
    c = make_config(cfg)
    pin, din = _ptr(W_in)
    pout, dout = _ptr(W_out)
    if not (din and dout):
        raise ValueError("hgks_step_noalloc takes device tensors")
    import torch
    dev = torch.cuda.current_device()
    if W_in.device.index != dev or W_out.device.index != dev:
        raise ValueError("W_in and W_out must live on the current CUDA device (%d)" % dev)
    n = (c.dim + 2) * c.nx * c.ny
    if W_in.numel() != n or W_out.numel() != n:
        raise ValueError("W_in and W_out must hold (dim+2)*nx*ny = %d values (got %d and %d)"
                         % (n, W_in.numel(), W_out.numel()))
    ps = None
    if status is not None:
        if isinstance(status, np.ndarray):
            if status.dtype != np.int32 or status.size != 1 or not status.flags["C_CONTIGUOUS"]:
                raise ValueError("status must be one contiguous int32")
            ps = ctypes.c_void_p(status.ctypes.data)
        else:
            if str(status.dtype) != "torch.int32" or status.numel() != 1 or not status.is_contiguous():
                raise ValueError("status must be one contiguous int32")
            if status.is_cuda and status.device.index != dev:
                raise ValueError("status must live on the current CUDA device (%d)" % dev)
            ps = ctypes.c_void_p(status.data_ptr())
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    rc = lib().hgks_step_noalloc(ctypes.byref(c), pin, pout, ps, ctypes.c_void_p(st or 0))
    if rc != HGKS_OK:
        raise HGKSError(rc, lib().hgks_last_error(None).decode())
