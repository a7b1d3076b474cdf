"""Seeded, synthetic initial data for the test problems of arXiv 2304.05572.

This module is the single source of inputs shared by the CUDA library's tests
and benchmark and by the CPU oracle.  It holds problem definitions only (domain,
boundary conditions, initial primitive fields and their exact cell averages),
none of the scheme's arithmetic.

Every function returns ``(cfg, W, t_end)``: ``cfg`` is a plain dict with the
solver configuration (keys mirror ``hgks_config``), ``W`` the conservative cell
averages laid out ``[nv][ny][nx]`` (C order, FP64; nv = 3 in 1D, 4 in 2D) and
``t_end`` the end time the paper (or the benchmark configuration) uses.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4


def base_config(dim, nx, ny, x0, x1, y0=0.0, y1=1.0, **kw):
    cfg = dict(dim=dim, nx=nx, ny=ny if dim == 2 else 1, x0=x0, x1=x1, y0=y0, y1=y1,
               gamma=GAMMA, viscous=0, mu=0.0, prandtl=1.0, c1=0.01, c2=1.0, cfl=0.5,
               fixed_dt=0.0, tau_zero=0, bc=["periodic"] * 4, recon_mode="hybrid",
               zeta1_mode="B", gamma_hi=0.85, gamma_lo=0.85, eps=1e-8)
    cfg.update(kw)
    return cfg


def conservative(rho, u, v, p, gamma=GAMMA, dim=2):
    """Primitive (rho, u, v, p) -> conservative stack (pointwise)."""
    rho, u, v, p = (np.asarray(a, dtype=np.float64) for a in (rho, u, v, p))
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    if dim == 1:
        return np.stack([rho, rho * u, E])
    return np.stack([rho, rho * u, rho * v, E])


def _edges(lo, hi, n):
    return lo + (hi - lo) * np.arange(n + 1) / n


# ---------------------------------------------------------------- 1D problems

def sine_1d(n, recon_mode="hybrid", zeta1_mode="B"):
    """Sec. 3.1: rho = 1 + 0.2 sin(pi x), U = 1, p = 1 on [0, 2], periodic,
    dt = 0.2 dx fixed, tau = 0, t = 2.  Exact cell averages."""
    dx = 2.0 / n
    cfg = base_config(1, n, 1, 0.0, 2.0, fixed_dt=0.2 * dx, tau_zero=1, bc=["periodic"] * 4,
                      recon_mode=recon_mode, zeta1_mode=zeta1_mode)
    xe = _edges(0.0, 2.0, n)
    rho = 1.0 + 0.2 * (np.cos(math.pi * xe[:-1]) - np.cos(math.pi * xe[1:])) / (math.pi * dx)
    W = np.stack([rho, rho * 1.0, 1.0 / (GAMMA - 1.0) + 0.5 * rho])[:, None, :]
    return cfg, np.ascontiguousarray(W), 2.0


def sine_1d_exact(n, t):
    dx = 2.0 / n
    xe = _edges(0.0, 2.0, n)
    return 1.0 + 0.2 * (np.cos(math.pi * (xe[:-1] - t)) - np.cos(math.pi * (xe[1:] - t))) / (math.pi * dx)


def _piecewise_1d(n, x0, x1, breaks, states, **kw):
    """Exact cell averages of a piecewise-constant (rho, u, p) on [x0, x1]."""
    xe = _edges(x0, x1, n)
    W = np.zeros((3, n))
    bounds = [x0] + list(breaks) + [x1]
    for s, (rho, u, p) in enumerate(states):
        a, b = bounds[s], bounds[s + 1]
        frac = np.clip((np.minimum(xe[1:], b) - np.maximum(xe[:-1], a)) / (xe[1:] - xe[:-1]), 0.0, 1.0)
        W += frac[None, :] * conservative(rho, u, 0.0, p, dim=1)[:, None]
    cfg = base_config(1, n, 1, x0, x1, **kw)
    return cfg, np.ascontiguousarray(W[:, None, :])


def sod_1d(n=200, c1=0.05, cfl=0.5):
    """Sod tube on [0, 1], (1,0,1) | (0.125,0,0.1) at x = 0.5, non-reflecting
    ends, t = 0.2 (Sec. 3.2(a)); benchmark form: 200 cells, c1 = 0.05."""
    cfg, W = _piecewise_1d(n, 0.0, 1.0, [0.5], [(1.0, 0.0, 1.0), (0.125, 0.0, 0.1)],
                           c1=c1, c2=1.0, cfl=cfl, bc=["extrap"] * 4)
    return cfg, W, 0.2


def blast_1d(n=400, cfl=0.5):
    """Woodward-Colella blast wave, reflecting ends, t = 0.038 (Sec. 3.2(c))."""
    cfg, W = _piecewise_1d(n, 0.0, 1.0, [0.1, 0.9], [(1.0, 0.0, 1000.0), (1.0, 0.0, 0.01), (1.0, 0.0, 100.0)],
                           cfl=cfl, bc=["reflect"] * 4)
    return cfg, W, 0.038


def shu_osher_1d(n=400, cfl=0.5):
    """Shu-Osher shock/entropy-wave interaction on [0, 10], t = 1.8 (Sec. 3.2(b)).
    Both ends are taken as non-reflecting (the right end stays undisturbed up to t = 1.8)."""
    xe = _edges(0.0, 10.0, n)
    dx = 10.0 / n
    W = np.zeros((3, n))
    a, b = xe[:-1], xe[1:]
    left_frac = np.clip((np.minimum(b, 1.0) - a) / dx, 0.0, 1.0)
    W += left_frac[None, :] * conservative(3.857134, 2.629369, 0.0, 10.33333, dim=1)[:, None]
    lo = np.maximum(a, 1.0)
    right_len = np.clip(b - lo, 0.0, None)
    # exact average of 1 + 0.2 sin(5x) over [lo, b]
    with np.errstate(invalid="ignore", divide="ignore"):
        s_avg = np.where(right_len > 0, 1.0 + 0.2 * (np.cos(5 * lo) - np.cos(5 * b)) / (5 * np.where(right_len > 0, right_len, 1.0)), 0.0)
    frac = right_len / dx
    W[0] += frac * s_avg
    W[2] += frac * (1.0 / (GAMMA - 1.0))
    cfg = base_config(1, n, 1, 0.0, 10.0, cfl=cfl, bc=["extrap"] * 4)
    return cfg, np.ascontiguousarray(W[:, None, :]), 1.8


# ---------------------------------------------------------------- 2D problems

def sine_2d(n, recon_mode="hybrid", zeta1_mode="B", cfl=0.5):
    """Sec. 3.3: rho = 1 + 0.2 sin(pi (x + y)), U = V = 1, p = 1 on [0, 2]^2,
    periodic, CFL 0.5, tau = 0.  Reading: t = 2 (the end time of Sec. 3.1)."""
    h = 2.0 / n
    cfg = base_config(2, n, n, 0.0, 2.0, 0.0, 2.0, cfl=cfl, tau_zero=1, bc=["periodic"] * 4,
                      recon_mode=recon_mode, zeta1_mode=zeta1_mode)
    rho = sine_2d_exact(n, 0.0)
    W = np.stack([rho, rho, rho, 1.0 / (GAMMA - 1.0) + rho])
    return cfg, np.ascontiguousarray(W), 2.0


def sine_2d_exact(n, t):
    h = 2.0 / n
    e = _edges(0.0, 2.0, n)
    xl, xr = e[None, :-1], e[None, 1:]
    yl, yr = e[:-1, None], e[1:, None]
    pi = math.pi
    s = (np.sin(pi * (xr + yl - t)) - np.sin(pi * (xl + yl - t)) - np.sin(pi * (xr + yr - t))
         + np.sin(pi * (xl + yr - t))) / (pi * pi * h * h)
    return 1.0 + 0.2 * s


def _gauss_legendre(m):
    x, w = np.polynomial.legendre.leggauss(m)
    return 0.5 * x, 0.5 * w


def vortex_fields(x, y, t=0.0, strength=5.0, mean=(1.0, 1.0), center=(5.0, 5.0), L=10.0):
    """Isentropic vortex (standard closed form), translated by mean*t on the periodic box."""
    xc = (center[0] + mean[0] * t) % L
    yc = (center[1] + mean[1] * t) % L
    dxv = (x - xc + 0.5 * L) % L - 0.5 * L
    dyv = (y - yc + 0.5 * L) % L - 0.5 * L
    r2 = dxv * dxv + dyv * dyv
    f = strength / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u = mean[0] - f * dyv
    v = mean[1] + f * dxv
    T = 1.0 - (GAMMA - 1.0) * strength ** 2 / (8.0 * GAMMA * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (GAMMA - 1.0))
    p = rho * T
    return rho, u, v, p


def vortex_2d(n, t=0.0, strength=5.0, quad=6, mean=(1.0, 1.0)):
    """Isentropic vortex on the periodic [0, 10]^2 (benchmark configuration; not in
    the paper).  Conservative cell averages by quad x quad Gauss-Legendre points."""
    L = 10.0
    h = L / n
    cfg = base_config(2, n, n, 0.0, L, 0.0, L, cfl=0.5, tau_zero=1, bc=["periodic"] * 4)
    gx, gw = _gauss_legendre(quad)
    xc = (np.arange(n) + 0.5) * h
    W = np.zeros((4, n, n))
    for a in range(quad):
        for b in range(quad):
            X = xc[None, :] + gx[a] * h
            Y = xc[:, None] + gx[b] * h
            rho, u, v, p = vortex_fields(X, Y, t, strength, mean)
            W += gw[a] * gw[b] * conservative(rho, u, v, p)
    return cfg, np.ascontiguousarray(W), 2.0


def _quadrants(n_x, n_y, states, xs=0.5, ys=0.5, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
    """Exact cell averages of four constant quadrant states split at (xs, ys).
    states: [(rho,u,v,p) for x<xs,y<ys ; x>=xs,y<ys ; x>=xs,y>=ys ; x<xs,y>=ys]."""
    xe, ye = _edges(x0, x1, n_x), _edges(y0, y1, n_y)
    fx_lo = np.clip((np.minimum(xe[1:], xs) - xe[:-1]) / (xe[1:] - xe[:-1]), 0.0, 1.0)
    fy_lo = np.clip((np.minimum(ye[1:], ys) - ye[:-1]) / (ye[1:] - ye[:-1]), 0.0, 1.0)
    W = np.zeros((4, n_y, n_x))
    fr = [np.outer(fy_lo, fx_lo), np.outer(fy_lo, 1 - fx_lo), np.outer(1 - fy_lo, 1 - fx_lo),
          np.outer(1 - fy_lo, fx_lo)]
    for s, st in enumerate(states):
        W += fr[s][None] * conservative(*st)[:, None, None]
    return np.ascontiguousarray(W)


RIEMANN_SEED = 20230411


def riemann4_states(seed=RIEMANN_SEED):
    """Four quadrant states rho, p ~ U[0.1, 2], u, v ~ U[-1, 1] from numpy PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(4):
        rho = rng.uniform(0.1, 2.0)
        u = rng.uniform(-1.0, 1.0)
        v = rng.uniform(-1.0, 1.0)
        p = rng.uniform(0.1, 2.0)
        out.append((rho, u, v, p))
    return out


def riemann4_2d(n, seed=RIEMANN_SEED, cfl=0.5, ny=None):
    """Four-quadrant Riemann problem on [0, 1]^2 with seeded quadrant states,
    non-reflecting boundaries, c1 = 0.01, c2 = 1 (benchmark configuration)."""
    ny = n if ny is None else ny
    cfg = base_config(2, n, ny, 0.0, 1.0, 0.0, 1.0, cfl=cfl, c1=0.01, c2=1.0, bc=["extrap"] * 4)
    return cfg, _quadrants(n, ny, riemann4_states(seed)), 0.2


def riemann_config1(n=500):
    """Sec. 3.4(a), configuration 1 (four rarefactions), t = 0.2."""
    st = [(0.1072, -0.7259, -1.4045, 0.0439), (0.2579, 0.0, -1.4045, 0.15), (1.0, 0.0, 0.0, 1.0),
          (0.5197, -0.7259, 0.0, 0.4)]
    cfg = base_config(2, n, n, 0.0, 1.0, 0.0, 1.0, cfl=0.5, bc=["extrap"] * 4)
    return cfg, _quadrants(n, n, st), 0.2


def riemann_config6(n=500):
    """Sec. 3.4(b), configuration 6 (four contacts), CFL 0.95, t = 0.6."""
    st = [(1.0, -0.75, 0.5, 1.0), (3.0, -0.75, -0.5, 1.0), (1.0, -0.75, -0.5, 1.0), (2.0, 0.75, 0.5, 1.0)]
    cfg = base_config(2, n, n, 0.0, 1.0, 0.0, 1.0, cfl=0.95, bc=["extrap"] * 4)
    return cfg, _quadrants(n, n, st), 0.6


def viscous_shock_tube(nx=500, ny=None, Re=200.0, prandtl=1.0, cfl=0.3):
    """Sec. 3.6: [0,1] x [0,0.5], (120,0,120/g) | (1.2,0,1.2/g) at x = 0.5, mu = 1/Re,
    no-slip adiabatic walls left, right and bottom, symmetry on top, t = 1."""
    ny = nx // 2 if ny is None else ny
    cfg = base_config(2, nx, ny, 0.0, 1.0, 0.0, 0.5, viscous=1, mu=1.0 / Re, prandtl=prandtl, cfl=cfl,
                      c1=0.0, c2=1.0, bc=["noslip", "noslip", "noslip", "symmetry"])
    g = GAMMA
    st_l, st_r = (120.0, 0.0, 0.0, 120.0 / g), (1.2, 0.0, 0.0, 1.2 / g)
    W = _quadrants(nx, ny, [st_l, st_r, st_r, st_l], xs=0.5, ys=0.25, y0=0.0, y1=0.5)
    return cfg, W, 1.0


# ---- double Mach reflection (Sec. 3.5)
DMR_POST = (8.0, 4.125 * math.sqrt(3.0), -4.125, 116.5)     # (rho, U, V, p) behind the Mach 10 shock
DMR_PRE = (1.4, 0.0, 0.0, 1.0)                               # ahead of it
DMR_X0 = 1.0 / 6.0                                           # the shock meets the wall at x = 1/6 at t = 0
DMR_COT = 1.0 / math.sqrt(3.0)                               # cot 60 deg: the shock is inclined 60 deg to the x-axis
DMR_SPEED = 20.0                                             # line x = 1/6 + (y + 20 t)/sqrt(3) (normal speed 10)


def _halfplane_fraction(xe, ye, a, c):
    """Exact area fraction of each cell [xe_i, xe_i+1] x [ye_j, ye_j+1] lying in x < a + c y (c > 0)."""
    xl, xr = xe[None, :-1], xe[None, 1:]
    yl, yr = ye[:-1, None], ye[1:, None]
    dx = xr - xl

    def ramp_integral(z):              # int_{-inf}^{z} clip(s, 0, dx) ds
        return np.where(z <= 0.0, 0.0, np.where(z <= dx, 0.5 * z * z, 0.5 * dx * dx + dx * (z - dx)))

    area = (ramp_integral(a + c * yr - xl) - ramp_integral(a + c * yl - xl)) / c
    return np.clip(area / (dx * (yr - yl)), 0.0, 1.0)


def _oblique_shock_state(nx, ny, x0, x1, y0, y1, t=0.0):
    """Exact cell averages of the straight Mach 10 shock of Sec. 3.5 at time t (no wall)."""
    frac = _halfplane_fraction(_edges(x0, x1, nx), _edges(y0, y1, ny), DMR_X0 + DMR_COT * DMR_SPEED * t, DMR_COT)
    post, pre = conservative(*DMR_POST), conservative(*DMR_PRE)
    return np.ascontiguousarray(frac[None] * post[:, None, None] + (1.0 - frac[None]) * pre[:, None, None])


def double_mach(nx=960, ny=240, cfl=0.8):
    """Sec. 3.5: [0, 4] x [0, 1], the Mach 10 shock at 60 deg through (1/6, 0), the post-shock
    state flowing in on the left and on the bottom up to x = 1/6, a slip wall beyond, the top
    following the exact shock motion, the right end non-reflecting; c1 = 0, c2 = 1, t = 0.2."""
    post = conservative(*DMR_POST)
    cfg = base_config(2, nx, ny, 0.0, 4.0, 0.0, 1.0, cfl=cfl, c1=0.0, c2=1.0,
                      bc=["inflow", "extrap", "shock_wall", "shock_track"],
                      bc_state=[list(post), [0.0] * 4, list(post), list(post)],
                      shock_pre=list(conservative(*DMR_PRE)), shock_x0=DMR_X0, shock_cot=DMR_COT,
                      shock_speed=DMR_SPEED)
    return cfg, _oblique_shock_state(nx, ny, 0.0, 4.0, 0.0, 1.0), 0.2


def oblique_shock(nx=64, ny=32, cfl=0.8, x1=1.0, y1=0.5):
    """The straight Mach 10 shock of Sec. 3.5 alone (no wall): post-shock inflow on the left,
    both y-sides following the exact shock motion, non-reflecting right end.  Its exact
    solution is the initial discontinuity translated at the shock speed."""
    post = conservative(*DMR_POST)
    cfg = base_config(2, nx, ny, 0.0, x1, 0.0, y1, cfl=cfl, c1=0.0, c2=1.0,
                      bc=["inflow", "extrap", "shock_track", "shock_track"],
                      bc_state=[list(post), [0.0] * 4, list(post), list(post)],
                      shock_pre=list(conservative(*DMR_PRE)), shock_x0=DMR_X0, shock_cot=DMR_COT,
                      shock_speed=DMR_SPEED)
    return cfg, _oblique_shock_state(nx, ny, 0.0, x1, 0.0, y1)


def oblique_shock_exact(nx, ny, t, x1=1.0, y1=0.5):
    return _oblique_shock_state(nx, ny, 0.0, x1, 0.0, y1, t)


def uniform_2d(n, state=(1.3, 0.4, -0.7, 2.1), bc="periodic", ny=None):
    ny = n if ny is None else ny
    cfg = base_config(2, n, ny, 0.0, 1.0, 0.0, 1.0, bc=[bc] * 4)
    W = np.broadcast_to(conservative(*state)[:, None, None], (4, ny, n)).copy()
    return cfg, W, 0.1


def random_smooth_2d(nx, ny, seed=7, amp=0.1, bc="periodic"):
    """Smooth random periodic field (a few Fourier modes) for parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    def field(base):
        f = np.full_like(X, base)
        for _ in range(3):
            kx, ky = rng.integers(1, 3, size=2)
            ph = rng.uniform(0, 2 * math.pi)
            f += amp * base * rng.uniform(-1, 1) * np.sin(2 * math.pi * (kx * X + ky * Y) + ph)
        return f
    rho = field(1.0)
    u = field(0.5) - 0.25
    v = field(0.5) - 0.25
    p = field(1.0)
    cfg = base_config(2, nx, ny, 0.0, 1.0, 0.0, 1.0, bc=[bc] * 4)
    return cfg, np.ascontiguousarray(conservative(rho, u, v, p)), 0.05


# ---------------------------------------------------------------- many-solve workloads

BATCH_SEED = 20230412
SERVE_SEED = 20230413


def batched_workload(n_solves=256, seed=BATCH_SEED, lo=64, hi=1024):
    """Independent four-quadrant Riemann solves with sides drawn log-uniformly in [lo, hi]
    (numpy PCG64), each with its own seeded quadrant states.  Returns a list of (cfg, W)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_solves))).astype(int)
    out = []
    for k, n in enumerate(sides):
        cfg, W, _ = riemann4_2d(int(n), seed=seed + 1 + k)
        out.append((cfg, W))
    return out


def served_trace(n_requests=1000, rate=200.0, seed=SERVE_SEED, max_1d=8192, max_2d=1024, max_ns=2048):
    """Poisson-arrival stream of mixed solves: one third each 1D Sod-type shock tubes
    (256..max_1d cells, log-uniform), 2D Euler four-quadrant Riemann or isentropic-vortex
    problems (side 64..max_2d), 2D Navier-Stokes viscous shock tubes (nx 128..max_ns,
    ny = nx/2, Re ~ U[200, 2000]); end times t_end ~ U[0.05, 0.3].  A maximum below its
    range's lower end lowers that end to it (small traces for tests).
    Returns a list of dicts {id, arrival, kind, cfg, W, t_end} sorted by arrival time."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo_1d, lo_2d, lo_ns = min(256, max_1d), min(64, max_2d), min(128, max_ns)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        kind = int(rng.integers(0, 3))
        t_end = float(rng.uniform(0.05, 0.3))
        if kind == 0:
            n = int(np.rint(math.exp(rng.uniform(math.log(lo_1d), math.log(max_1d)))))
            cfg, W, _ = sod_1d(n)
            name = "sod1d_%d" % n
        elif kind == 1:
            n = int(np.rint(math.exp(rng.uniform(math.log(lo_2d), math.log(max_2d)))))
            if rng.uniform() < 0.5:
                cfg, W, _ = riemann4_2d(n, seed=seed + 7919 * (i + 1))
                name = "riemann_%d" % n
            else:
                cfg, W, _ = vortex_2d(n)
                name = "vortex_%d" % n
        else:
            nx = int(np.rint(math.exp(rng.uniform(math.log(lo_ns), math.log(max_ns)))))
            nx += nx % 2
            Re = float(rng.uniform(200.0, 2000.0))
            cfg, W, _ = viscous_shock_tube(nx, nx // 2, Re=Re)
            name = "ns_%dx%d_Re%.0f" % (nx, nx // 2, Re)
        out.append(dict(id=i, arrival=t, kind=name, cfg=cfg, W=W, t_end=t_end))
    return out
