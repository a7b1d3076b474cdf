"""Problems whose exact discrete answer is known independently of any implementation of
the scheme (test inputs and expected values; no arithmetic of the scheme)."""
import numpy as np

from paper_2304_05572_gb300 import problems as P


def _poly_avg(xl, xr, c, shift=0.0):
    """Exact average over [xl, xr] of sum_k c_k (x - shift)^k."""
    a, b = xl - shift, xr - shift
    return sum(ck * (b ** (k + 1) - a ** (k + 1)) / (k + 1) for k, ck in enumerate(c)) / (xr - xl)


def quartic_advection(dim, n, cfl):
    """Density a quartic (per direction), constant velocity and pressure, tau = 0: the exact
    solution is the profile translated, and every time derivative beyond the fourth vanishes.
    Returns (cfg, W, exact state after one step of dt)."""
    G = 1.4
    cx = np.array([2.0, 1.0, -1.0, 2.0, 30.0])
    cy = np.array([0.0, -1.0, 2.0, 1.0, 20.0])
    U, V, p = (0.7, -0.4, 40.0) if dim == 2 else (0.7, 0.0, 40.0)
    e = np.linspace(0.0, 1.0, n + 1)

    def cons(t):
        if dim == 1:
            rho = _poly_avg(e[:-1], e[1:], cx, U * t)[None, :]
            return np.stack([rho, rho * U, p / (G - 1) + 0.5 * rho * U * U])
        rho = _poly_avg(e[None, :-1], e[None, 1:], cx, U * t) + _poly_avg(e[:-1, None], e[1:, None], cy, V * t)
        return np.stack([rho, rho * U, rho * V, p / (G - 1) + 0.5 * rho * (U * U + V * V)])

    W = cons(0.0)
    dt = cfl * (1.0 / n) / (np.hypot(U, V) + np.sqrt(G * p / W[0].min()))
    cfg = P.base_config(dim, n, n, 0.0, 1.0, 0.0, 1.0, fixed_dt=dt, tau_zero=1, bc=["extrap"] * 4,
                        recon_mode="linear")
    return cfg, np.ascontiguousarray(W), cons(dt), dt


def all_troubled_1d(n=24, seed=5):
    """A periodic 1D state whose density and pressure alternate between two levels from cell
    to cell (with seeded noise): every cell is an extremum, so the indicator flags every cell
    in both stages and the hybrid scheme is WENO-AO everywhere."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.arange(n)
    rho = np.where(x % 2 == 0, 1.0, 3.0) * (1 + 0.2 * rng.random(n))
    u = 0.1 * rng.standard_normal(n)
    p = np.where(x % 2 == 0, 1.0, 2.5) * (1 + 0.2 * rng.random(n))
    W = P.conservative(rho, u, 0 * u, p, dim=1)[:, None, :]
    cfg = P.base_config(1, n, 1, 0.0, 1.0, bc=["periodic"] * 4)
    return cfg, np.ascontiguousarray(W)
