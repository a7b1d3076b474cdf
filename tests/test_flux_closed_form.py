"""The closed-form gas-kinetic flux of the CUDA kernels (csrc/hgks_math.cuh), evaluated on
the host, against the oracle's literal moment integration (Sec. 2.1, Eqs. (6)-(12),
(46)-(47)): both time integrals of Eq. (12) in the combinations the two S2O4 stages use
(Eqs. (17)-(20)), for Euler with tau > 0 and tau = 0, Navier-Stokes with Pr = 1 and with
the Prandtl fix, in 2D and 1D.  This checks the kernels' flux algebra without a GPU."""
import numpy as np
import pytest

import oracle
from paper_2304_05572_gb300 import flopcount, problems as P

RNG = np.random.default_rng(20230414)


def _state(dim, rho, u, v, p):
    return P.conservative(rho, u, v, p, dim=dim)[: dim + 2]


def _cases(dim, n=6):
    out = []
    for _ in range(n):
        Wl = _state(dim, RNG.uniform(0.3, 2.0), RNG.uniform(-1, 1), RNG.uniform(-1, 1), RNG.uniform(0.2, 2.0))
        Wr = _state(dim, RNG.uniform(0.3, 2.0), RNG.uniform(-1, 1), RNG.uniform(-1, 1), RNG.uniform(0.2, 2.0))
        d = [RNG.normal(0, 0.3, dim + 2) for _ in range(4)]
        out.append((Wl, d[0], d[1] if dim == 2 else np.zeros(dim + 2), Wr, d[2], d[3] if dim == 2 else np.zeros(dim + 2)))
    return out


@pytest.mark.parametrize("dim", [2, 1])
@pytest.mark.parametrize("kind", ["euler", "tau0", "ns", "ns_prfix"])
def test_closed_form_flux_matches_oracle(dim, kind):
    dt = 2e-3
    kw = dict(gamma=1.4, c1=0.01, c2=1.0)
    if kind == "tau0":
        kw.update(tau_zero=True)
    if kind.startswith("ns"):
        kw.update(viscous=True, mu=1e-3, c1=0.0, prandtl=0.73 if kind == "ns_prfix" else 1.0)
    cfg = P.base_config(dim, 8, 8 if dim == 2 else 1, 0.0, 1.0, viscous=int(kw.get("viscous", False)),
                        mu=kw.get("mu", 0.0), prandtl=kw.get("prandtl", 1.0), c1=kw["c1"], c2=kw["c2"],
                        tau_zero=int(kw.get("tau_zero", False)))
    for Wl, Wlx, Wly, Wr, Wrx, Wry in _cases(dim):
        Fd, Fh = oracle.point_flux(cfg, Wl, Wlx, Wr, Wrx, dt, Wly=Wly if dim == 2 else None,
                                   Wry=Wry if dim == 2 else None)
        ok0, o0, o1 = flopcount.flux_values(dim, 0, Wl, Wlx, Wly, Wr, Wrx, Wry, dt, **kw)
        ok1, p0, _ = flopcount.flux_values(dim, 1, Wl, Wlx, Wly, Wr, Wrx, Wry, dt, **kw)
        assert ok0 and ok1
        scale = np.abs(Fd).max()
        np.testing.assert_allclose(o0, Fh, rtol=0, atol=1e-13 * scale)
        np.testing.assert_allclose(o1, (8.0 * Fh - Fd) / 3.0, rtol=0, atol=1e-13 * scale)
        np.testing.assert_allclose(p0, 4.0 / 3.0 * (Fd - 2.0 * Fh), rtol=0, atol=1e-13 * scale)
