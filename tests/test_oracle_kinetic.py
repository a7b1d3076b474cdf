"""Pins of the oracle's kinetic layer (Sec. 2.1) against results fixed by the
mathematics: Gaussian integrals by adaptive quadrature, the exact logarithmic
derivative of a Maxwellian, the Euler equations, and the Navier-Stokes
(Chapman-Enskog, Pr = 1) flux."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2304_05572_gb300 import problems as P

G = 1.4


@pytest.mark.parametrize("U,lam", [(0.3, 0.7), (-1.2, 2.5), (0.0, 1.0), (2.0, 0.4)])
def test_moments_match_quadrature(U, lam):
    K = oracle.dof_K(2, G)
    u, up, un, v, x = oracle.moments(2, K, U, -0.4, lam)
    w = lambda s: math.sqrt(lam / math.pi) * math.exp(-lam * (s - U) ** 2)
    for n in range(8):
        full = integrate.quad(lambda s: s ** n * w(s), -np.inf, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]
        pos = integrate.quad(lambda s: s ** n * w(s), 0, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]
        neg = integrate.quad(lambda s: s ** n * w(s), -np.inf, 0, epsabs=0, epsrel=1e-13, limit=200)[0]
        scale = max(1.0, abs(full))
        assert abs(u[n] - full) <= 1e-11 * scale
        assert abs(up[n] - pos) <= 1e-11 * max(1.0, abs(pos))
        assert abs(un[n] - neg) <= 1e-11 * max(1.0, abs(neg))
        assert abs(up[n] + un[n] - u[n]) <= 1e-11 * scale
    # internal energy: K independent Gaussians of variance 1/(2 lam)
    assert x[1] == pytest.approx(K / (2 * lam), rel=1e-14)
    assert x[2] == pytest.approx(K * (K + 2) / (4 * lam * lam), rel=1e-14)


def test_internal_dof():
    # 2D: K = (5 - 3g)/(g - 1) + 1 = 3 at g = 1.4; 1D reading: (3 - g)/(g - 1) = 4
    assert oracle.dof_K(2, 1.4) == pytest.approx(3.0, abs=1e-14)
    assert oracle.dof_K(1, 1.4) == pytest.approx(4.0, abs=1e-14)


def _prim_to_cons(r, u, v, p, dim=2):
    return P.conservative(r, u, v, p, dim=dim)


@pytest.mark.parametrize("dim", [1, 2])
def test_micro_slope_is_log_derivative_of_maxwellian(dim):
    """<a> = dW/dx (Eq. 8) is solved exactly by a = d(ln g)/dx, expanded in psi."""
    r, u, v, p = 1.3, 0.4, (-0.3 if dim == 2 else 0.0), 0.9
    dr, du, dv, dp = 0.11, -0.07, (0.05 if dim == 2 else 0.0), 0.23
    lam = r / (2 * p)
    dlam = (dr * p - r * dp) / (2 * p * p)
    K = oracle.dof_K(dim, G)
    N = K + dim
    # ln g = ln r + (N/2) ln lam - lam((u-U)^2 + (v-V)^2 + xi^2): derivative in psi = (1, u, v, |u|^2/2)
    a4 = -2 * dlam
    a2 = 2 * dlam * u + 2 * lam * du
    a3 = 2 * dlam * v + 2 * lam * dv
    a1 = dr / r + 0.5 * N * dlam / lam - dlam * (u * u + v * v) - 2 * lam * (u * du + v * dv)
    exact = np.array([a1, a2, a3, a4]) if dim == 2 else np.array([a1, a2, a4])
    h = 1e-6
    W = _prim_to_cons(r, u, v, p, dim)
    dW = (_prim_to_cons(r + h * dr, u + h * du, v + h * dv, p + h * dp, dim)
          - _prim_to_cons(r - h * dr, u - h * du, v - h * dv, p - h * dp, dim)) / (2 * h)
    a = oracle.micro_slope(dim, G, W, dW)
    np.testing.assert_allclose(a, exact, rtol=1e-8, atol=1e-9)


def _euler_fluxes(W, dim=2):
    if dim == 1:
        r, ru, E = W
        u = ru / r
        p = (G - 1) * (E - 0.5 * r * u * u)
        return np.array([ru, ru * u + p, u * (E + p)]), None
    r, ru, rv, E = W
    u, v = ru / r, rv / r
    p = (G - 1) * (E - 0.5 * r * (u * u + v * v))
    return (np.array([ru, ru * u + p, ru * v, u * (E + p)]),
            np.array([rv, rv * u, rv * v + p, v * (E + p)]))


def _dirder(f, W, d, h=1e-5):
    # 4th-order central difference of f along d
    return (-f(W + 2 * h * d) + 8 * f(W + h * d) - 8 * f(W - h * d) + f(W - 2 * h * d)) / (12 * h)


def test_time_slope_reproduces_euler_equations():
    """<a1 u + a2 v + A> = 0 (Eq. 9) makes int psi A g = W_t = -(F_x + G_y) of the Euler equations."""
    W = _prim_to_cons(1.3, 0.4, -0.3, 0.9)
    Wx = np.array([0.1, -0.05, 0.07, 0.2])
    Wy = np.array([-0.03, 0.02, 0.05, -0.1])
    a1 = oracle.micro_slope(2, G, W, Wx)
    a2 = oracle.micro_slope(2, G, W, Wy)
    A = oracle.time_slope(2, G, W, a1, a2)
    Wt = oracle.slope_moment(2, G, W, A, 0)
    F = lambda w: _euler_fluxes(w)[0]
    Gf = lambda w: _euler_fluxes(w)[1]
    expect = -(_dirder(F, W, Wx) + _dirder(Gf, W, Wy))
    np.testing.assert_allclose(Wt, expect, rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("tau_mode", ["zero", "inviscid", "viscous"])
def test_uniform_state_flux_is_euler_flux(dim, tau_mode):
    """For a uniform state and any tau, F(delta) = delta F_Euler(W) (Eq. 12)."""
    W = _prim_to_cons(0.8, -0.6, 0.3 if dim == 2 else 0.0, 1.7, dim)
    z = np.zeros(dim + 2)
    kw = dict(tau_zero=1) if tau_mode == "zero" else (dict(viscous=1, mu=0.01) if tau_mode == "viscous" else {})
    cfg = P.base_config(dim, 8, 8, 0, 1, **kw)
    dt = 0.013
    Fd, Fh = oracle.point_flux(cfg, W, z, W, z, dt)
    FE = _euler_fluxes(W, dim)[0]
    np.testing.assert_allclose(Fd, dt * FE, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(Fh, 0.5 * dt * FE, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("dim", [1, 2])
def test_tau_zero_flux_is_lax_wendroff(dim):
    """tau = 0: F(delta) = delta F(W) + delta^2/2 dF/dW W_t with W_t from the Euler equations."""
    W = _prim_to_cons(1.3, 0.4, -0.3 if dim == 2 else 0.0, 0.9, dim)
    Wx = np.array([0.1, -0.05, 0.07, 0.2])[: dim + 2] if dim == 2 else np.array([0.1, -0.05, 0.2])
    Wy = np.array([-0.03, 0.02, 0.05, -0.1]) if dim == 2 else None
    cfg = P.base_config(dim, 8, 8, 0, 1, tau_zero=1)
    d = 2e-3
    Fd, _ = oracle.point_flux(cfg, W, Wx, W, Wx, d, Wly=Wy, Wry=Wy)
    F = lambda w: _euler_fluxes(w, dim)[0]
    Wt = -_dirder(F, W, Wx)
    if dim == 2:
        Wt = Wt - _dirder(lambda w: _euler_fluxes(w)[1], W, Wy)
    expect = d * F(W) + 0.5 * d * d * _dirder(F, W, Wt)
    np.testing.assert_allclose(Fd, expect, rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("prandtl", [1.0, 0.73, 2.0])
def test_viscous_flux_is_navier_stokes(dim, prandtl):
    """With equal sides and tau = mu/p, F^n of Eq. (17) is the Chapman-Enskog
    Navier-Stokes flux of the BGK model (Pr = 1): stress mu(grad U + grad U^T - 2/(K+D) div U I),
    heat flux -mu c_p grad T with c_p = (K + D + 2)/2.  With the Prandtl-number fix of the
    energy flux (an extension: the paper's flux has Pr = 1) the heat flux is -mu c_p/Pr grad T
    and nothing else changes."""
    mu = 2e-3
    r, u, v, p = 1.3, 0.4, (-0.3 if dim == 2 else 0.0), 0.9
    W = _prim_to_cons(r, u, v, p, dim)
    Wx = np.array([0.1, -0.05, 0.07, 0.2]) if dim == 2 else np.array([0.1, -0.05, 0.2])
    Wy = np.array([-0.03, 0.02, 0.05, -0.1]) if dim == 2 else None
    cfg = P.base_config(dim, 8, 8, 0, 1, viscous=1, mu=mu, c2=0.0, prandtl=prandtl)
    d = 1e-3
    Fd, Fh = oracle.point_flux(cfg, W, Wx, W, Wx, d, Wly=Wy, Wry=Wy)
    Fn = (4 * Fh - Fd) / d
    K = oracle.dof_K(dim, G)

    def prim(w):
        if dim == 1:
            rr, ru, E = w
            uu = ru / rr
            pp = (G - 1) * (E - 0.5 * rr * uu * uu)
            return np.array([uu, 0.0, pp / rr])
        rr, ru, rv, E = w
        uu, vv = ru / rr, rv / rr
        pp = (G - 1) * (E - 0.5 * rr * (uu * uu + vv * vv))
        return np.array([uu, vv, pp / rr])

    gx = _dirder(prim, W, Wx)
    gy = _dirder(prim, W, Wy) if dim == 2 else np.zeros(3)
    div = gx[0] + gy[1]
    sxx = mu * (2 * gx[0] - 2.0 / (K + dim) * div)
    sxy = mu * (gy[0] + gx[1])
    q = -mu / prandtl * (K + dim + 2) / 2 * gx[2]
    FE = _euler_fluxes(W, dim)[0]
    if dim == 1:
        Fv = np.array([0.0, sxx, u * sxx - q])
    else:
        Fv = np.array([0.0, sxx, sxy, u * sxx + v * sxy - q])
    np.testing.assert_allclose(Fn, FE - Fv, rtol=1e-9, atol=1e-10)


def test_flux_upwinds_by_particle_direction():
    """Free transport limit (tau >> dt, no slopes): the flux is the kinetic flux-vector
    split of the two sides: particles with u > 0 come from the left state."""
    Wl = _prim_to_cons(1.0, 0.3, 0.0, 1.0, 1)
    Wr = _prim_to_cons(0.2, -0.1, 0.0, 0.3, 1)
    z = np.zeros(3)
    cfg = P.base_config(1, 8, 1, 0, 1, c1=1e6, c2=0.0)   # tau = 1e6 dt: the g0 terms are O(dt/tau)
    dt = 1e-3
    Fd, _ = oracle.point_flux(cfg, Wl, z, Wr, z, dt)
    K = oracle.dof_K(1, G)

    def half_flux(W, sign):
        r, ru, E = W
        U = ru / r
        p = (G - 1) * (E - 0.5 * r * U * U)
        lam = r / (2 * p)
        w = lambda s: r * math.sqrt(lam / math.pi) * math.exp(-lam * (s - U) ** 2)
        lo, hi = (0, np.inf) if sign > 0 else (-np.inf, 0)
        m = [integrate.quad(lambda s, n=n: s ** n * w(s), lo, hi, epsabs=0, epsrel=1e-13)[0] for n in range(4)]
        xi2 = K / (2 * lam)
        return np.array([m[1], m[2], 0.5 * (m[3] + m[1] * xi2)])

    expect = dt * (half_flux(Wl, +1) + half_flux(Wr, -1))
    np.testing.assert_allclose(Fd, expect, rtol=2e-6)


def test_flux_rejects_nonphysical_state():
    cfg = P.base_config(1, 8, 1, 0, 1)
    bad = np.array([1.0, 0.0, -1.0])
    with pytest.raises(RuntimeError):
        oracle.point_flux(cfg, bad, np.zeros(3), bad, np.zeros(3), 1e-3)
