"""Pins of the oracle's reconstruction layer (Sec. 2.3.1) against exact results:
polynomial exactness of the linear and sub-stencil reconstructions, smoothness
indicators by exact symbolic integration of the fitted polynomials (Eq. 39),
hand-computed indicator decisions (Steps 1-4), and the eigen-decomposition of
the Euler Jacobian used by the characteristic projection."""
import math

import numpy as np
import pytest

import oracle

G = 1.4


def _avgs(coeffs, offsets=range(-2, 3)):
    """Exact cell averages (cell units) of sum c_k xi^k over cells [m - 1/2, m + 1/2]."""
    out = []
    for m in offsets:
        s = 0.0
        for k, c in enumerate(coeffs):
            s += c * (((m + 0.5) ** (k + 1) - (m - 0.5) ** (k + 1)) / (k + 1))
        out.append(s)
    return np.array(out)


def _val(coeffs, x):
    return sum(c * x ** k for k, c in enumerate(coeffs))


def _der(coeffs, x):
    return sum(k * c * x ** (k - 1) for k, c in enumerate(coeffs) if k > 0)


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_linear_face_exact_up_to_quartics(deg):
    rng = np.random.default_rng(deg)
    c = rng.uniform(-1, 1, deg + 1)
    q = _avgs(c)
    h = 0.37
    vL, dL = oracle.linear_face(q, h, +1)
    vR, dR = oracle.linear_face(q, h, -1)
    assert vL == pytest.approx(_val(c, 0.5), abs=1e-13)
    assert dL == pytest.approx(_der(c, 0.5) / h, abs=1e-12)
    assert vR == pytest.approx(_val(c, -0.5), abs=1e-13)
    assert dR == pytest.approx(_der(c, -0.5) / h, abs=1e-12)


def test_linear_face_constant_and_mirror():
    q = np.full(5, 2.75)
    v, d = oracle.linear_face(q, 0.1, +1)
    assert v == 2.75 and d == 0.0
    rng = np.random.default_rng(3)
    for _ in range(50):
        q = rng.uniform(-2, 2, 5)
        vL, dL = oracle.linear_face(q, 0.2, +1)
        vR, dR = oracle.linear_face(q[::-1], 0.2, -1)
        assert vL == vR and dL == -dR          # mirrored windows give mirrored values exactly


def test_betas_match_exact_integration():
    sp = pytest.importorskip("sympy")
    xi = sp.symbols("xi")
    rng = np.random.default_rng(11)
    for trial in range(3):
        q = [sp.Rational(int(v), 97) for v in rng.integers(-300, 300, 5)]
        def fit(offs, deg, vals):
            cs = sp.symbols("c0:%d" % (deg + 1))
            p = sum(cs[k] * xi ** k for k in range(deg + 1))
            eqs = [sp.integrate(p, (xi, o - sp.Rational(1, 2), o + sp.Rational(1, 2))) - v for o, v in zip(offs, vals)]
            return p.subs(sp.solve(eqs, cs))
        polys = [fit([-2, -1, 0], 2, q[0:3]), fit([-1, 0, 1], 2, q[1:4]), fit([0, 1, 2], 2, q[2:5]),
                 fit([-2, -1, 0, 1, 2], 4, q)]
        degs = [2, 2, 2, 4]
        exact = [float(sum(sp.integrate(sp.diff(p, xi, r) ** 2, (xi, -sp.Rational(1, 2), sp.Rational(1, 2)))
                           for r in range(1, d + 1))) for p, d in zip(polys, degs)]
        b = oracle.ao_betas([float(v) for v in q])
        np.testing.assert_allclose(b, exact, rtol=1e-13)


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_ao_face_exact_up_to_quadratics(deg):
    rng = np.random.default_rng(10 + deg)
    c = rng.uniform(-1, 1, deg + 1)
    q = _avgs(c)
    for side, x in ((+1, 0.5), (-1, -0.5)):
        v, d = oracle.ao_face_scalar(q, side)
        assert v == pytest.approx(_val(c, x), abs=1e-13)
        assert d == pytest.approx(_der(c, x), abs=1e-12)


def test_ao_reduces_to_linear_when_smooth():
    """All beta equal (linear data) -> delta = 0, omega = gamma, and Eq. (41) collapses to the quartic."""
    q = _avgs([0.3, -1.7])
    b = oracle.ao_betas(q)
    assert np.ptp(b) == pytest.approx(0.0, abs=1e-13)
    vAO, dAO = oracle.ao_face_scalar(q, +1)
    vL, dL = oracle.linear_face(q, 1.0, +1)
    assert vAO == pytest.approx(vL, abs=1e-14) and dAO == pytest.approx(dL, abs=1e-13)


def test_ao_is_nonoscillatory_at_a_step():
    q = np.array([0.0, 0.0, 0.0, 1.0, 1.0])
    vL, _ = oracle.linear_face(q, 1.0, +1)
    vA, _ = oracle.ao_face_scalar(q, +1)
    # the quartic overshoots into the jump; the AO value stays close to the sub-stencil that avoids it
    assert abs(vA - 1.0 / 3.0) < abs(vL - 1.0 / 3.0) + 1e-12 or vA < vL
    assert 0.0 - 1e-12 <= vA <= 1.0


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_gauss_point_linear_exact(deg):
    rng = np.random.default_rng(20 + deg)
    c = rng.uniform(-1, 1, deg + 1)
    q = _avgs(c)
    g = 0.5 / math.sqrt(3.0)
    v, d = oracle.gauss_scalar(q, use_ao=False)
    np.testing.assert_allclose(v, [_val(c, -g), _val(c, g)], atol=1e-13)
    np.testing.assert_allclose(d, [_der(c, -g), _der(c, g)], atol=1e-12)
    if deg <= 2:
        va, da = oracle.gauss_scalar(q, use_ao=True)
        np.testing.assert_allclose(va, [_val(c, -g), _val(c, g)], atol=1e-13)
        np.testing.assert_allclose(da, [_der(c, -g), _der(c, g)], atol=1e-12)


# ---- troubled-cell indicator, Steps 1-3 ----

def test_indicator_smooth_data_not_troubled():
    Z1 = oracle.zeta1_scaled("B", 0.1)
    assert oracle.indicator(np.full(5, 3.0), Z1) == 0
    assert oracle.indicator(_avgs([1.0, 0.5]), Z1) == 0
    # strong curvature (fails Step 1) but a smooth extremum at the centre: Step 3 keeps it smooth
    q = _avgs([0.0, 0.0, 40.0])
    assert abs(4 * q[0] + q[1] - 10 * q[2] + q[3] + 4 * q[4]) > Z1
    assert oracle.indicator(q, Z1) == 0
    # extremum far outside the stencil: Step 2
    q = _avgs([100.0, -20.0, 1.0])     # vertex at xi = 10
    assert oracle.indicator(q, Z1) == 0


@pytest.mark.parametrize("h", [0.05, 0.1, 0.2])
def test_indicator_step_threshold_reading_B(h):
    """A jump J between cells i and i+1 gives |2 abar2| = 5J/(17 h^2) (Eq. 24); with
    zeta1 = 5/(17 h) Step 1 passes it exactly when J > h, and Step 3 then flags it."""
    Z1 = oracle.zeta1_scaled("B", h)
    for J, expect in ((0.9 * h, 0), (1.1 * h, 1), (50 * h, 1)):
        q = np.array([0.0, 0.0, 0.0, J, J])
        assert oracle.indicator(q, Z1) == expect
        assert oracle.indicator(-q, Z1) == expect
        assert oracle.indicator(q[::-1].copy(), Z1) == expect


def test_indicator_readings():
    h = 0.1
    assert oracle.zeta1_scaled("B", h) == pytest.approx(5 * h)
    assert oracle.zeta1_scaled("A", h) == pytest.approx(5 * h ** 3)
    assert oracle.zeta1_scaled("C", h) == pytest.approx(5.0)


def test_indicator_step3_zero_curvature_guard():
    # ahat2 == 0 and ahat1 != 0: xhat is pushed to +-1e30, far from xbar -> troubled
    q = np.array([2.0, 0.0, 1.0, 2.0, 1.0])   # D = 4 (fails Step 1), xbar = 0 (inside)
    assert 0.5 * ((q[1] + q[3]) - 2 * q[2]) == 0.0
    assert oracle.indicator(q, 1e-3) == 1


# ---- characteristic decomposition ----

def _jac(dim, W, n, h=1e-6):
    def flux(w):
        if dim == 1:
            r, ru, E = w
            u = ru / r
            p = (G - 1) * (E - 0.5 * r * u * u)
            return np.array([ru, ru * u + p, u * (E + p)])
        r, ru, rv, E = w
        u, v = ru / r, rv / r
        p = (G - 1) * (E - 0.5 * r * (u * u + v * v))
        F = np.array([ru, ru * u + p, ru * v, u * (E + p)])
        Gf = np.array([rv, rv * u, rv * v + p, v * (E + p)])
        return n[0] * F + n[1] * Gf
    J = np.zeros((len(W), len(W)))
    for k in range(len(W)):
        e = np.zeros(len(W)); e[k] = h
        J[:, k] = (-flux(W + 2 * e) + 8 * flux(W + e) - 8 * flux(W - e) + flux(W - 2 * e)) / (12 * h)
    return J


@pytest.mark.parametrize("dim,n", [(1, (1.0, 0.0)), (2, (1.0, 0.0)), (2, (0.0, 1.0)), (2, (0.6, 0.8))])
def test_eigenvectors_diagonalise_jacobian(dim, n):
    from paper_2304_05572_gb300 import problems as P
    W = P.conservative(1.2, 0.3, -0.5 if dim == 2 else 0.0, 0.8, dim=dim)
    L, R = oracle.eigvec(dim, G, W, *n)
    np.testing.assert_allclose(L @ R, np.eye(dim + 2), atol=1e-13)
    J = _jac(dim, W, n)
    D = L @ J @ R
    np.testing.assert_allclose(D - np.diag(np.diag(D)), 0.0, atol=1e-8)
    r, u, v, p = 1.2, 0.3, (-0.5 if dim == 2 else 0.0), 0.8
    c = math.sqrt(G * p / r)
    un = u * n[0] + v * n[1]
    lams = [un - c, un] + ([un] if dim == 2 else []) + [un + c]
    np.testing.assert_allclose(np.diag(D), lams, atol=1e-8)


def test_characteristic_ao_exact_on_linear_data():
    """On linear data AO is exact per characteristic component, and projection is linear,
    so the characteristic WENO-AO face value is the exact linear value."""
    from paper_2304_05572_gb300 import problems as P
    base = P.conservative(1.0, 0.2, -0.1, 1.0)
    slope = np.array([0.05, 0.01, -0.02, 0.1])
    Qw = np.array([base + m * slope for m in range(-2, 3)])
    Qs = 0.5 * (Qw[2] + Qw[3])
    v, d = oracle.weno_ao_face(2, G, Qw, Qs, 1.0, 0.0, +1)
    np.testing.assert_allclose(v, base + 0.5 * slope, atol=1e-13)
    np.testing.assert_allclose(d, slope, atol=1e-12)
