"""Scheme-level pins of the oracle: the paper's printed accuracy tables (Sec. 3.1,
Tables 1-2; Sec. 3.3, Table 4), convergence orders, free-stream preservation,
conservation on periodic domains, mirror symmetry, the exact Riemann solution
for the Sod tube, hybrid == linear when nothing is flagged, robustness on the
blast wave, and the boundary and time-step rules."""
import math
import os

import numpy as np
import pytest

import exact_riemann as ER
import oracle
from paper_2304_05572_gb300 import problems as P

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    rows = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows[int(parts[0].split("/")[1])] = np.array([float(v) for v in parts[1:4]])
    return rows


def _norms(e):
    e = np.asarray(e).ravel()
    return np.array([np.mean(np.abs(e)), math.sqrt(np.mean(e * e)), np.max(np.abs(e))])


def _sine1d(inv_h, mode):
    n = 2 * inv_h
    cfg, W, t_end = P.sine_1d(n, recon_mode=mode)
    W2, t, steps, _ = oracle.run(cfg, W, t_end, threads=1)
    return _norms(W2[0, 0] - P.sine_1d_exact(n, t)), W2


# tolerances on the relative mismatch with the printed tables, per mesh (coarse meshes
# amplify the unpublished choices: gamma_Hi, gamma_Lo, error-norm conventions)
TOL1 = {5: 0.03, 10: 0.02, 20: 0.005, 40: 0.0015, 80: 0.0025}


@pytest.mark.parametrize("inv_h", [5, 10, 20, 40, 80])
def test_sine1d_reproduces_table1_wenoao(inv_h):
    ref = _golden("table1_sine1d_wenoao.txt")[inv_h]
    err, _ = _sine1d(inv_h, "wenoao")
    np.testing.assert_array_less(np.abs(err / ref - 1.0), TOL1[inv_h])


@pytest.mark.parametrize("inv_h", [5, 10, 20, 40, 80])
def test_sine1d_hybrid_matches_table2(inv_h):
    """Soft pin: no cell of the smooth sine is troubled (Steps 1-3), so the hybrid run is the
    linear-upwind run; Table 2 lies within 2.5% of it on every mesh."""
    ref = _golden("table2_sine1d_hybrid.txt")[inv_h]
    err, _ = _sine1d(inv_h, "hybrid")
    np.testing.assert_array_less(np.abs(err / ref - 1.0), 0.03)


@pytest.mark.parametrize("inv_h", [10, 20])
def test_sine1d_wenoao_over_linear_ratio_matches_tables(inv_h):
    """The smooth sine flags no cell, so Table 2 is the linear-upwind run and the
    Table 1 / Table 2 ratio isolates what the nonlinear weights of Eq. (37) do.  With
    delta/(beta_k + eps) squared and gamma_Hi = gamma_Lo = 0.85 the oracle's
    WENO-AO / linear ratio matches the printed one (L1 and Linf to 1% of its deviation from 1)."""
    t1 = _golden("table1_sine1d_wenoao.txt")[inv_h]
    t2 = _golden("table2_sine1d_hybrid.txt")[inv_h]
    e_ao, _ = _sine1d(inv_h, "wenoao")
    e_lin, _ = _sine1d(inv_h, "linear")
    paper = t1 / t2 - 1.0
    ours = e_ao / e_lin - 1.0
    np.testing.assert_allclose(ours[[0, 2]], paper[[0, 2]], rtol=0.01)   # L1, Linf
    np.testing.assert_allclose(ours[1], paper[1], rtol=0.05)             # L2 (definition unprinted)


def test_sine1d_fifth_order_and_hybrid_equals_linear():
    errs = []
    for inv_h in (10, 20, 40):
        e_h, W_h = _sine1d(inv_h, "hybrid")
        e_l, W_l = _sine1d(inv_h, "linear")
        assert np.array_equal(W_h, W_l)          # nothing flagged -> identical bits
        errs.append(e_h)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 4.85


def test_sine1d_no_flags_and_wenoao_all_flags():
    cfg, W, _ = P.sine_1d(20)
    _, _, fl = oracle.step_flags(cfg, W)
    assert fl[(0, 0, "normal")].sum() == 0 and fl[(1, 0, "normal")].sum() == 0
    cfg["recon_mode"] = "wenoao"
    _, _, fl = oracle.step_flags(cfg, W)
    assert fl[(0, 0, "normal")].all() and fl[(1, 0, "normal")].all()


@pytest.mark.parametrize("inv_h", [5, 10])
def test_sine2d_wenoao_matches_table4(inv_h):
    """Sec. 3.3 reads no end time; with t = 2 (as in Sec. 3.1) the errors lie within 5% of Table 4."""
    n = 2 * inv_h
    cfg, W, t_end = P.sine_2d(n, recon_mode="wenoao")
    W2, t, _, _ = oracle.run(cfg, W, t_end)
    err = _norms(W2[0] - P.sine_2d_exact(n, t))
    ref = _golden("table4_sine2d_wenoao.txt")[inv_h]
    np.testing.assert_array_less(np.abs(err / ref - 1.0), 0.05)


def test_sine2d_fifth_order():
    errs = []
    for n in (10, 20):
        cfg, W, t_end = P.sine_2d(n)
        W2, t, _, _ = oracle.run(cfg, W, t_end)
        errs.append(_norms(W2[0] - P.sine_2d_exact(n, t)))
    assert np.log2(errs[0] / errs[1]).min() > 4.8


@pytest.mark.parametrize("bc", ["periodic", "extrap", "reflect", "noslip"])
def test_free_stream_preserved_bitwise(bc):
    state = (1.3, 0.4, -0.7, 2.1) if bc in ("periodic", "extrap") else (1.3, 0.0, 0.0, 2.1)
    cfg, W, _ = P.uniform_2d(12, state=state, bc=bc, ny=9)
    W2, _, steps, _ = oracle.run(cfg, W, 10.0, max_steps=3)
    assert steps == 3
    assert np.array_equal(W2, W)


def test_free_stream_preserved_1d():
    cfg, W, _ = P.sod_1d(40)
    W[:] = W[:, :, :1]
    W2, _, _, _ = oracle.run(cfg, W, 10.0, max_steps=3)
    assert np.array_equal(W2, W)


def test_conservation_periodic_2d():
    cfg, W, _ = P.riemann4_2d(24)
    cfg["bc"] = ["periodic"] * 4
    s0 = W.sum(axis=(1, 2))
    W2, _, steps, _ = oracle.run(cfg, W, 10.0, max_steps=4)
    s1 = W2.sum(axis=(1, 2))
    assert np.all(np.abs(s1 - s0) <= 1e-13 * np.abs(W).sum() * steps)


def test_conservation_periodic_1d():
    cfg, W, _ = P.sod_1d(64)
    cfg["bc"] = ["periodic"] * 4
    s0 = W.sum(axis=(1, 2))
    W2, _, steps, _ = oracle.run(cfg, W, 10.0, max_steps=10)
    assert np.all(np.abs(W2.sum(axis=(1, 2)) - s0) <= 1e-13 * np.abs(W).sum() * steps)


def test_sod_mirror_symmetry():
    cfg, W, t_end = P.sod_1d(100)
    Wm = W[:, :, ::-1].copy()
    Wm[1] = -Wm[1]
    A, _, _, _ = oracle.run(cfg, W, t_end)
    B, _, _, _ = oracle.run(cfg, Wm, t_end)
    Bm = B[:, :, ::-1].copy()
    Bm[1] = -Bm[1]
    assert np.max(np.abs(A - Bm)) <= 1e-12 * np.max(np.abs(A))


def test_riemann2d_diagonal_symmetry():
    """Quadrant data symmetric under x <-> y with u <-> v stays symmetric."""
    st = [(1.0, 0.2, 0.2, 1.0), (0.5, 0.1, -0.3, 0.6), (0.8, -0.4, -0.4, 0.9), (0.5, -0.3, 0.1, 0.6)]
    cfg = P.base_config(2, 20, 20, 0, 1, 0, 1, bc=["extrap"] * 4)
    W = P._quadrants(20, 20, st)
    np.testing.assert_allclose(W[0], W[0].T, atol=1e-15)
    W2, _, _, _ = oracle.run(cfg, W, 1.0, max_steps=5)
    np.testing.assert_allclose(W2[0], W2[0].T, atol=1e-13)
    np.testing.assert_allclose(W2[1], W2[2].T, atol=1e-13)
    np.testing.assert_allclose(W2[3], W2[3].T, atol=1e-13)


def test_sod_against_exact_riemann_solution():
    errs = []
    for n in (100, 200):
        cfg, W, t_end = P.sod_1d(n)
        W2, t, _, _ = oracle.run(cfg, W, t_end)
        ex = ER.cell_averages((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, t, np.linspace(0, 1, n + 1))
        errs.append(np.mean(np.abs(W2[0, 0] - ex[0])))
    assert errs[1] < 2.5e-3
    assert errs[0] / errs[1] > 1.5            # first-order convergence at the discontinuities


def test_sod_hybrid_flags_only_near_waves():
    cfg, W, t_end = P.sod_1d(200)
    W2, _, _, _ = oracle.run(cfg, W, t_end)
    _, _, fl = oracle.step_flags(cfg, W2)
    f = fl[(0, 0, "normal")][0, 1:-1].astype(bool)
    assert 0.02 < f.mean() < 0.3
    assert not f[:40].any()       # undisturbed left state (x < 0.2)


def test_blast_wave_robust():
    cfg, W, t_end = P.blast_1d(200)
    W2, t, steps, _ = oracle.run(cfg, W, t_end)
    assert abs(t - t_end) < 1e-12
    assert np.all(W2[0] > 0)


def test_spreading_step4():
    """A single raw-troubled cell flags itself and both neighbours (Step 4)."""
    n = 40
    cfg = P.base_config(1, n, 1, 0.0, 1.0, bc=["extrap"] * 4)
    rho = np.ones(n)
    rho[20:] = 0.5
    W = P.conservative(rho, np.zeros(n), 0 * rho, np.ones(n), dim=1)[:, None, :]
    _, _, fl = oracle.step_flags(cfg, np.ascontiguousarray(W))
    f = fl[(0, 0, "normal")][0]          # cells -1..n
    Z1 = oracle.zeta1_scaled("B", 1.0 / n)
    raw = []
    for i in range(-2, n + 2):
        q = [rho[min(max(k, 0), n - 1)] for k in range(i - 2, i + 3)]
        raw.append(oracle.indicator(np.array(q), Z1))
    raw = np.array(raw)
    expect = raw[:-2] | raw[1:-1] | raw[2:]
    assert np.array_equal(f, expect.astype(np.uint8))
    assert f.sum() >= 3


def test_ghost_fill_rules():
    cfg, W, _ = P.random_smooth_2d(6, 5)
    NG = oracle.NG
    cfg["bc"] = ["periodic", "extrap", "reflect", "noslip"]
    Wp = oracle.fill_ghosts(cfg, W)
    nx, ny = 6, 5
    I = lambda i: i + NG
    J = lambda j: j + NG
    for l in range(1, NG + 1):
        np.testing.assert_array_equal(Wp[:, J(0):J(ny), I(-l)], W[:, :, nx - l])            # periodic x-lo
        np.testing.assert_array_equal(Wp[:, J(0):J(ny), I(nx - 1 + l)], W[:, :, nx - 1])    # extrap x-hi
        m = W[:, l - 1, :].copy(); m[2] = -m[2]                                              # reflect y-lo
        np.testing.assert_array_equal(Wp[:, J(-l), I(0):I(nx)], m)
        m = W[:, ny - l, :].copy(); m[1] = -m[1]; m[2] = -m[2]                               # no-slip y-hi
        np.testing.assert_array_equal(Wp[:, J(ny - 1 + l), I(0):I(nx)], m)


def test_cfl_time_step_rule():
    cfg, W, _ = P.riemann4_2d(16)
    r = W[0]; u = W[1] / r; v = W[2] / r
    p = 0.4 * (W[3] - 0.5 * r * (u * u + v * v))
    a = np.sqrt(1.4 * p / r)
    h = 1.0 / 16
    assert oracle.cfl_dt(cfg, W) == pytest.approx(0.5 * np.min(h / (np.sqrt(u * u + v * v) + a)), rel=1e-14)
    cfg2, W2, _ = P.viscous_shock_tube(16, 8, Re=50.0)
    r = W2[0]; u = W2[1] / r; v = W2[2] / r
    p = 0.4 * (W2[3] - 0.5 * r * (u * u + v * v))
    a = np.sqrt(1.4 * p / r)
    h = 1.0 / 16
    nu = (1 / 50.0) / r
    expect = 0.3 * np.min(np.minimum(h / (np.sqrt(u * u + v * v) + a), h * h / (4 * nu)))
    assert oracle.cfl_dt(cfg2, W2) == pytest.approx(expect, rel=1e-14)


def test_viscous_shock_tube_runs():
    cfg, W, _ = P.viscous_shock_tube(40, 20, Re=200.0)
    W2, t, steps, _ = oracle.run(cfg, W, 1.0, max_steps=5)
    assert steps == 5 and np.all(np.isfinite(W2)) and np.all(W2[0] > 0)
    # a no-slip mirror (both velocities negated, y kept) is not a symmetry of the BGK
    # equation once tangential gradients exist, so the wall mass flux is only nearly zero
    assert abs(W2[0].sum() - W[0].sum()) <= 1e-5 * W[0].sum()
    cfg["bc"] = ["reflect"] * 4           # slip walls: exact mirror symmetry -> no wall flux
    W3, _, _, _ = oracle.run(cfg, W, 1.0, max_steps=5)
    assert abs(W3[0].sum() - W[0].sum()) <= 1e-13 * W[0].sum()


def test_t_end_is_hit_exactly():
    cfg, W, _ = P.sod_1d(50)
    W2, t, steps, last = oracle.run(cfg, W, 0.0123)
    assert t == pytest.approx(0.0123, abs=1e-15) and last > 0


# ---------------------------------------------------------------- double Mach reflection (Sec. 3.5)

def _rh_residuals(post, pre, normal, speed, gamma=1.4):
    """Rankine-Hugoniot residuals (relative) of a shock moving at `speed` along `normal`."""
    def fluxes(state):
        rho, u, v, p = state
        un = u * normal[0] + v * normal[1]
        ut = -u * normal[1] + v * normal[0]
        E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
        w = un - speed
        return np.array([rho * w, rho * un * w + p, rho * ut * w, E * w + p * un])
    a, b = fluxes(post), fluxes(pre)
    return np.abs(a - b) / np.maximum(np.abs(a), np.abs(b))


def test_double_mach_states_satisfy_rankine_hugoniot():
    """The printed post-/pre-shock states are the exact Mach 10 shock at 60 deg (the line
    x = 1/6 + (y + 20 t)/sqrt(3) moves at 10 along its normal (sin 60, -cos 60))."""
    cot = P.DMR_COT
    sin = 1.0 / np.sqrt(1.0 + cot * cot)
    normal = (sin, -cot * sin)
    speed = P.DMR_SPEED * cot * sin
    assert speed == pytest.approx(10.0, rel=1e-15)
    res = _rh_residuals(P.DMR_POST, P.DMR_PRE, normal, speed)
    assert np.all(res[[0, 1, 3]] <= 1e-13), res
    assert abs(P.DMR_POST[0] * (P.DMR_POST[1] * -normal[1] + P.DMR_POST[2] * normal[0])) <= 1e-13   # no tangential jump
    # Mach number of the normal shock in the pre-shock gas
    assert speed / np.sqrt(1.4 * P.DMR_PRE[3] / P.DMR_PRE[0]) == pytest.approx(10.0, rel=1e-15)


def _crossings(rho, x1):
    """x where each row first drops through the mid density (linear interpolation between centres)."""
    nx = rho.shape[1]
    dx = x1 / nx
    mid = 0.5 * (P.DMR_POST[0] + P.DMR_PRE[0])
    out = []
    for row in rho:
        k = int(np.argmax(row < mid))
        f = (row[k - 1] - mid) / (row[k - 1] - row[k])
        out.append((k - 0.5 + f) * dx)
    return np.array(out)


def test_oblique_shock_travels_at_the_exact_speed():
    """With inflow behind, the y-sides following the exact motion and a non-reflecting end,
    the captured Mach 10 shock stays on the exact line in every row, including the rows next
    to the moving boundaries (a boundary that lags the motion drags its rows behind)."""
    n = 64
    cfg, W = P.oblique_shock(n, n // 2)
    Wo, t, steps, _ = oracle.run(cfg, W, 0.02)
    assert steps > 10 and t == 0.02
    yc = (np.arange(n // 2) + 0.5) * (0.5 / (n // 2))
    exact = P.DMR_X0 + P.DMR_COT * (yc + P.DMR_SPEED * t)
    got = _crossings(Wo[0], 1.0)
    assert np.max(np.abs(got - exact)) <= 1.0 / n, np.abs(got - exact).max() * n
    # planting a frozen boundary (the line not moving with time) moves the boundary rows
    frozen = dict(cfg, shock_speed=0.0)
    Wf, _, _, _ = oracle.run(frozen, W, 0.02)
    bad = np.abs(_crossings(Wf[0], 1.0) - exact)
    assert max(bad[0], bad[-1]) > 2.0 / n


def test_double_mach_robust_and_quiet_ahead_of_the_shock():
    """The full problem runs to a later time at CFL 0.8 with positive density and pressure,
    and the gas at rest more than 8 cells ahead of the shock stays at rest to 1e-8 (only the
    high-order stencils' far tails reach it)."""
    nx, ny = 96, 24
    cfg, W, _ = P.double_mach(nx, ny)
    Wo, t, steps, _ = oracle.run(cfg, W, 0.05)
    assert t == 0.05
    rho = Wo[0]
    p = 0.4 * (Wo[3] - 0.5 * (Wo[1] ** 2 + Wo[2] ** 2) / rho)
    assert rho.min() > 0 and p.min() > 0
    xc = (np.arange(nx) + 0.5) * (4.0 / nx)
    yc = (np.arange(ny) + 0.5) * (1.0 / ny)
    ahead = xc[None, :] > P.DMR_X0 + P.DMR_COT * (yc[:, None] + P.DMR_SPEED * t) + 8 * (4.0 / nx)
    pre = P.conservative(*P.DMR_PRE)
    scale = np.abs(pre).max()
    for k in range(4):
        assert np.max(np.abs(Wo[k][ahead] - pre[k])) <= 1e-8 * scale
    assert ahead.sum() > nx * ny // 4


def test_prescribed_boundary_ghosts():
    """Inflow ghosts hold the prescribed state; the shock wall is the prescribed state up to
    x = 1/6 and a slip wall beyond; the tracking boundary switches at the shock line."""
    nx, ny = 24, 6
    cfg, W, _ = P.double_mach(nx, ny)
    NG = oracle.NG
    t = 0.03
    Wp = oracle.fill_ghosts(cfg, W, t)
    post, pre = P.conservative(*P.DMR_POST), P.conservative(*P.DMR_PRE)
    dx, dy = 4.0 / nx, 1.0 / ny
    for l in range(1, NG + 1):
        np.testing.assert_array_equal(Wp[:, NG:NG + ny, NG - l], np.repeat(post[:, None], ny, axis=1))
        for i in range(-NG, nx + NG):
            xc = (i + 0.5) * dx
            g = Wp[:, NG - l, NG + i]
            if xc < P.DMR_X0:
                np.testing.assert_array_equal(g, post)
            elif 0 <= i < nx:
                m = W[:, l - 1, i].copy(); m[2] = -m[2]
                np.testing.assert_array_equal(g, m)
            yc = (ny - 1 + l + 0.5) * dy
            behind = xc < P.DMR_X0 + P.DMR_COT * (yc + P.DMR_SPEED * t)
            np.testing.assert_array_equal(Wp[:, NG + ny - 1 + l, NG + i], post if behind else pre)


# ---------------------------------------------------------------- S2O4 time integration (Sec. 2.2)

@pytest.mark.parametrize("dim", [1, 2])
def test_s2o4_advects_a_quartic_exactly(dim):
    from exact_cases import quartic_advection
    """Two-stage fourth-order step with tau = 0 on a quartic density advected at constant
    velocity and pressure: the reconstruction is exact for quartics, the tau = 0 flux is the
    exact second-order time expansion at the interface, and S2O4 reproduces the Taylor series
    to fourth order, which for a quartic is the exact solution.  Away from the (non-reflecting)
    ends the step is exact to round-off, while the fourth-order term alone is ~1e-9..1e-8."""
    n = 64 if dim == 1 else 40
    cfg, W, exact, dt = quartic_advection(dim, n, 0.9)
    Wo, _, steps, _ = oracle.run(cfg, W, 1.0, max_steps=1)
    assert steps == 1
    inner = (slice(None), slice(12, n - 12)) if dim == 1 else (slice(12, n - 12), slice(12, n - 12))
    for k in range(W.shape[0]):
        scale = np.abs(exact[k]).max()
        assert np.abs(Wo[k][inner] - exact[k][inner]).max() <= 2e-15 * max(scale, 1.0) * 10
    fourth = (0.7 + 0.4) ** 4 * dt ** 4 * 30.0 / (4 * 3 * 2) * 24
    assert fourth > 1e-9


def test_hybrid_equals_wenoao_when_every_cell_is_troubled():
    """The converse of hybrid = linear on smooth data: when the indicator flags every cell
    (alternating two-level data), the hybrid step is the WENO-AO step, bit for bit."""
    from exact_cases import all_troubled_1d
    cfg, W = all_troubled_1d()
    Wh, dt, fl = oracle.step_flags(cfg, W)
    assert all(np.all(f == 1) for f in fl.values())
    Wa, dta, _ = oracle.step_flags(dict(cfg, recon_mode="wenoao"), W)
    Wl, _, _ = oracle.step_flags(dict(cfg, recon_mode="linear"), W)
    assert dt == dta and np.array_equal(Wh, Wa)
    assert not np.array_equal(Wh, Wl)
