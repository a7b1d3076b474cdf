"""The operation counts behind the benchmark's roofline numerator.

* The counting build of the oracle (oracle/opcount.cpp: hgks_oracle.c compiled with a
  counting stand-in for double) computes exactly what the plain oracle computes, and its
  counts agree with a count by hand of the formulas as the oracle writes them.
* The oracle's Gauss-point flux takes a fixed number of operations whatever the (physical)
  data, so per-cell-stage figures can be split into the flux and the rest.
* The closed-form flux of the CUDA library, counted on the host (flopcount.py), takes far
  fewer operations than the oracle's literal moment integration.
"""
import numpy as np
import pytest

import oracle
from oracle import opcount
from paper_2304_05572_gb300 import problems as P

W_L, W_LX, W_LY = [1.0, 0.1, 0.2, 2.5], [0.1, 0.05, -0.02, 0.3], [-0.05, 0.01, 0.03, -0.1]
W_R, W_RX, W_RY = [0.8, -0.1, 0.05, 2.0], [0.1, 0.05, -0.02, 0.3], [-0.05, 0.01, 0.03, -0.1]


def test_counting_build_computes_the_oracle_bits():
    import ctypes
    cfg, W, _ = P.riemann4_2d(24, ny=20)
    Wo, _, n, _ = oracle.run(cfg, W, 1e9, max_steps=2, threads=1)
    c = oracle.make_config(cfg, 1)
    Wc = np.ascontiguousarray(W, dtype=np.float64).copy()
    t, k, ld = ctypes.c_double(0.0), ctypes.c_int(0), ctypes.c_double(0.0)
    L = opcount.lib()
    assert L.or_run(ctypes.byref(c), oracle._dp(Wc), ctypes.byref(t), 1e9, 2, ctypes.byref(k), ctypes.byref(ld)) == 0
    assert k.value == n == 2
    assert np.array_equal(Wc, Wo)


def test_linear_face_count_matches_a_count_by_hand():
    """Eqs. (26)-(27) as the oracle writes them: value = (((2 q0 - 13 q1) + 47 q2 + 27 q3 - 3 q4)/60
    as one multiply, four fma and a multiply by 1/60; derivative = ((q1 - 15 q2) + 15 q3 - q4)
    times 1/(12 dx) as two fma, one subtraction and one multiply."""
    c = opcount.count_linear_face([1.0, 2.0, 3.5, 2.0, 1.5], 0.1, 0)
    assert c == {"add": 1, "mul": 3, "fma": 6, "div": 0, "sqrt": 0, "exp": 0, "erfc": 0}
    assert opcount.flop(c) == 16


def test_oracle_flux_count_does_not_depend_on_the_data():
    cfg, _, _ = P.riemann4_2d(16)
    a = opcount.count_point_flux(cfg, W_L, W_LX, W_LY, W_R, W_RX, W_RY, 1e-3)
    b = opcount.count_point_flux(cfg, [0.5, -0.3, 0.1, 1.2], [1.0, 0.0, 0.5, -0.2], [0.0, 0.2, 0.0, 0.1],
                                 [2.0, 0.4, -0.2, 6.0], [-0.3, 0.1, 0.0, 0.4], [0.1, 0.0, -0.1, 0.0], 2e-3)
    assert a == b
    assert a["exp"] >= 3 and a["erfc"] >= 2 and a["sqrt"] >= 2


def test_step_table_splits_flux_and_rest():
    tab = opcount.step_table(16, threads=1)
    assert tab["gauss_points_per_cell_stage"] == pytest.approx(4 * 17 / 16)
    for mode in ("linear", "hybrid", "wenoao"):
        m = tab[mode]
        assert m["non_flux_flop_per_cell_stage"] > 0
        assert m["flop_per_cell_stage"] == pytest.approx(
            m["non_flux_flop_per_cell_stage"] + tab["gauss_points_per_cell_stage"] * tab["oracle_flux_flop_per_gp"])
    assert tab["linear"]["non_flux_flop_per_cell_stage"] < tab["hybrid"]["non_flux_flop_per_cell_stage"] \
        < tab["wenoao"]["non_flux_flop_per_cell_stage"]


def test_closed_form_flux_count():
    from paper_2304_05572_gb300 import flopcount
    cnt = flopcount.count_flux()
    assert all(v["ok"] for v in cnt.values())
    cfg, _, _ = P.riemann4_2d(16)
    lit = opcount.flop(opcount.count_point_flux(cfg, W_L, W_LX, W_LY, W_R, W_RX, W_RY, 1e-3))
    closed = cnt["2d_euler_stage1"]["flop"]
    assert closed < lit / 3
    # tau = 0 drops every non-equilibrium term; the Prandtl fix adds the heat-flux moments
    assert cnt["2d_tau0_stage1"]["flop"] < closed < cnt["2d_ns_prfix_stage1"]["flop"]


def test_fused_gauss_point_reconstruction_count():
    """The flux kernel's share of the tangential reconstruction (the smooth passes at its own
    Gauss point) enters the flux roofline with the closed-form count 236: 24 quartic
    evaluations (16 values: 4 passes x 4 components; 8 derivatives: the Q^l, Q^r passes) of
    one multiply and four fma each (9 operations), 2 positivity tests (rho E - |m|^2/2 > 0:
    m_y^2, fma for m_x^2 + m_y^2, the half, rho E and the difference: 6) and 8 derivative
    scalings.  The oracle evaluates the same quartics from the printed formulas at
    more than twice that (its count of one window's 2 values and 2 derivatives), so, as for
    the flux, the closed form is the lower figure; the whole-step numerator takes this part
    from the oracle's count of the reconstruction and not from the flux kernel's."""
    import bench
    per_quartic = 1 + 2 * 4
    assert bench.FLUX_KERNEL_TANG_FLOP_PER_GP == (16 + 8) * per_quartic + 2 * 6 + 8 == 236
    c = opcount.count_gauss_scalar([1.0, 2.0, 3.5, 2.0, 1.5])
    assert opcount.flop(c) / 4 > 2 * per_quartic
