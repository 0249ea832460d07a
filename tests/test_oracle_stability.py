"""Sec. 4's stability analysis (Eqs. 19-25) on the oracle: the finite-
difference Jacobian pinned by closed forms, then the diagnostics reported
(not gated): Eq. 25 along STEV trajectories of the 8-species workload and the
spectral stiffness of 16 initial states of the 32-species workload."""
import numpy as np
import pytest

import oracle
from oracle import diagnostics as dg
from paper_1905_09395_b300 import synth
from mechs import P_ATM, isomer_pair


def test_isomer_jacobian_is_the_linear_rate_matrix():
    """A <=> B with equal molar masses, zero activation energy and T
    exponent, and equal enthalpies (T constant): dY_A/dt = -kf Y_A + kr Y_B,
    so the Y block of A is [[-kf, kr], [kf, -kr]] with eigenvalues 0 and
    -(kf + kr), kf = A, kr = A / K; the T column is zero (no T dependence)
    and so is the T row (no heat release)."""
    A_pre, K = 2.0e3, 3.0
    m = isomer_pair(A=A_pre, K=K)
    J = dg.jacobian_fd(m, 1500.0, P_ATM, np.array([0.7, 0.3]), alpha=0.0, dft_on=0)
    kf, kr = A_pre, A_pre / K
    np.testing.assert_allclose(J[:2, :2], [[-kf, kr], [kf, -kr]], rtol=1e-6, atol=1e-6)
    assert np.all(np.abs(J[:, 2]) < 1e-6 * kf) and np.all(np.abs(J[2, :]) < 1e-6 * kf)
    lam = np.sort(np.linalg.eigvals(J[:2, :2]).real)
    np.testing.assert_allclose(lam, [-(kf + kr), 0.0], rtol=1e-6, atol=1e-6)
    ratio, rho, ninf = dg.spectral_ratio(m, 1500.0, P_ATM, np.array([0.7, 0.3]), alpha=0.0)
    assert rho == pytest.approx(kf + kr, rel=1e-6)
    assert ninf == pytest.approx(kf + kr, rel=1e-6)   # row sums |-kf| + |kr|, |kf| + |-kr|


def test_eq25_holds_on_the_isomer_time_cap_steps():
    """With Y_step^max out of the way (1.0) the time cap binds (h = delta t_f
    = 1e-5 s; the 0.9 y candidate is ~5e-4 s), and h (kf + kr) = 0.0267 <= 2
    on every step: Eq. 25 holds everywhere."""
    m = isomer_pair(A=2.0e3, K=3.0)
    r = dg.eq25_report(m, 1500.0, P_ATM, np.array([0.7, 0.3]), 1e-3, alpha=0.0, dft_on=0,
                       y_step_max=1.0)
    assert r["steps"] == 100
    assert r["frac_eq25_inf"] == 1.0 and r["frac_eq25_rho"] == 1.0
    assert r["max_h_rho"] == pytest.approx(1e-5 * (2.0e3 + 2.0e3 / 3.0), rel=1e-5)


def test_stability_report():
    """Reported, not gated: the fraction of STEV steps inside Eq. 25's bound
    and the spectral stiffness ratio of the 32/150 workload's states."""
    mech, T, P, Y, dt = synth.small_case(4)
    for c in range(4):
        r = dg.eq25_report(mech, T[c], P[c], Y[c], dt, samples=100)
        print("8/20 cell %d: %s" % (c, r))
        assert 0.0 <= r["frac_eq25_inf"] <= 1.0
    big = synth.scale_mechanism()
    Tb, Pb, Yb = synth.make_cells(big, 16, seed=1, T_range=(800.0, 2200.0),
                                  P_atm_range=(1.0, 5.0), dirichlet=0.5)
    ratios = [dg.spectral_ratio(big, Tb[c], Pb[c], Yb[c])[0] for c in range(16)]
    print("32/150, 16 initial states: spectral stiffness ratio median %.3g, min %.3g, max %.3g"
          % (np.median(ratios), np.min(ratios), np.max(ratios)))
    assert np.all(np.isfinite(ratios))
