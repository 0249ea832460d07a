"""Pins of the oracle's right-hand side and integrator against physics.

- mass (sum dY/dt = 0) and element conservation: every reaction is balanced;
- energy: adiabatic constant-pressure means total enthalpy is constant,
  d/dt sum_i Y_i H_i/W_i + cp dT/dt = 0 (pins the temperature equation);
- chemical equilibrium: the composition with sum_i nu_i mu_i = 0,
  mu_i/RT = G_i/RT + ln(x_i P/P0), has zero net rate (pins K of Eq. 30, its
  dN term and the 1 atm standard state), and long integrations end there;
- Eqs. 6-7: gamma -> 1 for y >> alpha, rate ~ y^2/alpha for y << alpha;
- an isomerisation A<=>B has a closed form, exact for forward Euler
  (Eq. 18) step by step and first-order close to the exact exponential.
"""
import numpy as np
import pytest

import oracle
from paper_1905_09395_b300 import synth
from mechs import P_ATM, R_U, constant_cp_block, isomer_pair, tiny_mechanism


@pytest.fixture(scope="module")
def scale():
    mech = synth.scale_mechanism()
    T, P, Y = synth.make_cells(mech, 16, seed=5, T_range=(800, 2200), P_atm_range=(1, 5),
                               dirichlet=0.5)
    return mech, T, P, Y


def test_mass_fraction_rates_sum_to_zero(scale):
    mech, T, P, Y = scale
    for c in range(16):
        r = oracle.rates(mech, T[c], P[c], Y[c])
        d = r["dYdt"]
        assert abs(d.sum()) <= 1e-13 * np.abs(d).sum()


def test_enthalpy_is_conserved_by_the_rhs(scale):
    mech, T, P, Y = scale
    W = mech.mol_weight
    for c in range(16):
        r = oracle.rates(mech, T[c], P[c], Y[c])
        cpR, hRT, _ = oracle.thermo(mech, T[c])
        H = hRT * R_U * T[c]                            # J/mol
        cp = R_U * np.sum(Y[c] * cpR / W)               # J/(kg K)
        terms = H / W * r["dYdt"]
        total = terms.sum() + cp * r["dTdt"]
        assert abs(total) <= 1e-11 * (np.abs(terms).sum() + abs(cp * r["dTdt"]))
        assert r["dTdt"] != 0.0


def _element_totals(mech, Y):
    return (Y / mech.mol_weight) @ mech.elements


def test_mass_and_elements_conserved_over_solve():
    mech, T, P, Y, dt = synth.small_case(32)
    To, Yo, it, st = oracle.solve(mech, T, P, Y, dt)
    assert (st == oracle.CELL_OK).all()
    np.testing.assert_allclose(Yo.sum(axis=1), Y.sum(axis=1), rtol=0, atol=2e-12)
    e0, e1 = _element_totals(mech, Y), _element_totals(mech, Yo)
    scale_ = np.abs(e0).max(axis=1, keepdims=True)
    assert np.all(np.abs(e1 - e0) <= 2e-11 * scale_)


def _mu_over_rt(mech, T, P, x):
    cpR, hRT, sR = oracle.thermo(mech, T)
    return hRT - sR + np.log(x * P / P_ATM)


def _equilibrium_mix(mech, T, P, reaction, x_known, inert):
    """Solve sum nu mu = 0 for the one unknown product species (a log-linear
    equation), fill the rest with an inert species."""
    cpR, hRT, sR = oracle.thermo(mech, T)
    g = hRT - sR
    x = dict(x_known)
    unknown = [s for s in reaction if s not in x]
    assert len(unknown) == 1
    u = unknown[0]
    acc = sum(nu * (g[s] + np.log(x[s] * P / P_ATM)) for s, nu in reaction.items() if s != u)
    nu_u = reaction[u]
    x[u] = np.exp((-acc / nu_u) - g[u]) * P_ATM / P
    x[inert] = 1.0 - sum(x.values())
    assert x[inert] > 0
    xs = np.array([x.get(i, 0.0) for i in range(len(mech.mol_weight))])
    Y = xs * mech.mol_weight / np.sum(xs * mech.mol_weight)
    return xs, Y


def _abc_mech():
    # A + B <=> C (dN = -1); D inert.  a7 of C puts dG/RT near 0 at 1400 K,
    # so K ~ RT/P0 and neither direction is stiff (forward Euler stays stable
    # at h = delta t_f, k ~ 1.4e2/s)
    WA, WB = 0.016, 0.032
    blocks = [constant_cp_block(3.5, a6=-2000.0, a7=4.0),
              constant_cp_block(3.8, a6=1000.0, a7=6.0),
              constant_cp_block(5.1, a6=-1000.0, a7=23.7),
              constant_cp_block(3.5, a6=0.0, a7=5.0)]
    rx = [{0: -1, 1: -1, 2: 1}]
    return tiny_mechanism([WA, WB, WA + WB, 0.028], blocks, rx, A=[1.0], beta=[0.3], Ea=[2e3])


@pytest.mark.parametrize("T,P", [(900.0, P_ATM), (1500.0, 3 * P_ATM), (2600.0, 0.5 * P_ATM)])
def test_equilibrium_composition_has_zero_net_rate(T, P):
    m = _abc_mech()
    rx = {0: -1, 1: -1, 2: 1}
    x, Y = _equilibrium_mix(m, T, P, rx, {0: 0.2, 1: 0.1}, inert=3)
    mu = _mu_over_rt(m, T, P, x)
    assert abs(sum(nu * mu[s] for s, nu in rx.items())) < 1e-12
    q_eq = oracle.rates(m, T, P, Y, alpha=0.0)["qraw"][0]
    Yp = Y.copy()
    Yp[2] *= 1.01
    q_off = oracle.rates(m, T, P, Yp, alpha=0.0)["qraw"][0]
    assert q_off != 0.0
    assert abs(q_eq) <= 1e-9 * abs(q_off)
    # the other direction (dN = +1) must give the same equilibrium
    m2 = _abc_mech()
    m2.rxn_nu = -m2.rxn_nu
    q_eq2 = oracle.rates(m2, T, P, Y, alpha=0.0)["qraw"][0]
    q_off2 = oracle.rates(m2, T, P, Yp, alpha=0.0)["qraw"][0]
    assert abs(q_eq2) <= 1e-9 * abs(q_off2)


@pytest.mark.parametrize("dft_on", [0, 1])
def test_long_integration_reaches_chemical_equilibrium(dft_on):
    # the fixed point of forward Euler is f(Y, T) = 0 exactly, so a long
    # stable integration ends at the chemical equilibrium of its final T
    m = _abc_mech()
    x0 = np.array([0.3, 0.3, 0.1, 0.3])
    Y0 = x0 * m.mol_weight / np.sum(x0 * m.mol_weight)
    T0, P = 1400.0, 2 * P_ATM
    res = oracle.solve_cell_trace(m, T0, P, Y0, 0.5, trace_cap=1, alpha=0.0, dft_on=dft_on)
    assert res["status"] == oracle.CELL_OK
    Y, T = res["Y"], res["T"]
    x = (Y / m.mol_weight) / np.sum(Y / m.mol_weight)
    mu = _mu_over_rt(m, T, P, x)
    assert abs(mu[2] - mu[0] - mu[1]) < 1e-9

    # the enthalpy is conserved along the way (first order in h)
    def H(Yv, Tv):
        return np.sum(Yv / m.mol_weight * oracle.thermo(m, Tv)[1] * R_U * Tv)
    assert abs(H(Y, T) - H(Y0, T0)) < 1e-3 * abs(H(Y0, T0))


def test_gamma_limits():
    # irreversible A -> B; rate of progress is kf * C_A**
    m = tiny_mechanism([0.03, 0.03], [constant_cp_block(3.5), constant_cp_block(3.5)],
                       [{0: -1, 1: 1}], A=[10.0], reversible=[0])
    T, P = 1000.0, P_ATM
    big = np.array([0.4, 0.6])
    q0 = oracle.rates(m, T, P, big, alpha=0.0)["qraw"][0]
    q1 = oracle.rates(m, T, P, big, alpha=1e-5)["qraw"][0]
    assert q1 == pytest.approx(q0 * 0.4 / (0.4 + 1e-5), rel=1e-14)   # gamma ~ 1
    tiny1 = np.array([1e-10, 1 - 1e-10])
    tiny2 = np.array([2e-10, 1 - 2e-10])
    r1 = oracle.rates(m, T, P, tiny1, alpha=1e-5)["qraw"][0]
    r2 = oracle.rates(m, T, P, tiny2, alpha=1e-5)["qraw"][0]
    assert r2 / r1 == pytest.approx(4.0, rel=1e-4)                    # ~ y^2/alpha
    plain = oracle.rates(m, T, P, tiny1, alpha=0.0)["qraw"][0]
    assert r1 < 2e-5 * plain                                           # gamma ~ 0
    # negative mass fractions do not react (max(Y, 0))
    assert oracle.rates(m, T, P, np.array([-1e-12, 1.0]), alpha=1e-5)["qraw"][0] == 0.0


def test_isomerisation_discrete_closed_form():
    # A <=> B, same W and H: T stays constant and dY_A/dt = -kf Y_A + kr Y_B,
    # so forward Euler gives Y_A,n = Y_eq + (Y_A0 - Y_eq) prod_j (1 - k h_j)
    K, A = 3.0, 1.0e3
    m = isomer_pair(A=A, K=K)
    kf, kr = A, A / K
    k = kf + kr
    Y0 = np.array([0.9, 0.1])
    Yeq = kr * Y0.sum() / k
    for dft_on in (0, 1):
        tr = oracle.solve_cell_trace(m, 1200.0, P_ATM, Y0, 1e-3, alpha=0.0, y_step_max=1.0,
                                     dft_on=dft_on)
        assert tr["status"] == oracle.CELL_OK
        assert tr["T"] == 1200.0
        h = tr["h"]
        pred = Yeq + (Y0[0] - Yeq) * np.cumprod(1.0 - k * h)
        got = np.append(tr["Y_trace"][1:, 0], tr["Y"][0])
        np.testing.assert_allclose(got, pred, rtol=1e-13, atol=0)
        assert tr["Y"].sum() == pytest.approx(1.0, abs=1e-15)


def test_isomerisation_first_order_error():
    # global error of forward Euler for y' = -k (y - y_eq):
    # (1 - kh)^n - e^{-k t} ~ -e^{-k t} k^2 h t / 2
    K, A = 3.0, 1.0e3
    m = isomer_pair(A=A, K=K)
    k = A + A / K
    Y0 = np.array([0.9, 0.1])
    Yeq = (A / K) / k
    errs = []
    for delta in (0.01, 0.001):
        tr = oracle.solve_cell_trace(m, 1200.0, P_ATM, Y0, 1e-3, alpha=0.0, y_step_max=1.0,
                                     delta_max=delta)
        exact = Yeq + (Y0[0] - Yeq) * np.exp(-k * 1e-3)
        err = tr["Y"][0] - exact
        predicted = -np.exp(-k * 1e-3) * k ** 2 * (1e-3 * delta) * 1e-3 / 2 * (Y0[0] - Yeq)
        assert err == pytest.approx(predicted, rel=0.02)
        errs.append(abs(err))
    assert errs[0] / errs[1] == pytest.approx(10.0, rel=0.02)
