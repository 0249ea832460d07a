"""Pins of the oracle's global rate laws (Sec. 7.1, Eqs. 26-30): real reaction
orders (Eq. 28: C_CH4^0.5 C_O2^0.65) and non-integer stoichiometry (Eq. 26:
1.5 O2; Eq. 27: 0.5 O2).

- an irreversible A -> B of order a has the closed form
  C^(1-a) = C0^(1-a) - (1-a) k t, which forward Euler approaches at first
  order (pins the exponent of every concentration);
- real stoichiometry still conserves mass and elements over whole solves of
  the BFER mechanism;
- COROX (dN = -1/2): the composition with sum nu mu = 0, from chemical
  potentials written here, has zero net rate (pins K of Eq. 30 with a
  half-integer dN and the 0.5 order of O2 in the forward rate)."""
import copy

import numpy as np
import pytest

import oracle
from paper_1905_09395_b300 import synth
from mechs import P_ATM, R_U, constant_cp_block, tiny_mechanism
from test_oracle_physics import _equilibrium_mix, _mu_over_rt


def _decay(order, A):
    # A -> B, same W and constant cp, same enthalpy: T and rho stay constant
    W = 0.028
    blk = constant_cp_block(3.5, a6=-1000.0, a7=0.0)
    m = tiny_mechanism([W, W], [blk, blk], [{0: -1, 1: 1}], A=[A], reversible=[0])
    m.rxn_order = np.array([order, 1.0])
    return m, W


@pytest.mark.parametrize("order,A", [(0.5, 2120.0), (1.5, 300.0)])
def test_real_order_decay_closed_form(order, A):
    m, W = _decay(order, A)
    T, P, t_f = 1200.0, P_ATM, 1e-3
    rho = P * W / (R_U * T)
    Y0 = np.array([0.9, 0.1])
    C0 = rho * Y0[0] / W
    exact_C = (C0 ** (1 - order) - (1 - order) * A * t_f) ** (1 / (1 - order))
    exact = exact_C * W / rho
    assert 0.2 < exact / Y0[0] < 0.8                   # well inside the decay
    errs = []
    for delta in (0.01, 0.001):
        tr = oracle.solve_cell_trace(m, T, P, Y0, t_f, alpha=0.0, y_step_max=1.0,
                                     delta_max=delta, dft_on=0)
        assert tr["status"] == oracle.CELL_OK and tr["T"] == T
        errs.append(abs(tr["Y"][0] - exact))
        assert tr["Y"].sum() == pytest.approx(1.0, abs=1e-14)
    assert errs[1] < 2e-3 * exact
    assert errs[0] / errs[1] == pytest.approx(10.0, rel=0.1)   # first order in h


def test_real_stoichiometry_conserves_mass_and_elements():
    mech = synth.bfer_mechanism()
    T, P, Y = synth.bfer_cells(mech, 32)
    To, Yo, it, st = oracle.solve(mech, T, P, Y, 1e-3)
    assert (st == oracle.CELL_OK).all()
    assert To.mean() > T.mean() + 100.0                 # methane burns
    np.testing.assert_allclose(Yo.sum(axis=1), Y.sum(axis=1), rtol=0, atol=2e-12)
    e0 = (Y / mech.mol_weight) @ mech.elements
    e1 = (Yo / mech.mol_weight) @ mech.elements
    assert np.all(np.abs(e1 - e0) <= 2e-11 * np.abs(e0).max(axis=1, keepdims=True))


def _corox_only():
    m = copy.deepcopy(synth.bfer_mechanism())
    k0, k1 = int(m.rxn_ptr[1]), int(m.rxn_ptr[2])
    m.rxn_species = m.rxn_species[k0:k1].copy()
    m.rxn_nu = m.rxn_nu[k0:k1].copy()
    m.rxn_order = m.rxn_order[k0:k1].copy()
    m.rxn_ptr = np.array([0, k1 - k0], dtype=np.int32)
    for f in ("A", "beta", "Ea", "reversible"):
        setattr(m, f, getattr(m, f)[1:2].copy())
    return m


@pytest.mark.parametrize("T,P", [(1200.0, P_ATM), (2000.0, 3 * P_ATM), (2800.0, 0.5 * P_ATM)])
def test_half_stoichiometry_equilibrium(T, P):
    m = _corox_only()
    CO, O2, CO2, N2 = 2, 1, 4, 5
    rx = {CO: -1.0, O2: -0.5, CO2: 1.0}
    x, Y = _equilibrium_mix(m, T, P, rx, {O2: 0.1, CO2: 0.1}, inert=N2)   # solve for CO
    mu = _mu_over_rt(m, T, P, np.where(x > 0, x, 1.0))
    assert abs(sum(nu * mu[s] for s, nu in rx.items())) < 1e-12
    q_eq = oracle.rates(m, T, P, Y, alpha=0.0)["qraw"][0]
    Yp = Y.copy()
    Yp[CO2] *= 1.01
    q_off = oracle.rates(m, T, P, Yp, alpha=0.0)["qraw"][0]
    assert q_off != 0.0
    assert abs(q_eq) <= 1e-9 * abs(q_off)
