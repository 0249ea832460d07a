"""Pins of the multiphase oracle (Sec. 7.2, Eqs. 31-56, Table 2), each
independent of the rate laws' own formulas:

* reactions 31-41 conserve mass (with the pseudo-species' molecular weights
  read from Eqs. 31 and 37) and every element of the species with a formula;
  whole solves conserve total mass and C, H, O, N, S (Tar's and CV's
  compositions follow from Eqs. 37 and 31);
* pyrolysis alone (Eq. 42, first order in the volatile matter's partial
  density at gamma = 1) follows the discrete closed form of forward Euler,
  c_n = c_0 (1 - k h)^n, k = MW_CV A e^(-Ea/T_s), to 1e-13;
* moisture release alone (Eq. 56, first order in the solid's total mass
  through eps_s) follows u_n = u_0 (1 - kappa h)^n for the solid mass u;
* water-gas shift alone (Eq. 43, the only reversible reaction) ends at its
  equilibrium K_F X_CO X_H2O e^(-Ea_F/T_g) = K_R X_CO2 X_H2 e^(-Ea_R/T_g);
* the STEV integration converges at first order to scipy's Radau on the
  same right-hand side."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import multiphase as mp
from paper_1905_09395_b300 import synth

IDX = {s: i for i, s in enumerate(mp.SPECIES)}
AW = {"C": 12.011, "H": 1.00794, "O": 15.9994, "N": 14.0067, "S": 32.065}
FORMULA = {"O2": {"O": 2}, "CO": {"C": 1, "O": 1}, "CO2": {"C": 1, "O": 2}, "CH4": {"C": 1, "H": 4},
           "H2": {"H": 2}, "H2O": {"H": 2, "O": 1}, "H2S": {"H": 2, "S": 1},
           "C3H6": {"C": 3, "H": 6}, "HCN": {"H": 1, "C": 1, "N": 1}, "C2H4": {"C": 2, "H": 4},
           "C2H6": {"C": 2, "H": 6}, "SO3": {"S": 1, "O": 3}, "N2": {"N": 2}, "CC": {"C": 1},
           "CM": {"H": 2, "O": 1}}


def _elements():
    """Element matrix [18][5]; Tar and CV from the reactions that define them."""
    mw, nu = mp.tables()
    E = np.zeros((18, 5))
    keys = list(AW)
    for s, f in FORMULA.items():
        for e, k in f.items():
            E[IDX[s], keys.index(e)] = k
    tox = mp.REACTIONS.index("TOX")
    E[IDX["Tar"]] = sum(nu[tox][i] * E[i] for i in range(18) if i != IDX["Tar"])
    pyro = mp.REACTIONS.index("PYRO")
    E[IDX["CV"]] = sum(nu[pyro][i] * E[i] for i in range(18) if i != IDX["CV"])
    return E, np.array([AW[k] for k in keys])


def test_stoichiometry_conserves_mass_and_elements():
    mw, nu = mp.tables()
    E, aw = _elements()
    # molecular weights of the species with a formula are their atoms' sum
    for s in FORMULA:
        assert mw[IDX[s]] == pytest.approx(E[IDX[s]] @ aw, rel=1e-6)
    for k, name in enumerate(mp.REACTIONS):
        assert abs(nu[k] @ mw) <= 1e-12 * np.abs(nu[k] * mw).sum(), name
        assert np.all(np.abs(nu[k] @ E) <= 1e-12 * np.abs(nu[k][:, None] * E).sum(axis=0) + 1e-15), name
    # Tar is a C25 hydrocarbon-like pseudo-species: its mass from its atoms
    assert mw[IDX["Tar"]] == pytest.approx(E[IDX["Tar"]] @ aw, rel=1e-9)
    assert 400.0 < mw[IDX["Tar"]] < 450.0


def test_whole_solves_conserve_mass_and_elements():
    cells = synth.multiphase_cells(64, seed=1)
    out, rho_g, it, st = mp.solve(cells, 1e-3)
    assert (st == 0).all()
    mw, _ = mp.tables()
    E, _ = _elements()
    for k in range(len(cells)):
        c0 = mp.initial_densities(cells[k])
        es1 = out[k, mp.I_EPS]
        c1 = np.concatenate([(1.0 - es1) * rho_g[k] * out[k, :14],
                             es1 * cells[k, mp.I_RHOS] * out[k, 14:18]])
        assert c1.sum() == pytest.approx(c0.sum(), rel=1e-12)
        e0, e1 = (c0 / mw) @ E, (c1 / mw) @ E
        assert np.all(np.abs(e1 - e0) <= 1e-11 * np.abs(e0).max())


def _record(gas, solid, Tg=1200.0, Ts=1250.0, eps=0.1, rho_s=1200.0, dp=2e-4, P=101325.0):
    rec = np.zeros(24)
    for s, v in gas.items():
        rec[IDX[s]] = v
    for s, v in solid.items():
        rec[IDX[s]] = v
    rec[18:24] = [Tg, Ts, eps, rho_s, dp, P]
    return rec


def test_pyrolysis_alone_is_discrete_first_order_decay():
    rec = _record({"N2": 1.0}, {"CV": 0.3, "CA": 0.7})
    dt, delta = 1e-3, 0.01
    out, rho_g, it, st = mp.solve(rec[None, :], dt, alpha=0.0, y_step_max=1.0, delta_max=delta,
                                  dft_on=0)
    assert it[0] == 100
    mw, _ = mp.tables()
    k = mw[IDX["CV"]] * 5.39808917197452e-1 * np.exp(-2.02305749338465e3 / rec[mp.I_TS])
    c0 = rec[mp.I_EPS] * rec[mp.I_RHOS] * rec[IDX["CV"]]
    c_end = (c0 * (1.0 - k * delta * dt) ** 100)
    c1 = out[0, mp.I_EPS] * rec[mp.I_RHOS] * out[0, IDX["CV"]]
    assert c1 == pytest.approx(c_end, rel=1e-13)


def test_moisture_release_alone_is_discrete_first_order_in_solid_mass():
    rec = _record({"N2": 1.0}, {"CM": 0.2, "CA": 0.8})
    dt, delta = 1e-3, 0.01
    out, rho_g, it, st = mp.solve(rec[None, :], dt, alpha=0.0, y_step_max=1.0, delta_max=delta,
                                  dft_on=0)
    assert it[0] == 100
    mw, _ = mp.tables()
    kappa = mw[IDX["CM"]] * 1.0061447769396e-1 / (rec[mp.I_DP] * rec[mp.I_RHOS])
    u0 = rec[mp.I_EPS] * rec[mp.I_RHOS]
    cm = 0.2 * u0                                 # the ash stays, the moisture follows
    ash = 0.8 * u0
    for _ in range(100):                          # Euler on dc_CM/dt = -kappa (c_CM + ash)
        cm = cm - kappa * delta * dt * (cm + ash)
    u_end = cm + ash
    assert out[0, mp.I_EPS] * rec[mp.I_RHOS] == pytest.approx(u_end, rel=1e-12)
    # closed form of the same recursion: u_n - ... with v = c_CM + ash: v_{n+1} = v_n (1 - kappa h)
    v_end = u0 * (1.0 - kappa * delta * dt) ** 100
    assert u_end == pytest.approx(v_end, rel=1e-12)


@pytest.mark.parametrize("dft_on", [0, 1])
def test_water_gas_shift_ends_at_its_equilibrium(dft_on):
    rec = _record({"CO": 0.2, "H2O": 0.2, "CO2": 0.1, "H2": 0.02, "N2": 0.48}, {"CA": 1.0},
                  Tg=1100.0, Ts=1100.0, eps=0.2)
    out, _, it, st = mp.solve(rec[None, :], 3.0, alpha=0.0, dft_on=dft_on)
    assert st[0] == 0
    X = out[0]
    lhs = 2.87480073925354e0 * X[IDX["CO"]] * X[IDX["H2O"]] * np.exp(-8.42570940582151e3 / 1100.0)
    rhs = 1.08482987533646e2 * X[IDX["CO2"]] * X[IDX["H2"]] * np.exp(-1.23814194058215e4 / 1100.0)
    assert lhs == pytest.approx(rhs, rel=1e-6)


def test_first_order_convergence_to_radau():
    """All eleven reactions at once on one cell, gamma off, damper off."""
    rec = synth.multiphase_cells(1, seed=5)[0]
    mw, nu = mp.tables()
    c0 = mp.initial_densities(rec)
    args = (rec[mp.I_TG], rec[mp.I_TS], rec[mp.I_RHOS], rec[mp.I_DP], rec[mp.I_P])

    def f(t, c):
        return mw * (nu.T @ mp.rates(c, *args, alpha=0.0))

    dt = 2e-4
    ref = solve_ivp(f, (0.0, dt), c0, method="Radau", rtol=1e-12, atol=1e-14).y[:, -1]
    errs = []
    for delta in (1e-3, 1e-4):
        out, rho_g, it, st = mp.solve(rec[None, :], dt, alpha=0.0, dft_on=0, delta_max=delta,
                                      y_step_max=delta)
        es = out[0, mp.I_EPS]
        c1 = np.concatenate([(1 - es) * rho_g[0] * out[0, :14], es * rec[mp.I_RHOS] * out[0, 14:18]])
        errs.append(np.abs(c1 - ref).max() / np.abs(ref).max())
    print("relative error vs Radau:", errs)
    assert errs[1] < 1e-3
    assert 5.0 < errs[0] / errs[1] < 20.0      # first order: 10x per 10x smaller steps
