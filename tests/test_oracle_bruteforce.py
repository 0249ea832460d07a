"""The oracle's integrator against a tight-tolerance implicit brute force.

scipy's Radau (an implicit Runge-Kutta method independent of STEV) integrates
the same right-hand side at rtol 1e-12 on a tiny stiff mechanism (eigenvalues
-3e6 and -1e4 /s at the start).  STEV must land within the paper's "similar
degree of accuracy" at its defaults, and its error must fall like a
first-order method (Eq. 18) once delta^max and Y_step^max are small enough
that the limiter no longer rings (Sec. 2.1, Sec. 4)."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
from mechs import P_ATM, constant_cp_block, tiny_mechanism


def _mech():
    # A + B <=> C (fast), C <=> D (slower), exothermic; E inert
    W = [0.016, 0.032, 0.048, 0.048, 0.028]
    blocks = [constant_cp_block(3.5, a6=-2000.0, a7=4.0),
              constant_cp_block(3.8, a6=1000.0, a7=6.0),
              constant_cp_block(5.1, a6=-6000.0, a7=16.0),
              constant_cp_block(5.3, a6=-9000.0, a7=15.0),
              constant_cp_block(3.5, a6=0.0, a7=5.0)]
    return tiny_mechanism(W, blocks, [{0: -1, 1: -1, 2: 1}, {2: -1, 3: 1}], A=[2e3, 3e3],
                          beta=[0.5, 0.0], Ea=[3e4, 4e4])


@pytest.fixture(scope="module")
def case():
    m = _mech()
    om = oracle.OracleMechanism(m)
    P0, T0 = 2 * P_ATM, 1300.0
    x0 = np.array([0.3, 0.3, 0.05, 0.05, 0.3])
    Y0 = x0 * m.mol_weight / np.sum(x0 * m.mol_weight)

    def f(t, z):
        r = oracle.rates(om, z[-1], P0, z[:-1], alpha=0.0)
        return np.append(r["dYdt"], r["dTdt"])

    sol = solve_ivp(f, (0.0, 1e-3), np.append(Y0, T0), method="Radau", rtol=1e-12, atol=1e-15)
    assert sol.status == 0
    return om, P0, T0, Y0, sol.y[:, -1]


def _err(case, delta, ymax):
    om, P0, T0, Y0, ref = case
    tr = oracle.solve_cell_trace(om, T0, P0, Y0, 1e-3, trace_cap=1, alpha=0.0, dft_on=0,
                                 delta_max=delta, y_step_max=ymax)
    assert tr["status"] == oracle.CELL_OK
    return np.abs(tr["Y"] - ref[:-1]).max(), abs(tr["T"] - ref[-1])


def test_defaults_are_close_to_brute_force(case):
    eY, eT = _err(case, 0.01, 1e-3)
    assert eY <= 1e-3 and eT <= 1.0
    assert abs(case[4][-1] - case[2]) > 50.0        # the case does release heat


def test_first_order_convergence(case):
    e1 = _err(case, 1e-3, 1e-4)
    e2 = _err(case, 1e-4, 1e-5)
    assert e1[0] / e2[0] == pytest.approx(10.0, rel=0.3)
    assert e1[1] / e2[1] == pytest.approx(10.0, rel=0.3)
