"""Pins of the oracle's thermo (Sec. 3, Eqs. 15-16, and S/R) against physics.

None of these retypes the oracle's polynomials: they check calculus
identities (cp = dH/dT, dS/dT = cp/T), the textbook monatomic ideal gas and
the range switch at T_split."""
import numpy as np
import pytest

import oracle
from paper_1905_09395_b300 import synth
from mechs import constant_cp_block, tiny_mechanism


@pytest.fixture(scope="module")
def mech():
    return synth.scale_mechanism()


@pytest.mark.parametrize("T", [350.0, 640.0, 999.0, 1001.0, 1500.0, 2400.0, 3700.0])
def test_cp_is_derivative_of_enthalpy(mech, T):
    # H/R = (H/RT) * T; cp/R = d(H/R)/dT (Eq. 15 is the derivative of Eq. 16 x T)
    d = 1e-3
    _, hp, _ = oracle.thermo(mech, T + d)
    _, hm, _ = oracle.thermo(mech, T - d)
    cp, _, _ = oracle.thermo(mech, T)
    dHdT = (hp * (T + d) - hm * (T - d)) / (2 * d)
    np.testing.assert_allclose(dHdT, cp, rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("T", [350.0, 640.0, 1500.0, 2400.0, 3700.0])
def test_entropy_derivative_is_cp_over_T(mech, T):
    d = 1e-3
    _, _, sp = oracle.thermo(mech, T + d)
    _, _, sm = oracle.thermo(mech, T - d)
    cp, _, _ = oracle.thermo(mech, T)
    np.testing.assert_allclose((sp - sm) / (2 * d), cp / T, rtol=2e-6, atol=1e-9)


def test_continuity_at_split(mech):
    # the generator makes the two ranges continuous; the oracle must pick
    # the low block just below T_split and the high block at/above it.
    lo = oracle.thermo(mech, 1000.0 * (1 - 1e-13))
    hi = oracle.thermo(mech, 1000.0)
    for a, b in zip(lo, hi):
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-9)


def test_monatomic_ideal_gas():
    # cp = 5/2 R; H(T2)-H(T1) = 5/2 R (T2-T1); S(T2)-S(T1) = 5/2 R ln(T2/T1)
    m = tiny_mechanism([0.04], [constant_cp_block(2.5, a6=-745.0, a7=4.37)], [{0: -1}], A=[1.0])
    T1, T2 = 400.0, 2900.0
    c1, h1, s1 = oracle.thermo(m, T1)
    c2, h2, s2 = oracle.thermo(m, T2)
    assert c1[0] == 2.5 and c2[0] == 2.5
    assert abs((h2[0] * T2 - h1[0] * T1) - 2.5 * (T2 - T1)) < 1e-9
    assert abs((s2[0] - s1[0]) - 2.5 * np.log(T2 / T1)) < 1e-12


def test_range_selection():
    # cp/R = 2.5 below the split, 4.5 at and above it
    m = tiny_mechanism([0.04], [np.stack([constant_cp_block(2.5), constant_cp_block(4.5)])],
                       [{0: -1}], A=[1.0], t_split=1200.0)
    assert oracle.thermo(m, 1199.0)[0][0] == 2.5
    assert oracle.thermo(m, 1200.0)[0][0] == 4.5
    assert oracle.thermo(m, 5000.0)[0][0] == 4.5
