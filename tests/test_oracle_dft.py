"""Pins of the ringing detector (Sec. 2.3, Eqs. 8-14) in the oracle."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("seed", range(5))
def test_dft_magnitudes_match_fft(seed):
    # Eq. 9 against numpy's FFT, an independent computation of the DFT
    rng = np.random.default_rng(seed)
    x = rng.normal(size=13) * 10.0 ** rng.uniform(-9, 2)
    ref = np.abs(np.fft.fft(x))
    for j in range(13):
        assert abs(oracle.dft_mag(x, j) - ref[j]) <= 1e-13 * np.abs(x).sum()


def test_dft_rotation_invariant():
    # the ring buffer is never re-ordered: magnitudes ignore rotation
    x = np.random.default_rng(9).normal(size=13)
    for shift in range(13):
        y = np.roll(x, shift)
        for j in range(7):
            assert abs(oracle.dft_mag(y, j) - oracle.dft_mag(x, j)) < 1e-14 * np.abs(x).sum()


def test_constant_series_is_not_ringing():
    # all high-frequency bins of a constant window are 0 -> rOF grows back to 1
    x = np.full(13, 1e-9)
    assert oracle.ring_update(x, 0.25) == 0.5     # r_fac = 2 -> 0.25 * 2
    assert oracle.ring_update(x, 1.0) == 1.0      # Eq. 13 caps at 1


def test_alternating_series_near_equilibrium_is_damped():
    # +-a alternating: D0 = a (odd N), D6 = a/sin(pi/26) ~ 8.3 a -> f_ring ~ 0.12 < 0.5
    a = 1e-8
    x = a * (-1.0) ** np.arange(13)
    assert oracle.dft_mag(x, 0) == pytest.approx(a, rel=1e-12)
    assert oracle.dft_mag(x, 6) == pytest.approx(a / np.sin(np.pi / 26), rel=1e-12)
    assert oracle.ring_update(x, 1.0) == 0.5      # Eq. 12: 1/r_fac
    assert oracle.ring_update(x, 0.5) == 0.25
    # same ringing, but D0 = 1e-4 > Tol_freq: not at equilibrium -> no damping
    assert oracle.ring_update(x * 1e4, 0.5) == 1.0


def test_slow_drift_is_not_ringing():
    # a monotone ramp has its energy at low frequency: f_ring > 0.5
    x = 1e-9 * (1.0 + 0.01 * np.arange(13))
    assert oracle.ring_update(x, 0.5) == 1.0


def test_rof_stays_positive_and_bounded():
    x = 1e-9 * (-1.0) ** np.arange(13)
    r = 1.0
    for _ in range(200):
        r = oracle.ring_update(x, r)
        assert 0.0 < r <= 1.0
    assert r == oracle.DEFAULT_OPTS["rof_min"]
