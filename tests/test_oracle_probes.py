"""The conditioning probes of the oracle (test infrastructure for the parity
tests): what each one perturbs, pinned on cells whose behaviour is known.

- the uniform scalings (every kf, or every K, by a single-precision-sized
  factor) move small-mechanism cells by a rounding-sized amount over a full
  solve (over a few limiter-bound steps they move nothing: h scales with
  1/kf, so h r and hence Y do not change);
- the reverse-term noise probe (every reverse term times 1 + 2^-22 xi, xi a
  hash in [-1, 1)) perturbs at the same size on such a cell, differs between
  its two seeds, and is deterministic;
- on BFER cell 1875 (Sec. 7.1's mechanism), whose COROX net rate the FP64
  arithmetic cancels to exactly 0.0 while forward Euler at h = delta t_f is
  unstable for it (Eq. 4's time cap), the uniform scalings move the final
  state by far less than the noise probe does: they shift the exact fixed
  point without making it inexact."""
import numpy as np

import oracle
from paper_1905_09395_b300 import synth


def _cells():
    mech, T, P, Y, dt = synth.small_case(64)
    return mech, T[:8], P[:8], Y[:8], dt


def test_uniform_and_noise_probes_on_small_cells():
    mech, T, P, Y, dt = _cells()
    base = oracle.solve(mech, T, P, Y, dt)
    # a few limiter-bound steps: the uniform kf scaling moves nothing
    short = oracle.solve(mech, T, P, Y, dt, max_iters=5)
    short_up = oracle.solve(mech, T, P, Y, dt, max_iters=5, probe="kf32_up")
    assert np.abs(short_up[1] - short[1]).max() < 1e-15
    up = oracle.solve(mech, T, P, Y, dt, probe="kf32_up")
    a = oracle.solve(mech, T, P, Y, dt, probe="qnoise32_a")
    a2 = oracle.solve(mech, T, P, Y, dt, probe="qnoise32_a")
    b = oracle.solve(mech, T, P, Y, dt, probe="qnoise32_b")
    # full solves: rounding-sized moves (these cells are well-conditioned at
    # the single-precision level: well under the mixed path's 1e-4 target)
    for r in (up, a, b):
        assert 0.0 < np.abs(r[1] - base[1]).max() < 1e-5
    # the noise probe is seed-dependent and deterministic
    assert not np.array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[1], a2[1])
    np.testing.assert_array_equal(a[0], a2[0])


def test_exact_cancellation_cell_is_seen_only_by_the_noise_probe():
    mech = synth.bfer_mechanism()
    T, P, Y = synth.bfer_cells(mech, 2048)
    c = slice(1875, 1876)
    base = oracle.solve(mech, T[c], P[c], Y[c], 1e-3)
    uniform = max(np.abs(oracle.solve(mech, T[c], P[c], Y[c], 1e-3, probe=p)[1] - base[1]).max()
                  for p in ("kf32_up", "kf32_down", "K32_up", "K32_down"))
    noise = max(np.abs(oracle.solve(mech, T[c], P[c], Y[c], 1e-3, probe=p)[1] - base[1]).max()
                for p in ("qnoise32_a", "qnoise32_b"))
    assert uniform < 1e-6
    assert noise > 1e-4
