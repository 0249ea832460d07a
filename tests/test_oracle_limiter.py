"""Pins of the step-size limiter (Sec. 2.1, Eqs. 1-5) and of the per-step
invariants it guarantees along a whole trajectory (Sec. 2.4)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1905_09395_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "limiter_cases.json")


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["why"][:40])
def test_step_size_worked_cases(case):
    h = oracle.step_size(case["Y"], case["dYdt"], case["t_f"], case["y_step_max"], case["delta_max"])
    assert h == pytest.approx(case["h"], rel=1e-15)


@pytest.fixture(scope="module")
def traces():
    mech, T, P, Y, dt = synth.small_case(64)
    out = []
    for c in range(0, 64, 8):
        out.append((mech, dt, oracle.solve_cell_trace(mech, T[c], P[c], Y[c], dt)))
    return out


def test_trajectory_invariants(traces):
    d = oracle.DEFAULT_OPTS
    for mech, dt, tr in traces:
        assert tr["status"] == oracle.CELL_OK
        h, Yt = tr["h"], tr["Y_trace"]
        n = tr["iters"]
        assert len(h) == n
        # Eq. 4-5: h <= t_f * delta_max
        assert np.all(h <= dt * d["delta_max"] * (1 + 1e-15))
        assert np.all(h > 0)
        # each cell integrates exactly to t_f (Sec. 2.1)
        assert abs(h.sum() - dt) <= n * 2.3e-16 * dt
        # Sec. 2.4: every cell is active for at least 1/delta_max iterations
        assert n >= int(np.ceil(1.0 / d["delta_max"]))
        # Eqs. 2-3: consumption per step at most min(Ymax, 0.9 y) for y >= 1e-20
        Ynext = np.vstack([Yt[1:], tr["Y"][None, :]])
        drop = Yt - Ynext
        lim = np.minimum(d["y_step_max"], 0.9 * Yt)
        ok = (Yt < 1e-20) | (drop <= lim * (1 + 1e-9) + 1e-300)
        assert ok.all()
