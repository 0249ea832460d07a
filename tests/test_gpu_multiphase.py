"""Parity of the multiphase (gas-solid) CUDA path, stev_mp_solve (Sec. 7.2,
Eqs. 31-56, Table 2), with the FP64 multiphase oracle.

As for the single-phase path: step prefixes (max_iters = k) before any
divergence can build up must agree to 1e-10 with identical iteration counts
and statuses; full solves must agree to 1e-8 on every cell the oracle's own
probe (every rate constant changed by one ulp) leaves within 1e-10, and
elsewhere within the probe's spread (x1000) or twice Y_step^max; every
status must be the oracle's; the GPU result conserves mass."""
import numpy as np
import pytest

from oracle import multiphase as mp
from paper_1905_09395_b300 import binding, synth

pytestmark = pytest.mark.gpu


def _gpu(cells, dt, **opts):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(cells)).cuda()
    return tuple(x.cpu().numpy() for x in binding.mp_solve(d, dt, **opts))


@pytest.fixture(scope="module")
def cells():
    return synth.multiphase_cells(2048, seed=2)


@pytest.mark.parametrize("k", [1, 2, 13, 14, 50])
def test_prefix(cells, k):
    ref = mp.solve(cells, 1e-3, max_iters=k)
    got = _gpu(cells, 1e-3, max_iters=k)
    assert (got[2] == ref[2]).all() and (got[3] == ref[3]).all()
    assert np.abs(got[0][:, :18] - ref[0][:, :18]).max() <= 1e-10
    assert np.abs(got[0][:, mp.I_EPS] - ref[0][:, mp.I_EPS]).max() <= 1e-12
    np.testing.assert_array_equal(got[0][:, 18:20], cells[:, 18:20])
    np.testing.assert_array_equal(got[0][:, 21:], cells[:, 21:])


def test_full_solve(cells):
    base, dX, de = mp.conditioning(cells, 1e-3)
    got = _gpu(cells, 1e-3)
    assert (got[3] == base[3]).all()
    dev = np.abs(got[0][:, :18] - base[0][:, :18]).max(axis=1)
    deps = np.abs(got[0][:, mp.I_EPS] - base[0][:, mp.I_EPS])
    well = dX < 1e-10
    print("multiphase x 2048: well-conditioned %.3f, max |dX| there %.3g, overall %.3g; "
          "iteration match %.3f" % (well.mean(), dev[well].max() if well.any() else 0.0,
                                    dev.max(), np.mean(got[2] == base[2])))
    assert well.mean() >= 0.5
    assert np.all(dev[well] <= 1e-8) and np.all(deps[well] <= 1e-8)
    assert np.all(dev <= np.maximum(1e-8 + 1e3 * dX, 2e-3))
    # mass: gas and solid partial densities summed, before and after
    for c in range(0, len(cells), 97):
        c0 = mp.initial_densities(cells[c]).sum()
        es = got[0][c, mp.I_EPS]
        c1 = (1 - es) * got[1][c] + es * cells[c, mp.I_RHOS]
        assert c1 == pytest.approx(c0, rel=1e-12)


@pytest.mark.parametrize("n", [0, 1, 129])
def test_ragged_and_empty(cells, n):
    got = _gpu(cells[:n], 1e-3, max_iters=20)
    ref = mp.solve(cells[:n], 1e-3, max_iters=20)
    assert got[0].shape == (n, 24)
    if n:
        assert (got[2] == ref[2]).all()
        assert np.abs(got[0][:, :18] - ref[0][:, :18]).max() <= 1e-10


def test_in_place_equals_separate(cells):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(cells[:300])).cuda()
    sep = [x.cpu().numpy() for x in binding.mp_solve(d, 1e-3)]
    n = 300
    out = (d, torch.empty(n, dtype=torch.float64, device="cuda"),
           torch.empty(n, dtype=torch.int32, device="cuda"),
           torch.empty(n, dtype=torch.uint8, device="cuda"))
    binding.mp_solve(d, 1e-3, out=out)
    for a, b in zip(sep, out):
        np.testing.assert_array_equal(a, b.cpu().numpy())
