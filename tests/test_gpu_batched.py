"""Uneven independent batches in one persistent launch (stev_solve_batched):
every cell's result is the one a solve of its batch alone gives, whatever the
batch sizes and fluid time steps; and the 53-species / 325-reaction
mechanism's batched solve follows the oracle step for step."""
import numpy as np
import pytest

import oracle
from paper_1905_09395_b300 import FP64, MIXED, Mechanism, synth

pytestmark = pytest.mark.gpu


def _dev(*a):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_batched_equals_separate_solves(precision):
    mech, T, P, Y, _ = synth.small_case(4096)
    sizes = [1, 0, 137, 1000, 33, 2925]
    dts = [1e-3, 2e-3, 5e-4, 1e-3, 2.5e-4, 1e-3]
    m = Mechanism(mech, precision=precision)
    batches, o = [], 0
    for n in sizes:
        batches.append(tuple(_dev(T[o:o + n], P[o:o + n], Y[o:o + n])))
        o += n
    got = m.solve_batched(batches, dts)
    for (Tb, Pb, Yb), dt, g in zip(batches, dts, got):
        if Tb.shape[0] == 0:
            continue
        ref = m.solve(Tb, Pb, Yb, dt)
        for a, b in zip(g, ref):
            np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    m.close()


def test_large_mechanism_batched_prefix():
    # 53/325 mixed in uneven batches: the first 20 steps against the oracle
    mech = synth.large_mechanism()
    sizes = [5, 40, 19]
    T, P, Y = synth.make_cells(mech, sum(sizes), seed=4, T_range=(700, 2500),
                               P_atm_range=(1, 5), dirichlet=0.5)
    m = Mechanism(mech, precision=MIXED, max_iters=20)
    batches, o = [], 0
    for n in sizes:
        batches.append(tuple(_dev(T[o:o + n], P[o:o + n], Y[o:o + n])))
        o += n
    got = m.solve_batched(batches, 5e-4)
    Yg = np.concatenate([g[1].cpu().numpy() for g in got])
    itg = np.concatenate([g[2].cpu().numpy() for g in got])
    ref = oracle.solve(mech, T, P, Y, 5e-4, max_iters=20)
    assert (itg == ref[2]).all()
    assert np.abs(Yg - ref[1]).max() <= 1e-5
    m.close()
