"""Ragged and empty inputs on the mixed-precision kernels (Sec. 2.4's
variable load).

Cells are independent, and each cell's lane group reduces only over its own
lanes, so a cell's result cannot depend on how many cells share its launch,
its warp (four cells per warp with the 8-species mechanism's 8-lane groups)
or which slot it lands in.  A solve of the first n cells must therefore give,
bit for bit, the rows that a solve of a larger batch gives for them, for
counts that leave the last warp partly filled; an empty solve launches
nothing and returns empty arrays.  Covered: the generic kernel, the kernel
compiled for the mechanism, and the thermo-network kernel (whose warps share
their MMAs between the warp's cells), on the 8/20 mechanism, plus the
compiled network kernel on 32/150 (one cell per warp)."""
import numpy as np
import pytest

from paper_1905_09395_b300 import MIXED, THERMO_MLP, Mechanism, synth

pytestmark = pytest.mark.gpu

SIZES = (1, 3, 5, 33, 1000)


def _run(m, T, P, Y, dt):
    import torch
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (T, P, Y)]
    return tuple(x.cpu().numpy() for x in m.solve(*d, dt))


def _empty(m, S):
    import torch
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    out = m.solve(e, e, torch.empty((0, S), dtype=torch.float64, device="cuda"), 1e-3)
    assert all(x.numel() == 0 for x in out)


def _mechanism(kind, mech, max_iters):
    m = Mechanism(mech, precision=MIXED, max_iters=max_iters,
                  specialize=0 if kind == "generic" else 1)
    if kind == "network":
        T = np.random.default_rng(5).uniform(300.0, 3000.0, size=200_000)
        m.mlp_train(T, epochs=4, batch=4096, lr=2e-3, seed=1)
        m.set_options(thermo=THERMO_MLP)
    return m


@pytest.mark.parametrize("kind", ["generic", "specialised", "network"])
def test_ragged_counts_match_a_full_batch_8x20(kind):
    mech, T, P, Y, dt = synth.small_case(1024)
    m = _mechanism(kind, mech, max_iters=400)
    full = _run(m, T, P, Y, dt)
    for n in SIZES:
        part = _run(m, T[:n], P[:n], Y[:n], dt)
        for a, b in zip(part, full):
            assert np.array_equal(a, b[:n]), "n=%d" % n
    _empty(m, mech.n_species)
    m.close()


def test_ragged_counts_match_a_full_batch_network_32x150():
    mech = synth.scale_mechanism()
    T, P, Y = synth.make_cells(mech, 512, seed=2, T_range=(800, 2200), P_atm_range=(1, 5),
                               dirichlet=0.5)
    m = _mechanism("network", mech, max_iters=100)
    full = _run(m, T, P, Y, 1e-3)
    for n in SIZES[:-1]:
        part = _run(m, T[:n], P[:n], Y[:n], 1e-3)
        for a, b in zip(part, full):
            assert np.array_equal(a, b[:n]), "n=%d" % n
    _empty(m, mech.n_species)
    m.close()
