"""Edge cases of the CUDA path against the oracle: the largest mechanism the
library takes (64 species, 512 reactions), and the method's degenerate cells:
one at chemical equilibrium (the limiter's time cap alone sets h, so exactly
1/delta_max steps, Eq. 4), one whose T leaves [200, 6000] K, non-finite
input, and a fluid step far longer than the iteration cap allows."""
import numpy as np
import pytest

import oracle
from paper_1905_09395_b300 import (CELL_MAXITER, CELL_NONFINITE, CELL_OK, CELL_TRANGE, FP64,
                                   MIXED, Mechanism, synth)
from test_gpu_fp64 import PREFIX_T, PREFIX_Y, _gpu_solve
from test_oracle_physics import _abc_mech, _equilibrium_mix

pytestmark = pytest.mark.gpu

_cache = {}


def _max_mech():
    if "max" not in _cache:
        _cache["max"] = synth.make_mechanism(64, 512, seed=9, ea_max=200e3, name="syn64x512")
    return _cache["max"]


@pytest.mark.parametrize("k", [1, 3, 15])
def test_max_size_mechanism_prefix_fp64(k):
    mech = _max_mech()
    T, P, Y = synth.make_cells(mech, 64, seed=2, T_range=(1000, 2000), P_atm_range=(1, 3),
                               dirichlet=0.5)
    ref = oracle.solve(mech, T, P, Y, 1e-3, max_iters=k)
    gpu = _gpu_solve(mech, T, P, Y, 1e-3, max_iters=k)
    assert (gpu[2] == ref[2]).all() and (gpu[3] == ref[3]).all()
    assert np.abs(gpu[1] - ref[1]).max() <= PREFIX_Y
    assert np.abs(gpu[0] - ref[0]).max() <= PREFIX_T


def test_max_size_mechanism_mixed():
    mech = _max_mech()
    T, P, Y = synth.make_cells(mech, 64, seed=2, T_range=(1000, 2000), P_atm_range=(1, 3),
                               dirichlet=0.5)
    ref = oracle.solve(mech, T, P, Y, 1e-3, max_iters=5)
    m = Mechanism(mech, precision=MIXED, max_iters=5)
    assert m.resident_slots > 0
    import torch
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (T, P, Y)]
    gpu = [x.cpu().numpy() for x in m.solve(*d, 1e-3)]
    m.close()
    assert (gpu[2] == ref[2]).all()
    assert np.abs(gpu[1] - ref[1]).max() <= 1e-5


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_equilibrium_cell_takes_the_time_cap_steps(precision):
    m = _abc_mech()
    T, P = 1500.0, 3 * 101325.0
    _, Yeq = _equilibrium_mix(m, T, P, {0: -1, 1: -1, 2: 1}, {0: 0.2, 1: 0.1}, inert=3)
    Tc, Pc, Yc = np.array([T]), np.array([P]), Yeq[None, :]
    ref = oracle.solve(m, Tc, Pc, Yc, 1e-3)
    gpu = _gpu_solve(m, Tc, Pc, Yc, 1e-3, precision=precision)
    assert ref[2][0] == 100 and gpu[2][0] == 100          # 1 / delta_max
    assert gpu[3][0] == CELL_OK
    assert np.abs(gpu[1] - ref[1]).max() <= (1e-10 if precision == FP64 else 1e-6)
    assert np.abs(gpu[1] - Yc).max() <= 1e-6               # it stays at equilibrium


def test_temperature_range_and_nonfinite_status():
    mech, T, P, Y, dt = synth.small_case(8)
    T = T.copy()
    Y = Y.copy()
    T[0] = 150.0                 # below the 200 K floor: TRANGE after the first step
    T[1] = 7000.0                # above 6000 K
    Y[2, 3] = np.nan             # non-finite input: NONFINITE
    T[3] = np.inf
    ref = oracle.solve(mech, T, P, Y, dt)
    gpu = _gpu_solve(mech, T, P, Y, dt)
    assert (gpu[3] == ref[3]).all()
    assert gpu[3][0] == CELL_TRANGE and gpu[3][1] == CELL_TRANGE
    assert gpu[3][2] == CELL_NONFINITE and gpu[3][3] == CELL_NONFINITE
    assert (gpu[3][4:] == CELL_OK).all()
    assert (gpu[2][:4] == ref[2][:4]).all()   # the special cells stop at the same step
    # (the others ring, and ringing cells' iteration counts move with rounding)


def test_long_fluid_step_hits_the_iteration_cap():
    mech, T, P, Y, dt = synth.small_case(32)
    ref = oracle.solve(mech, T, P, Y, 1.0, max_iters=300)
    gpu = _gpu_solve(mech, T, P, Y, 1.0, max_iters=300)
    assert (ref[3] == CELL_MAXITER).all() and (gpu[3] == CELL_MAXITER).all()
    assert (gpu[2] == 300).all()
    assert np.abs(gpu[1] - ref[1]).max() <= 1e-9


def test_failed_option_change_keeps_the_previous_configuration():
    # 64/512 in FP64 fits one cell per warp but not four (lanes_per_cell = 8):
    # the change is refused and the mechanism keeps solving as before
    from paper_1905_09395_b300 import StevError
    mech = _max_mech()
    T, P, Y = synth.make_cells(mech, 8, seed=2, T_range=(1000, 2000), P_atm_range=(1, 3),
                               dirichlet=0.5)
    m = Mechanism(mech, max_iters=3)
    import torch
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (T, P, Y)]
    before = [x.cpu().numpy() for x in m.solve(*d, 1e-3)]
    slots = m.resident_slots
    with pytest.raises(StevError):
        m.set_options(lanes_per_cell=8, dft_n=9)
    assert m.options.lanes_per_cell == 0 and m.options.dft_n == 13
    assert m.resident_slots == slots
    after = [x.cpu().numpy() for x in m.solve(*d, 1e-3)]
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)
    m.close()


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_larger_mechanism_still_launches_after_a_smaller_one_on_the_same_kernel(precision):
    """Mechanisms with the same precision, lane group and thermo share one
    kernel function, and its dynamic shared-memory limit is a property of that
    function.  Configuring a smaller mechanism after a larger one must not
    leave the larger one unable to launch: the 32/150 mechanism is created
    first, then the 8/20 one with 32-lane groups (the same kernel instance,
    fewer bytes of shared memory), and both solve step prefixes that match the
    oracle."""
    big = synth.scale_mechanism()
    small = synth.small_mechanism()
    Tb, Pb, Yb = synth.make_cells(big, 64, seed=3, T_range=(1000, 2000), P_atm_range=(1, 3),
                                  dirichlet=0.5)
    _, Ts, Ps, Ys, dt = synth.small_case(64)
    import torch
    mb = Mechanism(big, precision=precision, max_iters=3)
    ms = Mechanism(small, precision=precision, max_iters=3, lanes_per_cell=32)
    tol = PREFIX_Y if precision == FP64 else 1e-5
    for m, mech, (T, P, Y) in ((mb, big, (Tb, Pb, Yb)), (ms, small, (Ts, Ps, Ys)),
                               (mb, big, (Tb, Pb, Yb))):
        d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (T, P, Y)]
        gpu = [x.cpu().numpy() for x in m.solve(*d, 1e-3)]
        ref = oracle.solve(mech, T, P, Y, 1e-3, max_iters=3)
        assert (gpu[2] == ref[2]).all() and (gpu[3] == ref[3]).all()
        assert np.abs(gpu[1] - ref[1]).max() <= tol
    mb.close()
    ms.close()
