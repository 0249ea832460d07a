"""Parity of the plain FP64 CUDA path with the FP64 CPU oracle.

The bar is max|dY| <= 1e-8 and |dT| <= 1e-6 K.  STEV's final state is not a
well-conditioned function of its input on every cell: the limiter's min over
species, the y < 1e-20 switch, the DFT thresholds and the last-step flag are
discontinuous, and a cell that rings at its limiter's amplitude ends at a
phase of the ringing that a one-ulp change of any rate can move (the oracle
against itself, with every kf changed by one ulp, moves 7% of the small
workload's cells by more than 1e-8, up to 2.4e-4).  So parity is checked as:

1. prefix parity: after k = 1..100 steps (max_iters = k) both sides hold the
   same state to 1e-10, before any divergence can build up;
2. full-solve parity at 1e-8 / 1e-6 K on every cell the oracle's own
   conditioning probe shows to be well-conditioned (spread < 1e-10);
3. on the remaining cells, the GPU lies within the spread the oracle itself
   shows under rounding-size rate changes (times a margin: the GPU's rates
   differ from the oracle's by tens of ulp, not the probes' one), its T
   within that plus the two trajectories' first-order enthalpy drift (forward
   Euler does not conserve H exactly), and it conserves mass and elements;
4. the GPU's deviations over the ill-conditioned cells are distributed like
   one probe run's: their median, 90th and 99th percentiles within a small
   factor of the largest single probe's (a dropped term or a wrong sign moves
   every cell, and these statistics with them, by far more);
5. identical per-cell status everywhere.
"""
import numpy as np
import pytest

import oracle
from paper_1905_09395_b300 import CELL_MAXITER, CELL_OK, Mechanism, synth

pytestmark = pytest.mark.gpu

TOL_Y, TOL_T = 1e-8, 1e-6          # the full-solve bar
PREFIX_Y, PREFIX_T = 1e-10, 1e-7   # before divergence can build up
WELL_Y, WELL_T = 1e-10, 1e-8       # oracle probe spread of a well-conditioned cell
SPREAD_MARGIN = 1e3                # 3: |gpu - oracle| <= margin * spread + bar
DISTRIB = 4.0                      # 4: median / p90 / p99 bound, multiples of a probe's


def _dev(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _gpu_solve(mech, T, P, Y, dt, **opts):
    m = Mechanism(mech, **opts)
    Td, Pd, Yd = _dev(T, P, Y)
    out = tuple(x.cpu().numpy() for x in m.solve(Td, Pd, Yd, dt))
    m.close()
    return out


def _prefix(gpu, ref, k):
    To, Yo, it, st = gpu
    rT, rY, rit, rst = ref
    assert (st == rst).all()
    assert (it == rit).all()
    assert (it <= k).all()
    dY = np.abs(Yo - rY).max()
    dT = np.abs(To - rT).max()
    assert dY <= PREFIX_Y and dT <= PREFIX_T, "k=%d: max|dY| %.3g max|dT| %.3g" % (k, dY, dT)
    return dY, dT


def _enthalpy(mech, T, Y):
    """Mixture enthalpy (J/kg) and cp (J/kg/K) per cell from the oracle's thermo."""
    H = np.zeros(len(T))
    cp = np.zeros(len(T))
    hW = np.zeros((len(T), mech.n_species))
    for c in range(len(T)):
        cpR, hRT, _ = oracle.thermo(mech, T[c])
        hW[c] = hRT * 8.314462618 * T[c] / mech.mol_weight
        H[c] = np.dot(Y[c], hW[c])
        cp[c] = 8.314462618 * np.dot(Y[c], cpR / mech.mol_weight)
    return H, cp, hW


def _distribution(dev, probes, ill, label, factor=DISTRIB):
    """The GPU's deviations over the ill-conditioned cells against each probe
    run's own deviations there (item 4)."""
    if ill.sum() < 20:
        return
    for q in (50, 90, 99):
        got = np.percentile(dev[ill], q)
        ref = max(np.percentile(p[ill], q) for p in probes)
        print("%s p%d: %.3g (largest probe's %.3g)" % (label, q, got, ref))
        assert got <= factor * ref, "%s: p%d %.3g over %g x the probes' %.3g" % (
            label, q, got, factor, ref)


def _full(gpu, ref, spread_Y, spread_T, mech=None, T0=None, Y0=None, y_step_max=1e-3,
          min_well=0.3, outliers=0.0, runs=None):
    """Full-solve parity (module docstring, items 2-5).  outliers: fraction of
    probe-well-conditioned cells allowed past the bar, each still within
    twice the limiter's per-step bound Y_step^max, for a sensitivity the
    rate-scaling probes cannot reach (an equilibrium that cancels exactly in
    the oracle's arithmetic, test_gpu_bfer).  runs: the probe runs' own
    per-cell deviations (oracle.conditioning's per_run) for item 4."""
    To, Yo, it, st = gpu
    rT, rY, rit, rst = ref
    assert (st == rst).all(), "status differs in %d cells" % int((st != rst).sum())
    dY = np.abs(Yo - rY).max(axis=1)
    dT = np.abs(To - rT)
    well = (spread_Y < WELL_Y) & (spread_T < WELL_T)
    assert well.mean() >= min_well, "only %.3f of cells are well-conditioned" % well.mean()
    bad = np.nonzero(well & ((dY > TOL_Y) | (dT > TOL_T)))[0]
    assert bad.size <= outliers * well.sum(), "well-conditioned cells over the bar: %s dY %s dT %s" % (
        bad[:8], dY[bad[:8]], dT[bad[:8]])
    assert np.all(dY[bad] <= 2.0 * y_step_max), "outliers beyond 2 Y_step^max: %s" % dY[bad]
    # the rest: Y within the oracle's own spread times the margin
    limY = TOL_Y + SPREAD_MARGIN * spread_Y
    limY[bad] = 2.0 * y_step_max
    over = np.nonzero(dY > limY)[0]
    assert over.size == 0, "cells beyond the Y bound: %s dY %s spread %s" % (
        over[:8], dY[over[:8]], spread_Y[over[:8]])
    limT = TOL_T + SPREAD_MARGIN * spread_T
    if mech is not None:
        # forward Euler conserves enthalpy to first order only: two valid
        # trajectories can end apart by their drifts plus the heat of their dY
        H0, _, _ = _enthalpy(mech, T0, Y0)
        Hg, cpg, hWg = _enthalpy(mech, To, Yo)
        Ho, _, _ = _enthalpy(mech, rT, rY)
        limT = limT + (np.abs(Hg - H0) + np.abs(Ho - H0) +
                       np.sum(np.abs(Yo - rY) * np.abs(hWg), axis=1)) / cpg
    overT = np.nonzero(dT > limT)[0]
    assert overT.size == 0, "cells beyond the T bound: %s dT %s" % (overT[:8], dT[overT[:8]])
    ratio = dY / np.maximum(spread_Y, 1e-300)
    print("|dY| / probe envelope: median %.3g p99 %.3g max %.3g (outside the %d allowed cells)"
          % (np.median(ratio), np.percentile(ratio, 99),
             np.delete(ratio, bad).max() if ratio.size > bad.size else 0.0, bad.size))
    if runs is not None:
        keep = np.ones(len(dY), bool)
        keep[bad] = False
        _distribution(dY, [r[0] for r in runs.values()], keep & (spread_Y >= 1e-2 * TOL_Y),
                      "|dY|")
        _distribution(dT, [r[1] for r in runs.values()], keep & (spread_T >= 1e-2 * TOL_T),
                      "|dT|")
    return dict(well=well.mean(), within_bar=np.mean((dY <= TOL_Y) & (dT <= TOL_T)),
                max_dY_well=dY[well].max() if well.any() else 0.0, max_dY=dY.max(),
                max_dT=dT.max(), iter_match=np.mean(it == rit))


# ------------------------------------------------------------- small 8 / 20
@pytest.fixture(scope="module")
def small():
    mech, T, P, Y, dt = synth.small_case(4096)
    runs = {}
    base, sY, sT = oracle.conditioning(mech, T, P, Y, dt, per_run=runs)
    return mech, T, P, Y, dt, base, sY, sT, runs


def test_small_full_solve(small):
    mech, T, P, Y, dt, ref, sY, sT, runs = small
    gpu = _gpu_solve(mech, T, P, Y, dt)
    r = _full(gpu, ref, sY, sT, mech, T, Y, runs=runs)
    print("8/20 x 4096:", {k: float("%.4g" % v) for k, v in r.items()})
    # conservation on the GPU result itself
    np.testing.assert_allclose(gpu[1].sum(axis=1), Y.sum(axis=1), rtol=0, atol=1e-12)
    e0 = (Y / mech.mol_weight) @ mech.elements
    e1 = (gpu[1] / mech.mol_weight) @ mech.elements
    assert np.all(np.abs(e1 - e0) <= 1e-11 * np.abs(e0).max(axis=1, keepdims=True))


@pytest.mark.parametrize("k", [1, 2, 13, 14, 50, 100])
def test_small_prefix(small, k):
    mech, T, P, Y, dt = small[:5]
    n = 2048
    ref = oracle.solve(mech, T[:n], P[:n], Y[:n], dt, max_iters=k)
    gpu = _gpu_solve(mech, T[:n], P[:n], Y[:n], dt, max_iters=k)
    _prefix(gpu, ref, k)
    assert (gpu[3] == CELL_MAXITER).all()


@pytest.mark.parametrize("n", [1, 31, 33, 1000])
def test_ragged_sizes(small, n):
    mech, T, P, Y, dt, ref, sY, sT, _ = small
    gpu = _gpu_solve(mech, T[:n], P[:n], Y[:n], dt)
    _full(gpu, tuple(r[:n] for r in ref), sY[:n], sT[:n], mech, T[:n], Y[:n], min_well=0.0)


def test_empty_is_noop(small):
    import torch
    mech = small[0]
    m = Mechanism(mech)
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    out = m.solve(e, e, torch.empty((0, mech.n_species), dtype=torch.float64, device="cuda"),
                  1e-3)
    assert all(x.numel() == 0 for x in out)
    m.close()


def test_soa_host_and_inplace_paths_are_identical(small):
    import torch
    mech, T, P, Y, dt = small[:5]
    n = 777
    m = Mechanism(mech)
    Td, Pd, Yd = _dev(T[:n], P[:n], Y[:n])
    ref = [x.cpu().numpy() for x in m.solve(Td, Pd, Yd, dt)]
    soa = [x.cpu().numpy() for x in m.solve(Td, Pd, Yd.t().contiguous(), dt, soa=True)]
    soa[1] = soa[1].T
    host = m.solve_host(T[:n], P[:n], Y[:n], dt)
    Ti, Yi = Td.clone(), Yd.clone()
    it = torch.empty(n, dtype=torch.int32, device="cuda")
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    m.solve(Ti, Pd, Yi, dt, out=(Ti, Yi, it, st))
    inplace = [x.cpu().numpy() for x in (Ti, Yi, it, st)]
    for other in (soa, host, inplace):
        for a, b in zip(ref, other):
            np.testing.assert_array_equal(a, b)
    m.close()


@pytest.mark.parametrize("opts", [dict(alpha=0.0), dict(dft_on=0), dict(tol_freq=1e-2),
                                  dict(delta_max=0.002, y_step_max=3e-4)])
def test_option_variants_prefix(small, opts):
    mech, T, P, Y, dt = small[:5]
    n = 1024
    for k in (14, 60):
        ref = oracle.solve(mech, T[:n], P[:n], Y[:n], dt, max_iters=k, **opts)
        gpu = _gpu_solve(mech, T[:n], P[:n], Y[:n], dt, max_iters=k, **opts)
        _prefix(gpu, ref, k)


def test_maxiter_status_mix(small):
    mech, T, P, Y, dt = small[:5]
    n = 1024
    ref = oracle.solve(mech, T[:n], P[:n], Y[:n], dt, max_iters=1150)
    gpu = _gpu_solve(mech, T[:n], P[:n], Y[:n], dt, max_iters=1150)
    assert (gpu[3] == CELL_MAXITER).any() and (gpu[3] == CELL_OK).any()
    # statuses are decided by iteration counts, which can move on ill-conditioned cells
    assert np.mean(gpu[3] == ref[3]) > 0.97


# -------------------------------------------------- 32 / 150 and 53 / 325
# Short step prefixes here, at the 1e-10 bar; full solves and prefixes of 50,
# 100 and 200 steps on the 32/150 workload against the oracle's stored probe
# runs are in test_gpu_scale_parity.
@pytest.fixture(scope="module")
def scale():
    mech = synth.scale_mechanism()
    T, P, Y = synth.make_cells(mech, 192, seed=11, T_range=(800, 2200), P_atm_range=(1, 5),
                               dirichlet=0.5)
    return mech, T, P, Y, 1e-3


@pytest.mark.parametrize("k", [1, 13, 14, 20])
def test_scale_prefix(scale, k):
    mech, T, P, Y, dt = scale
    ref = oracle.solve(mech, T, P, Y, dt, max_iters=k)
    gpu = _gpu_solve(mech, T, P, Y, dt, max_iters=k)
    _prefix(gpu, ref, k)


@pytest.mark.parametrize("k", [1, 14, 20])
def test_large_prefix(k):
    mech = synth.large_mechanism()
    T, P, Y = synth.make_cells(mech, 64, seed=12, T_range=(700, 2500), P_atm_range=(1, 5),
                               dirichlet=0.5)
    ref = oracle.solve(mech, T, P, Y, 5e-4, max_iters=k)
    gpu = _gpu_solve(mech, T, P, Y, 5e-4, max_iters=k)
    _prefix(gpu, ref, k)
