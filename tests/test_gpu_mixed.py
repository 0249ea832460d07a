"""Error of the mixed-precision CUDA path against the FP64 CPU oracle.

The mixed path evaluates rates, the limiter and the ringing test in FP32 and
keeps FP64 for Y, T and the Gibbs exponent of K.  Its target is
max|dY| <= 1e-4 and |dT| <= 0.5 K.  As for the FP64 path (test_gpu_fp64),
STEV's final state is ill-conditioned on ringing cells, so the target is
required on every cell that the oracle's single-precision-sized conditioning
probe (kf changed by 2^-22, K by 2^-18, the limiter and ringing thresholds by
2^-22) leaves within 1e-6 / 1e-3 K; every other cell must lie within the
target plus 100 times that probe's spread (T also within the first-order
enthalpy drift of test_gpu_fp64), and where the probe runs are given, the
deviations over the ill-conditioned cells must be distributed like one probe
run's (median, 90th and 99th percentiles within 4x of the largest probe's)."""
import numpy as np
import pytest

import oracle
from paper_1905_09395_b300 import MIXED, Mechanism, synth
from test_gpu_fp64 import _distribution, _enthalpy

pytestmark = pytest.mark.gpu

TOL_Y, TOL_T = 1e-4, 0.5
WELL_Y, WELL_T = 1e-6, 1e-3
ENVELOPE = 100.0   # elsewhere: |gpu - oracle| <= target + ENVELOPE * probe spread


def _solve(mech, T, P, Y, dt, **opts):
    import torch
    m = Mechanism(mech, precision=MIXED, **opts)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (T, P, Y)]
    out = tuple(x.cpu().numpy() for x in m.solve(*d, dt))
    m.close()
    return out


def _check(mech, T0, Y0, gpu, ref, sY, sT, label, outliers=0.0, outlier_cap=None, runs=None):
    """outliers: fraction of well-conditioned cells allowed over the target,
    each still within outlier_cap = (dY, dT) (for approximations such as the
    thermo network, whose error is systematic rather than rounding-sized, and
    for the exact equilibrium cancellation of test_gpu_bfer).  runs: the
    probe runs' own deviations (oracle.conditioning's per_run), for the
    distribution check."""
    To, Yo, it, st = gpu
    rT, rY, rit, rst = ref
    assert (st == rst).all(), "status differs in %d cells" % int((st != rst).sum())
    dY = np.abs(Yo - rY).max(axis=1)
    dT = np.abs(To - rT)
    well = (sY < WELL_Y) & (sT < WELL_T)
    bad = np.nonzero(well & ((dY > TOL_Y) | (dT > TOL_T)))[0]
    assert bad.size <= outliers * well.sum(), (
        "well-conditioned cells over target: %d, e.g. %s dY %s dT %s"
        % (bad.size, bad[:8], dY[bad[:8]], dT[bad[:8]]))
    if bad.size:
        assert np.all(dY[bad] <= outlier_cap[0]) and np.all(dT[bad] <= outlier_cap[1]), (
            "outliers beyond their cap: dY %s dT %s" % (dY[bad].max(), dT[bad].max()))
    keep = np.ones(len(dY), bool)
    keep[bad] = False
    limY = TOL_Y + ENVELOPE * sY
    over = np.nonzero(keep & (dY > limY))[0]
    assert over.size == 0, "Y beyond the probes' envelope: cells %s dY %s spread %s" % (
        over[:8], dY[over[:8]], sY[over[:8]])
    H0, _, _ = _enthalpy(mech, T0, Y0)
    Hg, cpg, hWg = _enthalpy(mech, To, Yo)
    Ho, _, _ = _enthalpy(mech, rT, rY)
    limT = TOL_T + ENVELOPE * sT + (np.abs(Hg - H0) + np.abs(Ho - H0) +
                                    np.sum(np.abs(Yo - rY) * np.abs(hWg), axis=1)) / cpg
    overT = np.nonzero(keep & (dT > limT))[0]
    assert overT.size == 0, "T beyond its bound: cells %s dT %s" % (overT[:8], dT[overT[:8]])
    if runs is not None:
        _distribution(dY, [r[0] for r in runs.values()], keep & (sY >= 1e-2 * TOL_Y),
                      label + " |dY|")
        _distribution(dT, [r[1] for r in runs.values()], keep & (sT >= 1e-2 * TOL_T),
                      label + " |dT|")
    # FP32 production rates sum to zero only to single precision (~1e-7
    # relative per step), so sum Y drifts by far less than the target
    np.testing.assert_allclose(Yo.sum(axis=1), Y0.sum(axis=1), rtol=0, atol=1e-6)
    within = np.mean((dY <= TOL_Y) & (dT <= TOL_T))
    print("%s: well-conditioned %.3f, within target %.4f (well-conditioned %.4f), max dY %.3g"
          " (well %.3g), max dT %.3g, iteration match %.3f, max (|dY| - target) / envelope %.3g"
          % (label, well.mean(), within, 1.0 - bad.size / max(well.sum(), 1), dY.max(),
             dY[well].max() if well.any() else 0, dT.max(), np.mean(it == rit),
             ((dY[keep] - TOL_Y).clip(0) / np.maximum(sY[keep], 1e-300)).max()
             if keep.any() else 0.0))
    return within


@pytest.mark.parametrize("lanes", [0, 8, 32])
def test_mixed_small_case(lanes):
    mech, T, P, Y, dt = synth.small_case(2048)
    ref, sY, sT = _small_conditioning()
    within = _check(mech, T, Y, _solve(mech, T, P, Y, dt, lanes_per_cell=lanes), ref, sY, sT,
                    "mixed 8/20 x 2048, lanes %d" % lanes, runs=_small_runs())
    assert within > 0.95


_cache = {}


def _small_conditioning():
    if "small" not in _cache:
        mech, T, P, Y, dt = synth.small_case(2048)
        runs = {}
        _cache["small"] = oracle.conditioning(mech, T, P, Y, dt, level="fp32", per_run=runs)
        _cache["small_runs"] = runs
    return _cache["small"]


def _small_runs():
    _small_conditioning()
    return _cache["small_runs"]


@pytest.mark.parametrize("k", [1, 14, 50])
def test_mixed_prefix(k):
    # a few steps in: single-precision rates move the state by ~1e-7 per unit
    mech, T, P, Y, dt = synth.small_case(2048)
    ref = oracle.solve(mech, T, P, Y, dt, max_iters=k)
    To, Yo, it, st = _solve(mech, T, P, Y, dt, max_iters=k)
    assert (it == ref[2]).all() and (st == ref[3]).all()
    assert np.abs(Yo - ref[1]).max() <= 1e-5
    assert np.abs(To - ref[0]).max() <= 1e-2


def test_mixed_large_mechanism_prefix():
    mech = synth.large_mechanism()
    T, P, Y = synth.make_cells(mech, 64, seed=12, T_range=(700, 2500), P_atm_range=(1, 5),
                               dirichlet=0.5)
    ref = oracle.solve(mech, T, P, Y, 5e-4, max_iters=20)
    To, Yo, it, st = _solve(mech, T, P, Y, 5e-4, max_iters=20)
    assert (it == ref[2]).all()
    assert np.abs(Yo - ref[1]).max() <= 1e-5
