"""Mixed precision with the thermo network (Sec. 3, "MLA-STEV"): accuracy
against the FP64 oracle and what the network gains over the polynomials.

THERMO_MLP takes cp/R from the network (inside its 300-3000 K training range),
THERMO_MLP_CPH also H/RT; G/RT for the equilibrium constants stays on the FP64
polynomials, whose precision Eq. 30 needs (a BF16 network's ~1e-3 error in
G/RT would move every equilibrium by ~0.1%).  Errors in H/RT shift the heat
release, hence T, hence every Arrhenius rate, so the cp-only mode is the one
held to the mixed-precision target; the cp+H mode is measured and reported."""
import time

import numpy as np
import pytest

import oracle
from paper_1905_09395_b300 import MIXED, THERMO_MLP, THERMO_MLP_CPH, Mechanism, synth
from test_gpu_mixed import TOL_T, TOL_Y, _check, _small_conditioning

pytestmark = pytest.mark.gpu


def _trained(mech, n=200_000, epochs=15, **opts):
    m = Mechanism(mech, precision=MIXED, **opts)
    T = np.random.default_rng(11).uniform(300.0, 3000.0, size=n)
    hist = m.mlp_train(T, epochs=epochs, batch=4096, lr=2e-3, seed=3)
    return m, hist


def _run(m, T, P, Y, dt):
    import torch
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (T, P, Y)]
    return tuple(x.cpu().numpy() for x in m.solve(*d, dt))


def test_mixed_mlp_small_case():
    mech, T, P, Y, dt = synth.small_case(2048)
    m, hist = _trained(mech, n=1_000_000, epochs=30)
    assert hist[-1] < 1e-3
    ref, sY, sT = _small_conditioning()
    # cp+H: measured and reported only
    m.set_options(thermo=THERMO_MLP_CPH)
    To, Yo, it, st = _run(m, T, P, Y, dt)
    dY = np.abs(Yo - ref[1]).max(axis=1)
    dT = np.abs(To - ref[0])
    print("mixed+MLP(cp, H) 8/20 x 2048: within 1e-4 / 0.5 K %.3f, median dT %.3g K, max dT %.3g K"
          % (np.mean((dY <= TOL_Y) & (dT <= TOL_T)), np.median(dT), dT.max()))
    # cp only: the mixed target on well-conditioned cells.  The network's cp
    # error (BF16 weights and activations: ~0.05% mean) is systematic, so a
    # few cells that rounding leaves alone still move by slightly more than
    # 1e-4; at most 2% of them may, and none by more than 3e-4 / 0.5 K.
    m.set_options(thermo=THERMO_MLP)
    within = _check(mech, T, Y, _run(m, T, P, Y, dt), ref, sY, sT, "mixed+MLP(cp) 8/20 x 2048",
                    outliers=0.02, outlier_cap=(3e-4, TOL_T))
    assert within > 0.9
    assert m.mlp_stalls == 0   # every network answer arrived within its bounded wait
    m.close()


def test_mlp_needs_training_first():
    from paper_1905_09395_b300 import StevError
    import torch
    mech, T, P, Y, dt = synth.small_case(8)
    m = Mechanism(mech, precision=MIXED, thermo=THERMO_MLP)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (T, P, Y)]
    with pytest.raises(StevError, match="trained network"):
        m.solve(*d, dt)
    m.close()


def test_network_gain_over_polynomials():
    """What the network gains: the same cells, the same kernel structure,
    cp/R from the network against the polynomials.  Throughput is compared on
    131,072 cells capped at 1,500 steps (every resident slot busy, no tail of
    long cells); accuracy on full solves of 8,192 cells.

    The network replaces five FP32 FMAs of polynomial per species and costs
    each warp 24 tensor-core MMAs, 32 weight-fragment loads and ~10 tanh per
    step: with one cell per warp (this 32-species mechanism) it runs at 0.77x
    the polynomial kernel's cell-steps/s (measured on B300), with four cells
    per warp sharing the MMAs (the 8-species mechanism,
    test_network_gain_with_four_cells_per_warp) at 0.99x.  The bounds below
    are those measurements less a margin for run-to-run noise."""
    import torch
    mech, T, P, Y, dt = synth.scale_case(131072)
    m, _ = _trained(mech, n=400_000, epochs=15)
    modes = {"poly": 0, "net": THERMO_MLP, "net_cph": THERMO_MLP_CPH}
    rate = {}
    m.set_options(max_iters=1500)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (T, P, Y)]
    for mode in ("poly", "net", "net_cph", "poly", "net", "net_cph"):
        m.set_options(thermo=modes[mode])
        torch.cuda.synchronize()
        t0 = time.time()
        out = m.solve(*d, dt)
        torch.cuda.synchronize()
        el = time.time() - t0
        rate[mode] = float(out[2].sum().item()) / el      # cell-steps/s (second run kept)
    m.set_options(max_iters=200000)
    n = 8192
    d = [x[:n] for x in d]
    outs = {}
    for mode in ("poly", "net"):
        m.set_options(thermo=modes[mode])
        outs[mode] = [x.cpu().numpy() for x in m.solve(*d, dt)]
    gain = rate["net"] / rate["poly"]
    dY = np.abs(outs["net"][1] - outs["poly"][1]).max(axis=1)
    dT = np.abs(outs["net"][0] - outs["poly"][0])
    print("network (cp) vs polynomial thermo, syn32x150: %.3g vs %.3g cell-steps/s (gain %.3fx;"
          " cp+H %.3g); cells within 1e-4 / 0.5 K of the polynomial run: %.3f, median dT %.3g K"
          % (rate["net"], rate["poly"], gain, rate["net_cph"],
             np.mean((dY <= TOL_Y) & (dT <= TOL_T)), np.median(dT)))
    assert (outs["net"][3] == 0).all()
    assert m.mlp_stalls == 0
    assert 0.7 <= gain <= 1.1
    m.close()


def test_network_gain_with_four_cells_per_warp():
    """The 8-species mechanism (lane groups of 8, four cells per warp sharing
    each MMA): the network costs about nothing against the polynomials."""
    import torch
    mech = synth.small_mechanism()
    T, P, Y = synth.make_cells(mech, 1 << 19, seed=0, T_range=(1200.0, 1800.0),
                               P_atm_range=(1.0, 1.0), dirichlet=1.0)
    m, _ = _trained(mech, n=400_000, epochs=15)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (T, P, Y)]
    rate = {}
    for mode in ("poly", "net", "poly", "net"):
        m.set_options(thermo=THERMO_MLP if mode == "net" else 0)
        torch.cuda.synchronize()
        t0 = time.time()
        out = m.solve(*d, 1e-3)
        torch.cuda.synchronize()
        rate[mode] = float(out[2].sum().item()) / (time.time() - t0)
    gain = rate["net"] / rate["poly"]
    print("network vs polynomial thermo, syn8x20 (4 cells per warp): gain %.3fx" % gain)
    assert 0.9 <= gain <= 1.1
    m.close()
