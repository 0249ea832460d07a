"""The thermo network (Sec. 3) on the GPU: gradients against the FP64
reference, training, tensor-core inference, and accuracy against the NASA-7
polynomials that generate its training data."""
import numpy as np
import pytest

import oracle
from oracle import mlp as ref
from paper_1905_09395_b300 import Mechanism, synth

pytestmark = pytest.mark.gpu


def _random_params(n_out, seed=0):
    rng = np.random.default_rng(seed)
    p = {k: rng.normal(scale=0.4, size=s) for k, s in ref.shapes(n_out).items()}
    return ref.flatten(p)


def test_gradients_match_fp64_reference():
    mech = synth.small_mechanism()
    m = Mechanism(mech)
    n_out = 3 * mech.n_species
    flat = _random_params(n_out).astype(np.float32)
    rng = np.random.default_rng(1)
    T = rng.uniform(300, 3000, size=300)
    target = rng.normal(size=(300, n_out)).astype(np.float32)
    loss_g, grad_g = m.mlp_loss_grad(flat, T, target)
    loss_r, g_r = ref.loss_and_grads(ref.unflatten(flat.astype(np.float64), n_out), T,
                                     target.astype(np.float64))
    grad_r = ref.flatten(g_r)
    assert loss_g == pytest.approx(loss_r, rel=1e-5)
    rel = np.linalg.norm(grad_g - grad_r) / np.linalg.norm(grad_r)
    assert rel <= 1e-3, rel
    big = np.abs(grad_r) > 1e-3 * np.abs(grad_r).max()
    assert np.all(np.abs(grad_g[big] - grad_r[big]) <= 1e-3 * np.abs(grad_r[big]) + 1e-6)
    m.close()


def test_training_is_reproducible():
    # gradients are summed over tiles in a fixed order: same inputs, same network
    mech = synth.small_mechanism()
    T = np.random.default_rng(3).uniform(300.0, 3000.0, size=100_000)
    runs = []
    for _ in range(2):
        m = Mechanism(mech)
        hist = m.mlp_train(T, epochs=3, batch=4096, lr=2e-3, seed=5)
        runs.append((hist, m.mlp_params()))
        m.close()
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for a, b in zip(runs[0][1], runs[1][1]):
        np.testing.assert_array_equal(a, b)


@pytest.fixture(scope="module")
def trained():
    mech = synth.scale_mechanism()
    m = Mechanism(mech)
    T = np.random.default_rng(2024).uniform(300.0, 3000.0, size=1_000_000)
    hist = m.mlp_train(T, epochs=30, batch=4096, lr=2e-3, seed=7)
    yield mech, m, hist
    m.close()


def test_training_converges(trained):
    mech, m, hist = trained
    print("loss per epoch:", np.array2string(hist, precision=2))
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 0.05 * hist[0]
    assert hist[-1] < 2e-3


def test_inference_matches_fp64_forward(trained):
    # tensor-core BF16 inference against the FP64 network with the same weights
    import torch
    mech, m, _ = trained
    p, mu, sd = m.mlp_params()
    n_out = 3 * mech.n_species
    T = np.linspace(300.0, 3000.0, 1003)
    got = m.mlp_eval(torch.from_numpy(T).cuda()).cpu().numpy()
    y, _ = ref.forward(ref.unflatten(p.astype(np.float64), n_out), T)
    want = y * sd + mu
    err = np.abs(got - want) / sd      # in units of each output's spread
    assert err.max() < 0.05, err.max()
    assert err.mean() < 0.01


def test_accuracy_against_polynomials(trained):
    # the paper's check (Fig. 3): network vs polynomial over the range
    import torch
    mech, m, _ = trained
    S = mech.n_species
    T = np.random.default_rng(5).uniform(300.0, 3000.0, size=4000)
    got = m.mlp_eval(torch.from_numpy(T).cuda()).cpu().numpy()
    want = np.array([np.concatenate(oracle.thermo(mech, t)) for t in T])
    want[:, S:2 * S] *= T[:, None]           # the network's second block is H/R (K)
    cp_rel = np.abs(got[:, :S] - want[:, :S]) / np.abs(want[:, :S])
    h_abs = np.abs(got[:, S:2 * S] - want[:, S:2 * S]) / T[:, None]   # back to H/RT units
    s_abs = np.abs(got[:, 2 * S:] - want[:, 2 * S:])
    print("cp/R relative error: max %.3f%%, mean %.3f%%; H/RT abs max %.3g mean %.3g;"
          " S/R abs max %.3g mean %.3g" % (100 * cp_rel.max(), 100 * cp_rel.mean(), h_abs.max(),
                                           h_abs.mean(), s_abs.max(), s_abs.mean()))
    assert cp_rel.mean() < 0.01
    assert cp_rel.max() < 0.1
