"""Levenberg-Marquardt training of the thermo network (Sec. 3 fits its
network with LMA): the Jacobian kernel against central differences of the
FP64 reference network, J^T r against the gradient kernel, and the trainer's
convergence from scratch and after Adam."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_1905_09395_b300 import Mechanism, synth
from mechs import isomer_pair

pytestmark = pytest.mark.gpu


def _random_params(n_out, seed):
    rng = np.random.default_rng(seed)
    shp = ref.shapes(n_out)
    return {k: rng.normal(0.0, 0.4, size=shp[k]) for k in ref.ORDER}


def test_jacobian_matches_central_differences():
    m = Mechanism(isomer_pair())               # S = 2: 6 outputs, 4,678 parameters
    n_out = 6
    params = _random_params(n_out, 1)
    flat = ref.flatten(params)
    T = np.array([450.0, 1500.0, 2800.0])
    J = m.mlp_jacobian(flat.astype(np.float32), T).astype(np.float64)
    p32 = flat.astype(np.float32).astype(np.float64)    # the kernel's parameters
    h = 1e-4
    fd = np.zeros_like(J)
    for k in range(len(p32)):
        up, dn = p32.copy(), p32.copy()
        up[k] += h
        dn[k] -= h
        yu, _ = ref.forward(ref.unflatten(up, n_out), T)
        yd, _ = ref.forward(ref.unflatten(dn, n_out), T)
        fd[:, k] = ((yu - yd) / (2 * h)).ravel()          # row = sample * n_out + output
    err = np.abs(J - fd)
    assert err.max() <= 1e-4 * np.abs(fd).max() + 1e-5, err.max()
    # the output layer's block is exact: a2 in its own output's row, zeros elsewhere
    off_W3 = 64 + 64 + 64 * 64 + 64
    assert np.all(J[1, off_W3:off_W3 + 64] == 0.0)        # sample 0, output 1: W3 row 0
    m.close()


def test_jacobian_times_residual_is_the_gradient():
    # 2/(N M) J^T r from the Jacobian kernel == the training kernel's gradient
    mech = synth.small_mechanism()
    m = Mechanism(mech)
    n_out = 3 * mech.n_species
    params = ref.flatten(_random_params(n_out, 2)).astype(np.float32)
    T = np.random.default_rng(3).uniform(300.0, 3000.0, size=64)
    target = np.random.default_rng(4).normal(size=(64, n_out)).astype(np.float32)
    J = m.mlp_jacobian(params, T).astype(np.float64)
    y, _ = ref.forward(ref.unflatten(params.astype(np.float64), n_out), T)
    r = (y - target).ravel()
    g_lm = 2.0 * J.T @ r / r.size
    _, g = m.mlp_loss_grad(params, T, target)
    big = np.abs(g_lm) > 1e-3 * np.abs(g_lm).max()
    assert np.all(np.abs(g[big] - g_lm[big]) <= 1e-3 * np.abs(g_lm[big]) + 1e-6)
    m.close()


def test_lm_converges_from_scratch():
    mech = synth.small_mechanism()
    m = Mechanism(mech)
    Ts = np.random.default_rng(5).uniform(300.0, 3000.0, size=20_000)
    hist = m.mlp_train_lm(Ts, iterations=25, batch=512, lambda0=1e-2, init=0, seed=3)
    print("LM loss:", np.array2string(hist, precision=2))
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 1e-2 * hist[:3].max()
    assert hist[-1] < 1e-3
    m.close()


def test_lm_continues_after_adam():
    mech = synth.small_mechanism()
    m = Mechanism(mech)
    Ts = np.random.default_rng(6).uniform(300.0, 3000.0, size=100_000)
    adam = m.mlp_train(Ts, epochs=3, batch=4096, lr=2e-3, seed=1)
    hist = m.mlp_train_lm(Ts, iterations=10, batch=1024, lambda0=1e-3, init=1)
    print("Adam %.3g -> LM %s" % (adam[-1], np.array2string(hist, precision=2)))
    assert hist[-1] < 0.5 * adam[-1]
    m.close()
