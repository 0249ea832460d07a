"""The FP64 reference of the thermo network against finite differences and
against its defining properties (its own formulas are not retyped here)."""
import numpy as np
import pytest

from oracle import mlp


def _params(n_out, seed=0, scale=0.5):
    rng = np.random.default_rng(seed)
    return {k: rng.normal(scale=scale, size=s) for k, s in mlp.shapes(n_out).items()}


def test_gradients_match_central_differences():
    n_out = 12
    p = _params(n_out)
    rng = np.random.default_rng(1)
    T = rng.uniform(300, 3000, size=17)
    target = rng.normal(size=(17, n_out))
    loss, g = mlp.loss_and_grads(p, T, target)
    flat = mlp.flatten(p)
    gflat = mlp.flatten(g)
    idx = rng.choice(len(flat), size=60, replace=False)
    for i in idx:
        e = 1e-6 * max(1.0, abs(flat[i]))
        fp, fm = flat.copy(), flat.copy()
        fp[i] += e
        fm[i] -= e
        lp, _ = mlp.loss_and_grads(mlp.unflatten(fp, n_out), T, target)
        lm, _ = mlp.loss_and_grads(mlp.unflatten(fm, n_out), T, target)
        num = (lp - lm) / (2 * e)
        # central-difference rounding is ~eps*loss/e ~ 1e-9 here
        assert abs(num - gflat[i]) <= 1e-6 * abs(num) + 1e-8 * max(loss, 1.0)


def test_forward_is_a_tanh_network_of_scaled_temperature():
    # a network with W3 = identity on the second hidden layer returns a2, whose
    # entries lie in (-1, 1) and are odd in t when all biases vanish
    n_out = mlp.HIDDEN
    p = _params(n_out, seed=3)
    p["b1"][:] = 0
    p["b2"][:] = 0
    p["b3"][:] = 0
    p["W3"] = np.eye(mlp.HIDDEN)
    T = np.array([mlp.T_MID - 700.0, mlp.T_MID + 700.0])
    y, _ = mlp.forward(p, T)
    assert np.all(np.abs(y) < 1)
    np.testing.assert_allclose(y[0], -y[1], rtol=1e-14, atol=1e-15)


def test_zero_loss_at_exact_fit():
    p = _params(6, seed=4)
    T = np.linspace(300, 3000, 11)
    y, _ = mlp.forward(p, T)
    loss, g = mlp.loss_and_grads(p, T, y)
    assert loss == 0.0
    assert all(np.abs(v).max() == 0.0 for v in g.values())
