"""FP64 reference of the thermo network (test infrastructure only).

Sec. 3 of the paper replaces the NASA-7 evaluation of species properties by a
small neural network of temperature.  This is the network the library trains
and evaluates on the GPU, written out plainly in numpy float64 so that tests
can check the GPU's forward pass, loss and gradients against it:

    t  = (T - T_mid) / T_half                     input scaling
    a1 = tanh(W1 t + b1)                          64
    a2 = tanh(W2 a1 + b2)                         64
    y  = W3 a2 + b3                               3S standardised outputs
    loss = mean over samples and outputs of (y - target)^2

Targets are the polynomial values (cp/R, H/R = H/RT * T in kelvin, S/R of
every species, in that order) standardised per output column:
(value - mean) / std.  Parameters are
a dict of arrays W1 [64][1], b1 [64], W2 [64][64], b2 [64], W3 [3S][64],
b3 [3S] (rows = outputs), flattened in that order when passed around.
"""
from __future__ import annotations

import numpy as np

T_MID, T_HALF = 1650.0, 1350.0      # the training range 300-3000 K maps to [-1, 1]
HIDDEN = 64
ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def shapes(n_out: int):
    return {"W1": (HIDDEN, 1), "b1": (HIDDEN,), "W2": (HIDDEN, HIDDEN), "b2": (HIDDEN,),
            "W3": (n_out, HIDDEN), "b3": (n_out,)}


def flatten(params) -> np.ndarray:
    return np.concatenate([np.asarray(params[k], dtype=np.float64).ravel() for k in ORDER])


def unflatten(flat, n_out: int):
    out, o = {}, 0
    for k in ORDER:
        shp = shapes(n_out)[k]
        size = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + size], dtype=np.float64).reshape(shp)
        o += size
    return out


def forward(params, T):
    """Standardised outputs y [n][n_out] and the activations for backward."""
    t = ((np.asarray(T, dtype=np.float64) - T_MID) / T_HALF)[:, None]
    a1 = np.tanh(t @ params["W1"].T + params["b1"])
    a2 = np.tanh(a1 @ params["W2"].T + params["b2"])
    y = a2 @ params["W3"].T + params["b3"]
    return y, (t, a1, a2)


def loss_and_grads(params, T, target):
    """Mean squared error and its gradient with respect to every parameter."""
    y, (t, a1, a2) = forward(params, T)
    n, m = y.shape
    d = y - target
    loss = float(np.mean(d * d))
    dy = 2.0 * d / (n * m)
    g = {"W3": dy.T @ a2, "b3": dy.sum(axis=0)}
    da2 = dy @ params["W3"]
    dz2 = da2 * (1.0 - a2 * a2)
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(axis=0)
    da1 = dz2 @ params["W2"]
    dz1 = da1 * (1.0 - a1 * a1)
    g["W1"] = dz1.T @ t
    g["b1"] = dz1.sum(axis=0)
    return loss, g
