"""Stability diagnostics of the oracle's integration (Sec. 4, Eqs. 19-25).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: reported, not gated.

Sec. 4 linearises the cell ODE X' = f(X) of Eq. 17 (X = the mass fractions
and the temperature) around the current state, A = df/dX (Eqs. 20-23), and
bounds the forward-Euler step by the infinity norm of A (Eq. 24); Eq. 25
compares STEV's own step h (Eqs. 1-5) with that bound.  Here:

  jacobian_fd      A by central finite differences of the oracle's right-hand
                   side (undamped rates, rOF = 1), the column of X_j from a
                   step of 1e-6 |X_j| (at least 1e-12 for a mass fraction);
  eq25_report      along a cell's STEV trajectory, the fraction of steps with
                   h ||A||_inf <= 2 (Eq. 25) and with h rho(A) <= 2 (the
                   spectral form of Eq. 24), on a sample of the steps;
  spectral_ratio   the stiffness of a state: the largest over the smallest
                   nonzero |eigenvalue| of A (eigenvalues below 1e-9 of the
                   largest are the conservation laws' zero modes and are left
                   out), with rho(A).

tests/test_oracle_stability.py pins these against closed forms and prints the
report quoted in the design notes.
"""
from __future__ import annotations

import numpy as np

from . import rates, solve_cell_trace


def rhs(mech, T: float, P: float, Y, **opts) -> np.ndarray:
    """f(X) of Eq. 17 with undamped rates: (dY/dt, dT/dt)."""
    r = rates(mech, T, P, Y, **opts)
    return np.append(r["dYdt"], r["dTdt"])


def jacobian_fd(mech, T: float, P: float, Y, rel: float = 1e-6, y_floor: float = 1e-12,
                **opts) -> np.ndarray:
    """A = df/dX at X = (Y, T) (Eq. 23) by central differences."""
    Y = np.asarray(Y, dtype=np.float64)
    S = len(Y)
    X = np.append(Y, T)
    A = np.zeros((S + 1, S + 1))
    for j in range(S + 1):
        d = rel * abs(X[j]) if j == S else max(rel * abs(X[j]), y_floor)
        up, dn = X.copy(), X.copy()
        up[j] += d
        dn[j] -= d
        A[:, j] = (rhs(mech, up[S], P, up[:S], **opts) - rhs(mech, dn[S], P, dn[:S], **opts)) / (2 * d)
    return A


def spectral_ratio(mech, T: float, P: float, Y, **opts):
    """(stiffness ratio max|lambda| / min nonzero |lambda|, rho(A), ||A||_inf)."""
    A = jacobian_fd(mech, T, P, Y, **opts)
    lam = np.abs(np.linalg.eigvals(A))
    rho = lam.max()
    nz = lam[lam > 1e-9 * rho]
    return rho / nz.min(), rho, np.abs(A).sum(axis=1).max()


def eq25_report(mech, T0: float, P: float, Y0, dt: float, samples: int = 200, **opts) -> dict:
    """Eq. 25 along one cell's STEV trajectory (the oracle's), on up to
    `samples` evenly spaced steps: fractions of steps with h ||A||_inf <= 2
    and with h rho(A) <= 2, and the largest h rho(A) seen."""
    tr = solve_cell_trace(mech, T0, P, Y0, dt, **opts)
    n = len(tr["h"])
    idx = np.unique(np.linspace(0, n - 1, min(samples, n)).astype(int))
    ok_inf, ok_rho, worst = 0, 0, 0.0
    rate_opts = {k: v for k, v in opts.items() if k == "alpha"}
    for k in idx:
        A = jacobian_fd(mech, tr["T_trace"][k], P, tr["Y_trace"][k], **rate_opts)
        h = tr["h"][k]
        norm_inf = np.abs(A).sum(axis=1).max()
        rho = np.abs(np.linalg.eigvals(A)).max()
        ok_inf += h * norm_inf <= 2.0
        ok_rho += h * rho <= 2.0
        worst = max(worst, h * rho)
    return {"steps": int(n), "sampled": int(len(idx)), "frac_eq25_inf": ok_inf / len(idx),
            "frac_eq25_rho": ok_rho / len(idx), "max_h_rho": float(worst)}
