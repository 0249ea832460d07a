"""Plain FP64 CPU oracle of STEV on the paper's multiphase coal gasification
cells (Sec. 7.2, Eqs. 31-56, Table 2), via ctypes.

TEST INFRASTRUCTURE ONLY, like the rest of oracle/.  The arithmetic lives in
stev_multiphase.c (plain C, one cell at a time, each function citing the
equations it follows, the readings in its header); this module only builds it
and marshals arrays.

A cell is a record of 24 doubles: gas mass fractions X_g[14] (O2 CO CO2 CH4
H2 H2O H2S C3H6 HCN C2H4 C2H6 Tar SO3 N2), solid mass fractions X_s[4] (CV CC
CM CA), T_g, T_s (K), eps_s, rho_s (kg/m^3), d_p (m), P (Pa).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

from . import DEFAULT_OPTS

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stev_multiphase.c")

GAS = ("O2", "CO", "CO2", "CH4", "H2", "H2O", "H2S", "C3H6", "HCN", "C2H4", "C2H6", "Tar", "SO3",
       "N2")
SOLID = ("CV", "CC", "CM", "CA")
SPECIES = GAS + SOLID
REACTIONS = ("PYRO", "WGS", "STG", "CG", "MEG", "COX", "TOX", "COOX", "HOX", "MEOX", "MR")
N_IN = 24
I_TG, I_TS, I_EPS, I_RHOS, I_DP, I_P = 18, 19, 20, 21, 22, 23

# probe builds: every rate constant scaled by 1 +- 1 ulp
PROBES = {"a_up": ["-DORACLE_MP_A_SCALE=(1.0+2.220446049250313e-16)"],
          "a_down": ["-DORACLE_MP_A_SCALE=(1.0-1.1102230246251565e-16)"]}


class _Opts(ctypes.Structure):
    _fields_ = [("y_step_max", ctypes.c_double), ("delta_max", ctypes.c_double),
                ("alpha", ctypes.c_double), ("dft_n", ctypes.c_int),
                ("dft_hi_first", ctypes.c_int), ("tol_ring", ctypes.c_double),
                ("tol_freq", ctypes.c_double), ("r_fac", ctypes.c_double),
                ("rof_min", ctypes.c_double), ("max_iters", ctypes.c_int),
                ("dft_on", ctypes.c_int)]


def _opts(**overrides) -> _Opts:
    d = dict(DEFAULT_OPTS)
    d.update(overrides)
    return _Opts(*[d[k] for k, _ in _Opts._fields_])


_libs = {}


def build(force: bool = False, probe: Optional[str] = None) -> str:
    out = os.path.join(_HERE, "liboracle_mp%s.so" % ("" if probe is None else "_" + probe))
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + ".%d.tmp" % os.getpid()
        defs = [] if probe is None else PROBES[probe]
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               *defs, "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, out)
    return out


def lib(probe: Optional[str] = None):
    if probe not in _libs:
        L = ctypes.CDLL(build(probe=probe))
        P, D = ctypes.c_void_p, ctypes.c_double
        L.mp_solve.argtypes = [P, ctypes.c_long, P, D, P, P, P, P, ctypes.c_int]
        L.mp_get_tables.argtypes = [P, P]
        L.mp_eval_rates.argtypes = [P, P, D, D, D, D, D, P]
        L.mp_initial_state.argtypes = [P, P]
        _libs[probe] = L
    return _libs[probe]


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def tables():
    """(MW[18] kg/kmol, nu[11][18] molar stoichiometry, reactants < 0)."""
    mw, nu = np.zeros(18), np.zeros((11, 18))
    lib().mp_get_tables(_ptr(mw), _ptr(nu))
    return mw, nu


def initial_densities(rec) -> np.ndarray:
    """Partial densities c[18] (kg/m^3) of an input record (rho_g from the
    ideal gas law at P, T_g and the gas's mean molar mass)."""
    rec = np.ascontiguousarray(rec, dtype=np.float64)
    c = np.zeros(18)
    lib().mp_initial_state(_ptr(rec), _ptr(c))
    return c


def rates(c, T_g: float, T_s: float, rho_s: float, d_p: float, P: float, **opts) -> np.ndarray:
    """Raw rates of progress r[11] (kmol/m^3/s) of Eqs. 42-56 at partial
    densities c[18]."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    r = np.zeros(11)
    o = _opts(**opts)
    lib().mp_eval_rates(ctypes.byref(o), _ptr(c), float(T_g), float(T_s), float(rho_s),
                        float(d_p), float(P), _ptr(r))
    return r


def solve(cells, dt: float, n_threads: Optional[int] = None, probe: Optional[str] = None,
          **opts):
    """All cells ([n][24] records): (out [n][24], rho_g [n], iters, status)."""
    cells = np.ascontiguousarray(cells, dtype=np.float64).reshape(-1, N_IN)
    n = len(cells)
    out, rho_g = np.zeros((n, N_IN)), np.zeros(n)
    iters, status = np.zeros(n, np.int32), np.zeros(n, np.uint8)
    if n == 0:
        return out, rho_g, iters, status
    nt = max(1, min(int(n_threads or os.cpu_count() or 1), n))
    o = _opts(**opts)
    lib(probe).mp_solve(ctypes.byref(o), n, _ptr(cells), float(dt), _ptr(out), _ptr(rho_g),
                        _ptr(iters), _ptr(status), nt)
    return out, rho_g, iters, status


def conditioning(cells, dt: float, base=None, **opts):
    """(base, dX spread [n], eps_s spread [n]) under every rate constant
    changed by one ulp (probe builds a_up, a_down)."""
    if base is None:
        base = solve(cells, dt, **opts)
    dX = np.zeros(len(base[0]))
    de = np.zeros(len(base[0]))
    for p in PROBES:
        r = solve(cells, dt, probe=p, **opts)
        dX = np.maximum(dX, np.abs(r[0][:, :18] - base[0][:, :18]).max(axis=1))
        de = np.maximum(de, np.abs(r[0][:, I_EPS] - base[0][:, I_EPS]))
    return base, dX, de
