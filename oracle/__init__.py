"""Plain FP64 CPU oracle of the STEV solver (arXiv:1905.09395), via ctypes.

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline leg may use it; the product path never does.  It imports nothing
from the product package; a mechanism is any object carrying the table
attributes (mol_weight, nasa7, t_range, rxn_ptr, rxn_species, rxn_nu, A, beta,
Ea, reversible).

The arithmetic lives in stev_oracle.c (plain C, one cell at a time, every
function citing the equation it follows); this module only marshals arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stev_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

DEFAULT_OPTS = dict(
    y_step_max=1e-3,   # Y_step^max (Eq. 3), mass fraction per step
    delta_max=0.01,    # delta^max (Eq. 4)
    alpha=1e-5,        # Eq. 7
    dft_n=13,          # N, the stored history length (Sec. 2.3)
    dft_hi_first=4,    # n, first high-frequency bin (Eq. 10)
    tol_ring=0.5,      # Tol_ring (Eq. 12)
    tol_freq=1e-6,     # Tol_freq (Eq. 12), mol/m^3
    r_fac=2.0,         # r_fac (Eq. 12)
    rof_min=1e-30,     # keeps rOF > 0
    max_iters=200000,  # per-cell cap
    dft_on=1,
)

CELL_OK, CELL_MAXITER, CELL_NONFINITE, CELL_TRANGE = 0, 1, 2, 3


class _Mech(ctypes.Structure):
    _fields_ = [
        ("n_species", ctypes.c_int), ("n_reactions", ctypes.c_int),
        ("mol_weight", ctypes.c_void_p), ("nasa7", ctypes.c_void_p),
        ("t_range", ctypes.c_void_p), ("rxn_ptr", ctypes.c_void_p),
        ("rxn_species", ctypes.c_void_p), ("rxn_nu", ctypes.c_void_p),
        ("A", ctypes.c_void_p), ("beta", ctypes.c_void_p), ("Ea", ctypes.c_void_p),
        ("reversible", ctypes.c_void_p), ("rxn_order", ctypes.c_void_p),
    ]


class _Opts(ctypes.Structure):
    _fields_ = [
        ("y_step_max", ctypes.c_double), ("delta_max", ctypes.c_double),
        ("alpha", ctypes.c_double), ("dft_n", ctypes.c_int), ("dft_hi_first", ctypes.c_int),
        ("tol_ring", ctypes.c_double), ("tol_freq", ctypes.c_double),
        ("r_fac", ctypes.c_double), ("rof_min", ctypes.c_double),
        ("max_iters", ctypes.c_int), ("dft_on", ctypes.c_int),
    ]


# conditioning-probe builds: every kf scaled by one ulp (1 + 2^-52, 1 - 2^-53),
# or every K by 64 ulp (1 +- 2^-46), the size of the rounding error of dG/RT
PROBES = {"kf_up": ["-DORACLE_KF_SCALE=(1.0+2.220446049250313e-16)"],
          "kf_down": ["-DORACLE_KF_SCALE=(1.0-1.1102230246251565e-16)"],
          "K_up": ["-DORACLE_K_SCALE=(1.0+1.4210854715202004e-14)"],
          "K_down": ["-DORACLE_K_SCALE=(1.0-1.4210854715202004e-14)"],
          # single-precision-sized changes: kf by 2^-22, K by 2^-18
          "kf32_up": ["-DORACLE_KF_SCALE=(1.0+2.384185791015625e-07)"],
          "kf32_down": ["-DORACLE_KF_SCALE=(1.0-2.384185791015625e-07)"],
          "K32_up": ["-DORACLE_K_SCALE=(1.0+3.814697265625e-06)"],
          "K32_down": ["-DORACLE_K_SCALE=(1.0-3.814697265625e-06)"],
          # concentrations or net rates rounded to float every step
          "round32_C": ["-DORACLE_ROUND32_C"],
          "round32_q": ["-DORACLE_ROUND32_Q"],
          # every reverse term times (1 + 2^-22 xi), xi a hash in [-1, 1): no
          # equilibrium cancels exactly (two seeds)
          "qnoise32_a": ["-DORACLE_Q_NOISE=2.384185791015625e-07", "-DORACLE_Q_NOISE_SEED=1"],
          "qnoise32_b": ["-DORACLE_Q_NOISE=2.384185791015625e-07", "-DORACLE_Q_NOISE_SEED=2"],
          # real-order powers C^a (global rate laws) changed by 4 ulp (math
          # libraries' pow differ by a few ulp), or by 2^-17 (a single-precision
          # 2^(a lg2 C) with |a lg2 C| up to ~32)
          "pow_up": ["-DORACLE_POW_SCALE=(1.0+8.881784197001252e-16)"],
          "pow_down": ["-DORACLE_POW_SCALE=(1.0-8.881784197001252e-16)"],
          "pow32_up": ["-DORACLE_POW_SCALE=(1.0+7.62939453125e-06)"],
          "pow32_down": ["-DORACLE_POW_SCALE=(1.0-7.62939453125e-06)"]}
PROBE_LEVELS = {"fp64": ("kf_up", "kf_down", "K_up", "K_down"),
                "fp32": ("kf32_up", "kf32_down", "K32_up", "K32_down", "round32_C",
                         "round32_q", "qnoise32_a", "qnoise32_b")}
# probes that only matter for mechanisms with real reaction orders
POW_PROBES = {"fp64": ("pow_up", "pow_down"), "fp32": ("pow32_up", "pow32_down")}
# single-precision-sized changes of the thresholds that take discrete
# decisions (the limiter's Y_step^max, the ringing tolerances of Eq. 12)
OPTION_PROBES = {"fp64": (), "fp32": ("y_step_max", "tol_freq", "tol_ring")}


def _lib_path(probe: Optional[str]) -> str:
    return _LIB if probe is None else os.path.join(_HERE, "liboracle_%s.so" % probe)


def build(force: bool = False, probe: Optional[str] = None) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    out = _lib_path(probe)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + ".%d.tmp" % os.getpid()
        defs = [] if probe is None else PROBES[probe]
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               *defs, "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, out)
    return out


_libs = {}


def lib(probe: Optional[str] = None):
    if probe not in _libs:
        _lib = ctypes.CDLL(build(probe=probe))
        P = ctypes.c_void_p
        _lib.oracle_thermo.argtypes = [P, ctypes.c_double, P, P, P]
        _lib.oracle_rates.argtypes = [P, P, ctypes.c_double, ctypes.c_double, P, P, P, P, P, P]
        _lib.oracle_step_size.argtypes = [ctypes.c_int, P, P, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double]
        _lib.oracle_step_size.restype = ctypes.c_double
        _lib.oracle_dft_mag.argtypes = [P, ctypes.c_int, ctypes.c_int]
        _lib.oracle_dft_mag.restype = ctypes.c_double
        _lib.oracle_ring_update.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double]
        _lib.oracle_ring_update.restype = ctypes.c_double
        _lib.oracle_solve_cell_trace.argtypes = [P, P, ctypes.c_double, ctypes.c_double, P,
                                                 ctypes.c_double, P, P, P, ctypes.c_int, P, P, P]
        _lib.oracle_solve_cell_trace.restype = ctypes.c_int
        _lib.oracle_solve.argtypes = [P, P, ctypes.c_long, P, P, P, ctypes.c_double, P, P, P, P,
                                      ctypes.c_int]
        _libs[probe] = _lib
    return _libs[probe]


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleMechanism:
    """Holds contiguous copies of a mechanism's tables and the C struct."""

    def __init__(self, mech):
        self.S = int(np.asarray(mech.mol_weight).shape[0])
        self.R = int(np.asarray(mech.A).shape[0])
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        self._arrays = dict(
            mol_weight=f64(mech.mol_weight), nasa7=f64(mech.nasa7), t_range=f64(mech.t_range),
            rxn_ptr=np.ascontiguousarray(mech.rxn_ptr, dtype=np.int32),
            rxn_species=np.ascontiguousarray(mech.rxn_species, dtype=np.int32),
            rxn_nu=f64(mech.rxn_nu), A=f64(mech.A), beta=f64(mech.beta), Ea=f64(mech.Ea),
            reversible=np.ascontiguousarray(mech.reversible, dtype=np.uint8))
        order = getattr(mech, "rxn_order", None)
        if order is not None:
            self._arrays["rxn_order"] = f64(order)
        a = self._arrays
        self.struct = _Mech(self.S, self.R, *(_ptr(a[k]) for k in (
            "mol_weight", "nasa7", "t_range", "rxn_ptr", "rxn_species", "rxn_nu", "A", "beta",
            "Ea", "reversible")), _ptr(a["rxn_order"]) if "rxn_order" in a else None)

    @property
    def ref(self):
        return ctypes.byref(self.struct)


def make_opts(**overrides) -> _Opts:
    d = dict(DEFAULT_OPTS)
    for k, v in overrides.items():
        if k not in d:
            raise KeyError(k)
        d[k] = v
    return _Opts(float(d["y_step_max"]), float(d["delta_max"]), float(d["alpha"]),
                 int(d["dft_n"]), int(d["dft_hi_first"]), float(d["tol_ring"]),
                 float(d["tol_freq"]), float(d["r_fac"]), float(d["rof_min"]),
                 int(d["max_iters"]), int(d["dft_on"]))


def _om(mech) -> OracleMechanism:
    return mech if isinstance(mech, OracleMechanism) else OracleMechanism(mech)


def thermo(mech, T: float):
    """(cp/R, H/RT, S/R) per species at T (Eqs. 15-16)."""
    om = _om(mech)
    cp, h, s = (np.zeros(om.S) for _ in range(3))
    lib().oracle_thermo(om.ref, float(T), _ptr(cp), _ptr(h), _ptr(s))
    return cp, h, s


def rates(mech, T: float, P: float, Y, rOF=None, **opts):
    """Right-hand side of the cell ODE: dict(qraw, wdot, dYdt, dTdt)."""
    om = _om(mech)
    o = make_opts(**opts)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    rOF = np.ones(om.R) if rOF is None else np.ascontiguousarray(rOF, dtype=np.float64)
    q, w, dy = np.zeros(om.R), np.zeros(om.S), np.zeros(om.S)
    dT = ctypes.c_double(0.0)
    lib().oracle_rates(om.ref, ctypes.byref(o), float(T), float(P), _ptr(Y), _ptr(rOF), _ptr(q),
                       _ptr(w), _ptr(dy), ctypes.addressof(dT))
    return dict(qraw=q, wdot=w, dYdt=dy, dTdt=dT.value)


def step_size(Y, dYdt, t_f, y_step_max=DEFAULT_OPTS["y_step_max"],
              delta_max=DEFAULT_OPTS["delta_max"]) -> float:
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    dYdt = np.ascontiguousarray(dYdt, dtype=np.float64)
    return lib().oracle_step_size(len(Y), _ptr(Y), _ptr(dYdt), float(t_f), float(y_step_max),
                                  float(delta_max))


def dft_mag(x, j: int) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().oracle_dft_mag(_ptr(x), len(x), int(j))


def ring_update(x, rOF: float, **opts) -> float:
    d = dict(DEFAULT_OPTS)
    d.update(opts)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().oracle_ring_update(_ptr(x), len(x), int(d["dft_hi_first"]), float(rOF),
                                    float(d["tol_ring"]), float(d["tol_freq"]),
                                    float(d["r_fac"]), float(d["rof_min"]))


def solve_cell_trace(mech, T0: float, P: float, Y0, dt: float, trace_cap: int = 100000, **opts):
    """One cell with its per-step trace (h, T, Y at the start of each step)."""
    om = _om(mech)
    o = make_opts(**opts)
    Y0 = np.ascontiguousarray(Y0, dtype=np.float64)
    Yo = np.zeros(om.S)
    To = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    cap = max(int(trace_cap), 1)
    th, tT, tY = np.zeros(cap), np.zeros(cap), np.zeros((cap, om.S))
    st = lib().oracle_solve_cell_trace(om.ref, ctypes.byref(o), float(T0), float(P), _ptr(Y0),
                                       float(dt), ctypes.addressof(To), _ptr(Yo),
                                       ctypes.addressof(it), int(trace_cap), _ptr(th), _ptr(tT),
                                       _ptr(tY))
    n = min(it.value, int(trace_cap))
    return dict(T=To.value, Y=Yo, iters=it.value, status=st, h=th[:n], T_trace=tT[:n],
                Y_trace=tY[:n])


def solve(mech, T, P, Y, dt: float, n_threads: Optional[int] = None,
          probe: Optional[str] = None, **opts):
    """All cells: returns (T_out, Y_out, iters, status).

    probe names one of the conditioning-probe builds in PROBES."""
    om = _om(mech)
    o = make_opts(**opts)
    T = np.ascontiguousarray(T, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(len(T), om.S)
    n = len(T)
    To, Yo = np.zeros(n), np.zeros((n, om.S))
    iters, status = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.uint8)
    if n == 0:
        return To, Yo, iters, status
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    n_threads = max(1, min(int(n_threads), n))
    lib(probe).oracle_solve(om.ref, ctypes.byref(o), n, _ptr(T), _ptr(P), _ptr(Y), float(dt), _ptr(To),
                       _ptr(Yo), _ptr(iters), _ptr(status), n_threads)
    return To, Yo, iters, status


def conditioning(mech, T, P, Y, dt: float, base=None, n_threads: Optional[int] = None,
                 level: str = "fp64", per_run: Optional[dict] = None, **opts):
    """Per-cell spread of the final state under rounding-size rate changes.

    Returns (base_result, dY_spread[cells], dT_spread[cells]): the largest
    |change| of Y (over species) and of T between the default build and the
    probe builds of the given level: "fp64" changes every kf by one ulp and
    every K by 64 ulp; "fp32" by 2^-22 and 2^-18, the size of the rounding
    of a single-precision rate and of its exponent, rounds every
    concentration or every net rate to float, perturbs every reverse term by
    a hashed relative 2^-22 (so that no equilibrium cancels exactly, as none
    does with FP32 rates), and moves the limiter's
    Y_step^max and the ringing tolerances by 2^-22; for mechanisms with real
    reaction orders also every power C^a by 4 ulp ("fp64") or 2^-17
    ("fp32").  A cell whose spread is far below a tolerance is
    well-conditioned at that tolerance.  per_run (a dict), if given,
    receives each probe run's own per-cell |change| of Y and T under the run's
    name."""
    if base is None:
        base = solve(mech, T, P, Y, dt, n_threads=n_threads, **opts)
    dY = np.zeros(len(T))
    dT = np.zeros(len(T))
    runs = [dict(probe=p) for p in PROBE_LEVELS[level]]
    order = getattr(mech, "rxn_order", None)
    real_orders = np.concatenate([np.abs(np.asarray(mech.rxn_nu, dtype=float)),
                                  np.asarray(order if order is not None else [], dtype=float)])
    if np.any(real_orders != np.round(real_orders)):
        runs += [dict(probe=p) for p in POW_PROBES[level]]
    for name in OPTION_PROBES[level]:
        v = opts.get(name, DEFAULT_OPTS[name])
        runs += [{name: v * (1.0 + 2.0 ** -22)}, {name: v * (1.0 - 2.0 ** -22)}]
    for extra in runs:
        kw = dict(opts)
        kw.update(extra)
        r = solve(mech, T, P, Y, dt, n_threads=n_threads, **kw)
        eY = np.abs(r[1] - base[1]).max(axis=1)
        eT = np.abs(r[0] - base[0])
        dY = np.maximum(dY, eY)
        dT = np.maximum(dT, eT)
        if per_run is not None:
            name = extra.get("probe")
            if name is None:
                opt, v = next(iter(extra.items()))
                name = opt + ("_up" if v > opts.get(opt, DEFAULT_OPTS[opt]) else "_down")
            per_run[name] = (eY, eT)
    return base, dY, dT
