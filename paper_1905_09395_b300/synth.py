"""Seeded synthetic mechanisms and cell states shaped like the paper's workloads.

This module is the only code that both the CUDA path and the CPU oracle
consume.  It creates *inputs* only: element vectors, molar masses, NASA-7
coefficient tables, balanced elementary reactions with Arrhenius parameters,
and initial cell states.  It evaluates no rate, no equilibrium constant, no
time step and no integration step of the STEV method.

The paper's own workloads (the BFER methane mechanism of Sec. 7.1, the C3M
gasification kinetics of Sec. 7.2, MFiX cell states) are not available as
data, so seeded stand-ins with the paper's structure are generated:

* species are small molecules over the elements C, H, O, N; molar masses are
  sums of atomic masses;
* every reaction is elementary and element-balanced, drawn from the
  templates A+B<=>C+D, A+B<=>C, A<=>B+C and A<=>B (at most two molecules a
  side, integer stoichiometry as the paper's Sec. 4 assumes);
* Arrhenius parameters follow k = A T^beta exp(-Ea/RT) (Eq. 29 form) with
  A log-uniform in cm-mol-s units (the paper's Table 1 convention),
  converted to SI by 1e-6^(order-1);
* NASA-7 thermo (Eqs. 15-16) is a least-squares fit of a smooth, saturating
  heat-capacity curve on two ranges split at 1000 K, made continuous in
  cp, h and s at the split, with the enthalpy and entropy constants set from
  drawn formation values at 298.15 K;
* each reaction is written in the direction that is downhill at 1500 K
  according to the drawn formation values (dH - T dS < 0), so the reverse
  constant kf/K never exceeds the forward one there by many decades.

Cell states: T0 uniform, P uniform (in atm, returned in Pa), Y0 drawn from a
symmetric Dirichlet distribution, all from one numpy Generator seed.
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Optional, Tuple

import numpy as np

R_U = 8.314462618          # J/(mol K)
P_ATM = 101325.0           # Pa
ELEMENTS = ("C", "H", "O", "N")
ATOMIC_MASS = np.array([12.011e-3, 1.008e-3, 15.999e-3, 14.007e-3])  # kg/mol
T_SPLIT = 1000.0
T_LOW, T_HIGH = 200.0, 6000.0


@dataclasses.dataclass
class Mechanism:
    """A mechanism in the boundary's table layout (SI units)."""

    elements: np.ndarray      # [S][4] int atom counts (C, H, O, N)
    mol_weight: np.ndarray    # [S] kg/mol
    nasa7: np.ndarray         # [S][2][7] low range, high range
    t_range: np.ndarray       # [S][3] T_low, T_split, T_high
    rxn_ptr: np.ndarray       # [R+1] int32 CSR row pointers
    rxn_species: np.ndarray   # [nnz] int32 species index
    rxn_nu: np.ndarray        # [nnz] float64, <0 reactant, >0 product
    A: np.ndarray             # [R] SI (m^3/mol)^(order-1)/s
    beta: np.ndarray          # [R]
    Ea: np.ndarray            # [R] J/mol
    reversible: np.ndarray    # [R] uint8
    seed: int = 0
    name: str = ""
    # [nnz] float64 or None: each entry's order in the forward (reactants) or
    # reverse (products) rate law; None = |nu| (mass action)
    rxn_order: Optional[np.ndarray] = None

    @property
    def n_species(self) -> int:
        return int(self.mol_weight.shape[0])

    @property
    def n_reactions(self) -> int:
        return int(self.A.shape[0])

    def nu_dense(self) -> np.ndarray:
        """[S][R] stoichiometric matrix (net nu)."""
        out = np.zeros((self.n_species, self.n_reactions))
        for r in range(self.n_reactions):
            for k in range(int(self.rxn_ptr[r]), int(self.rxn_ptr[r + 1])):
                out[int(self.rxn_species[k]), r] += self.rxn_nu[k]
        return out


# ----------------------------------------------------------------------------
# species and reactions
# ----------------------------------------------------------------------------

def _species_pool(n_species: int) -> np.ndarray:
    """Candidate element vectors, small enough that balanced sums are common."""
    if n_species <= 8:
        caps = (0, 2, 2, 0)       # the H/O system: H H2 O O2 OH H2O HO2 H2O2
    elif n_species <= 32:
        caps = (1, 4, 2, 1)
    else:
        caps = (2, 4, 2, 1)
    pool = [v for v in itertools.product(*(range(c + 1) for c in caps)) if any(v)]
    return np.array(pool, dtype=np.int64)


def _balanced_reactions(vecs: np.ndarray):
    """All distinct element-balanced reactions with <= 2 molecules a side.

    Returned as unordered pairs of sorted tuples (side1, side2)."""
    S = vecs.shape[0]
    keyed = {}
    for i in range(S):
        keyed.setdefault(tuple(vecs[i]), []).append((i,))
    for i in range(S):
        for j in range(i, S):
            keyed.setdefault(tuple(vecs[i] + vecs[j]), []).append((i, j))
    out = set()
    for sides in keyed.values():
        for a, b in itertools.combinations(sides, 2):
            if set(a) & set(b):
                continue
            out.add((a, b) if a < b else (b, a))
    return sorted(out)


def _cp_curve(T, c0, cinf, tau):
    return c0 + (cinf - c0) * (1.0 - np.exp(-(T - T_LOW) / tau))


def _fit_nasa7(rng: np.random.Generator, hf: float, s298: float) -> np.ndarray:
    """Two-range NASA-7 coefficients, continuous in cp, h, s at T_SPLIT."""
    c0 = rng.uniform(2.5, 4.5)
    cinf = rng.uniform(c0 + 0.5, 12.0)
    tau = rng.uniform(400.0, 1500.0)
    scale = 1000.0
    # Low range: plain least squares in t = T/1000.
    Tl = np.linspace(T_LOW, T_SPLIT, 161)
    Vl = np.vander(Tl / scale, 5, increasing=True)
    bl, *_ = np.linalg.lstsq(Vl, _cp_curve(Tl, c0, cinf, tau), rcond=None)
    low = bl / scale ** np.arange(5)
    cp_split = float(np.polyval(low[::-1], T_SPLIT))
    # High range: b0 fixed by continuity of cp at the split.
    Th = np.linspace(T_SPLIT, T_HIGH, 401)
    th = Th / scale
    ts = T_SPLIT / scale
    basis = np.stack([th ** k - ts ** k for k in range(1, 5)], axis=1)
    target = _cp_curve(Th, c0, cinf, tau) - cp_split
    bh, *_ = np.linalg.lstsq(basis, target, rcond=None)
    bh_full = np.concatenate([[cp_split - sum(bh[k - 1] * ts ** k for k in range(1, 5))], bh])
    high = bh_full / scale ** np.arange(5)

    def h_over_r_poly(a, T):     # integral of cp/R dT without the constant
        return sum(a[k] * T ** (k + 1) / (k + 1) for k in range(5))

    def s_over_r_poly(a, T):     # integral of cp/(R T) dT without the constant
        return a[0] * np.log(T) + sum(a[k] * T ** k / k for k in range(1, 5))

    T0 = 298.15
    a6_low = hf / R_U - h_over_r_poly(low, T0)
    a7_low = s298 / R_U - s_over_r_poly(low, T0)
    a6_high = h_over_r_poly(low, T_SPLIT) + a6_low - h_over_r_poly(high, T_SPLIT)
    a7_high = s_over_r_poly(low, T_SPLIT) + a7_low - s_over_r_poly(high, T_SPLIT)
    out = np.zeros((2, 7))
    out[0, :5], out[0, 5], out[0, 6] = low, a6_low, a7_low
    out[1, :5], out[1, 5], out[1, 6] = high, a6_high, a7_high
    return out


def make_mechanism(n_species: int, n_reactions: int, seed: int = 0,
                   ea_max: float = 200e3, a_lo: float = 1e6, a_hi: float = 1e14,
                   beta_range: Tuple[float, float] = (-1.0, 1.0),
                   min_stiffness: Optional[float] = None,
                   name: str = "") -> Mechanism:
    """Seeded synthetic mechanism with S species and R reversible reactions.

    min_stiffness: if given, resample the kinetics until the ratio of the
    largest to the smallest pseudo-first-order forward constant
    k_r * Cbar^(order-1) at 1500 K and 1 atm (Cbar = P/RT) reaches it."""
    rng = np.random.default_rng(seed)
    pool = _species_pool(n_species)
    for _ in range(10000):
        if n_species <= len(pool):
            idx = rng.choice(len(pool), size=n_species, replace=False)
        else:
            idx = rng.choice(len(pool), size=n_species, replace=True)
        vecs = pool[idx]
        cands = _balanced_reactions(vecs)
        if len(cands) >= n_reactions:
            break
    else:  # pragma: no cover
        raise RuntimeError("could not find enough balanced reactions")
    S = n_species
    W = vecs @ ATOMIC_MASS
    hf = rng.uniform(-400e3, 200e3, size=S)
    s298 = rng.uniform(150.0, 300.0, size=S)
    nasa7 = np.stack([_fit_nasa7(rng, hf[i], s298[i]) for i in range(S)])
    t_range = np.tile(np.array([T_LOW, T_SPLIT, T_HIGH]), (S, 1))

    pick = rng.choice(len(cands), size=n_reactions, replace=False)
    rxns = []
    for p in pick:
        a, b = cands[p]
        dH = sum(hf[i] for i in b) - sum(hf[i] for i in a)
        dS = sum(s298[i] for i in b) - sum(s298[i] for i in a)
        if dH - 1500.0 * dS > 0:   # write the downhill direction as forward
            a, b = b, a
        rxns.append((a, b))

    ptr, sp, nu = [0], [], []
    order = np.zeros(n_reactions)
    for r, (a, b) in enumerate(rxns):
        for side, sign in ((a, -1.0), (b, 1.0)):
            for s in sorted(set(side)):
                sp.append(s)
                nu.append(sign * side.count(s))
        ptr.append(len(sp))
        order[r] = len(a)

    Cbar = P_ATM / (R_U * 1500.0)
    for _ in range(10000):
        A_cgs = np.exp(rng.uniform(np.log(a_lo), np.log(a_hi), size=n_reactions))
        beta = rng.uniform(beta_range[0], beta_range[1], size=n_reactions)
        Ea = rng.uniform(0.0, ea_max, size=n_reactions)
        A = A_cgs * (1e-6) ** (order - 1.0)
        if min_stiffness is None:
            break
        kp = A * 1500.0 ** beta * np.exp(-Ea / (R_U * 1500.0)) * Cbar ** (order - 1.0)
        if kp.max() / kp.min() >= min_stiffness:
            break
    return Mechanism(
        elements=vecs.astype(np.int64), mol_weight=W.astype(np.float64),
        nasa7=nasa7.astype(np.float64), t_range=t_range.astype(np.float64),
        rxn_ptr=np.array(ptr, dtype=np.int32), rxn_species=np.array(sp, dtype=np.int32),
        rxn_nu=np.array(nu, dtype=np.float64), A=A.astype(np.float64),
        beta=beta.astype(np.float64), Ea=Ea.astype(np.float64),
        reversible=np.ones(n_reactions, dtype=np.uint8), seed=seed, name=name)


def make_cells(mech: Mechanism, n_cells: int, seed: int = 0,
               T_range: Tuple[float, float] = (1200.0, 1800.0),
               P_atm_range: Tuple[float, float] = (1.0, 1.0),
               dirichlet: float = 1.0):
    """Seeded cell states: T [cells], P [cells] (Pa), Y [cells][S] (AoS)."""
    rng = np.random.default_rng(seed + 7919)
    T = rng.uniform(T_range[0], T_range[1], size=n_cells)
    P = rng.uniform(P_atm_range[0], P_atm_range[1], size=n_cells) * P_ATM
    Y = rng.dirichlet(np.full(mech.n_species, dirichlet), size=n_cells)
    return T.astype(np.float64), P.astype(np.float64), np.ascontiguousarray(Y, dtype=np.float64)


# ----------------------------------------------------------------------------
# the workloads: small case, 1M-cell case, mixed+MLP, uneven batches, serving
# ----------------------------------------------------------------------------

def small_mechanism():
    """8 species / 20 reactions, A log-uniform 1e6-1e14, Ea 0-200 kJ/mol."""
    return make_mechanism(8, 20, seed=0, ea_max=200e3, name="syn8x20")


def small_case(n_cells: int = 4096):
    """8 species / 20 reactions, 4,096 cells, T0 U[1200,1800] K, 1 atm,
    Y0 Dirichlet(1), dt = 1e-3 s."""
    mech = small_mechanism()
    T, P, Y = make_cells(mech, n_cells, seed=0, T_range=(1200.0, 1800.0),
                         P_atm_range=(1.0, 1.0), dirichlet=1.0)
    return mech, T, P, Y, 1e-3


def scale_mechanism():
    """32 species / 150 reactions, Ea 0-250 kJ/mol, stiffness ratio >= 1e6."""
    return make_mechanism(32, 150, seed=1, ea_max=250e3, min_stiffness=1e6,
                          name="syn32x150")


def scale_case(n_cells: int = 1 << 20, seed: int = 1):
    """1,048,576 cells, T0 U[800,2200] K, P U[1,5] atm, Y0 Dirichlet(0.5),
    dt = 1e-3 s, on the 32/150 mechanism."""
    mech = scale_mechanism()
    T, P, Y = make_cells(mech, n_cells, seed=seed, T_range=(800.0, 2200.0),
                         P_atm_range=(1.0, 5.0), dirichlet=0.5)
    return mech, T, P, Y, 1e-3


def large_mechanism():
    """53 species / 325 reactions, Ea 0-250 kJ/mol, A log-uniform 1e6-1e11
    (cm-mol-s), stiffness ratio >= 1e6.  With A up to 1e14 nearly every cell
    of this mechanism needs more than 2e5 STEV iterations at dt = 5e-4 s (the
    paper reports STEV degrading on detailed mechanisms with many stiff
    reversible reactions); 1e11 keeps cells that the method finishes."""
    return make_mechanism(53, 325, seed=3, ea_max=250e3, a_hi=1e11, min_stiffness=1e6,
                          name="syn53x325")


def uneven_case(scale: float = 1.0, seed: int = 3):
    """64 independent batches, sizes log-uniform 1k-256k (times `scale`),
    T0 U[700,2500] K, P U[1,5] atm, Y0 Dirichlet(0.5), dt = 5e-4 s, on the
    53/325 mechanism.  Returns (mech, [(T, P, Y) per batch], dt)."""
    mech = large_mechanism()
    sizes = np.maximum(1, (uneven_batch_sizes(seed=seed) * scale).astype(np.int64))
    batches = []
    for b, n in enumerate(sizes):
        batches.append(make_cells(mech, int(n), seed=seed * 1000 + b, T_range=(700.0, 2500.0),
                                  P_atm_range=(1.0, 5.0), dirichlet=0.5))
    return mech, batches, 5e-4


def uneven_batch_sizes(n_batches: int = 64, lo: int = 1000, hi: int = 256000, seed: int = 3):
    rng = np.random.default_rng(seed + 104729)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_batches)).astype(np.int64)


def serving_requests(duration: float = 10.0, rate: float = 200.0, lo: int = 1000,
                     hi: int = 512 * 1024, n_mechanisms: int = 2, seed: int = 4):
    """Seeded request stream of the serving workload: Poisson arrivals at
    `rate` per second over `duration` seconds, sizes log-uniform [lo, hi]
    cells, each request on a mechanism drawn uniformly from n_mechanisms.
    Returns a list of (arrival time s, mechanism index, n_cells, pool offset),
    the offset placing the request's cells inside a pool of `hi` cells."""
    rng = np.random.default_rng(seed + 15485863)
    out, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        mi = int(rng.integers(n_mechanisms))
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        off = int(rng.integers(0, hi - n + 1))
        out.append((t, mi, n, off))


# ----------------------------------------------------------------------------
# the paper's BFER methane mechanism (Sec. 7.1, Eqs. 26-30, Table 1)
# ----------------------------------------------------------------------------

# species of the two-step mechanism and their standard formation enthalpies
# and entropies at 298.15 K (textbook values; J/mol, J/mol/K)
BFER_SPECIES = ("CH4", "O2", "CO", "H2O", "CO2", "N2")
_BFER_ELEMENTS = np.array([[1, 4, 0, 0], [0, 0, 2, 0], [1, 0, 1, 0], [0, 2, 1, 0],
                           [1, 0, 2, 0], [0, 0, 0, 2]], dtype=np.int64)
_BFER_HF = np.array([-74.6e3, 0.0, -110.5e3, -241.8e3, -393.5e3, 0.0])
_BFER_S298 = np.array([186.3, 205.2, 197.7, 188.8, 213.8, 191.6])
CAL = 4.184  # J/cal


def bfer_mechanism(seed: int = 5) -> Mechanism:
    """The BFER two-step methane mechanism of Sec. 7.1: MEPOX
    CH4 + 1.5 O2 -> CO + 2 H2O (irreversible, Eq. 28: orders 0.5 in CH4 and
    0.65 in O2) and COROX CO + 0.5 O2 <=> CO2 (Eq. 29: T^0.7, orders 1 and 0.5
    forward, 1 in CO2 backward, K from Eq. 30), with Table 1's constants
    (cm-mol-s-cal) converted to SI; N2 is inert.  The paper gives no NASA-7
    data, so each species' heat capacity is a seeded smooth curve (as for the
    other synthetic mechanisms) with textbook formation enthalpy and entropy."""
    rng = np.random.default_rng(seed)
    S = len(BFER_SPECIES)
    W = _BFER_ELEMENTS @ ATOMIC_MASS
    nasa7 = np.stack([_fit_nasa7(rng, _BFER_HF[i], _BFER_S298[i]) for i in range(S)])
    t_range = np.tile(np.array([T_LOW, T_SPLIT, T_HIGH]), (S, 1))
    CH4, O2, CO, H2O, CO2 = 0, 1, 2, 3, 4
    # CSR entries: species, nu, order (products of the irreversible MEPOX: order unused)
    mepox = [(CH4, -1.0, 0.5), (O2, -1.5, 0.65), (CO, 1.0, 1.0), (H2O, 2.0, 2.0)]
    corox = [(O2, -0.5, 0.5), (CO, -1.0, 1.0), (CO2, 1.0, 1.0)]
    ptr, sp, nu, order = [0], [], [], []
    for rx in (mepox, corox):
        for s_, n_, o_ in sorted(rx):
            sp.append(s_)
            nu.append(n_)
            order.append(o_)
        ptr.append(len(sp))
    fwd_order = np.array([0.5 + 0.65, 1.0 + 0.5])
    A = np.array([4.9e9, 2.0e8]) * (1e-6) ** (fwd_order - 1.0)
    return Mechanism(
        elements=_BFER_ELEMENTS.copy(), mol_weight=W.astype(np.float64),
        nasa7=nasa7.astype(np.float64), t_range=t_range.astype(np.float64),
        rxn_ptr=np.array(ptr, dtype=np.int32), rxn_species=np.array(sp, dtype=np.int32),
        rxn_nu=np.array(nu, dtype=np.float64), A=A, beta=np.array([0.0, 0.7]),
        Ea=np.array([35500.0, 12000.0]) * CAL, reversible=np.array([0, 1], dtype=np.uint8),
        seed=seed, name="bfer", rxn_order=np.array(order, dtype=np.float64))


def bfer_cells(mech: Mechanism, n_cells: int, seed: int = 6,
               T_range: Tuple[float, float] = (1200.0, 2200.0)):
    """Random fixed thermochemical states as in the paper's BFER benchmark
    (Sec. 7.1): T0 uniform, 1 atm, a methane-air-like mixture with products
    (CH4 0-0.1, O2 0.05-0.23, CO and CO2 0-0.05, H2O 0-0.1, the rest N2)."""
    rng = np.random.default_rng(seed + 7919)
    T = rng.uniform(T_range[0], T_range[1], size=n_cells)
    P = np.full(n_cells, P_ATM)
    Y = np.zeros((n_cells, mech.n_species))
    Y[:, 0] = rng.uniform(0.0, 0.1, n_cells)
    Y[:, 1] = rng.uniform(0.05, 0.23, n_cells)
    Y[:, 2] = rng.uniform(0.0, 0.05, n_cells)
    Y[:, 3] = rng.uniform(0.0, 0.1, n_cells)
    Y[:, 4] = rng.uniform(0.0, 0.05, n_cells)
    Y[:, 5] = 1.0 - Y[:, :5].sum(axis=1)
    return T, P, Y


# ----------------------------------------------------------------------------
# multiphase cells (Sec. 7.2): random gasifier-like thermochemical states
# ----------------------------------------------------------------------------
MP_GAS = ("O2", "CO", "CO2", "CH4", "H2", "H2O", "H2S", "C3H6", "HCN", "C2H4", "C2H6", "Tar",
          "SO3", "N2")
MP_SOLID = ("CV", "CC", "CM", "CA")


def multiphase_cells(n_cells: int, seed: int = 0, T_range: Tuple[float, float] = (900.0, 1500.0),
                     o2_max: float = 0.1) -> np.ndarray:
    """Seeded multiphase cell records [n][24]: gas mass fractions X_g[14]
    (nitrogen-rich, O2 up to o2_max), solid mass fractions X_s[4] (volatile
    matter, fixed carbon, moisture, ash), T_g uniform in T_range, T_s within
    100 K of it, eps_s U[0.02, 0.4], particle density rho_s U[1000, 1500]
    kg/m^3, d_p U[1e-4, 5e-4] m, P U[1, 5] atm (Pa)."""
    rng = np.random.default_rng(seed + 104729)
    gas_a = np.array([1, 1, 1, 0.5, 0.5, 1, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1, 4.0])
    Xg = rng.dirichlet(gas_a, size=n_cells)
    o2 = rng.uniform(0.0, o2_max, size=n_cells)
    Xg[:, 0] = 0.0
    Xg /= Xg.sum(axis=1, keepdims=True)
    Xg *= (1.0 - o2)[:, None]
    Xg[:, 0] = o2
    Xs = rng.dirichlet(np.array([1.0, 2.0, 0.5, 1.0]), size=n_cells)
    Tg = rng.uniform(T_range[0], T_range[1], size=n_cells)
    Ts = Tg + rng.uniform(-100.0, 100.0, size=n_cells)
    eps = rng.uniform(0.02, 0.4, size=n_cells)
    rho_s = rng.uniform(1000.0, 1500.0, size=n_cells)
    dp = rng.uniform(1e-4, 5e-4, size=n_cells)
    P = rng.uniform(1.0, 5.0, size=n_cells) * P_ATM
    return np.ascontiguousarray(np.column_stack([Xg, Xs, Tg, Ts, eps, rho_s, dp, P]),
                                dtype=np.float64)
