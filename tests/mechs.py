"""Hand-built tiny mechanisms for pin tests (inputs only, no STEV arithmetic)."""
import types

import numpy as np

R_U = 8.314462618
P_ATM = 101325.0


def constant_cp_block(cp_over_r, a6=0.0, a7=0.0):
    """NASA-7 block of a species with constant cp/R (a1 only)."""
    return [cp_over_r, 0.0, 0.0, 0.0, 0.0, a6, a7]


def tiny_mechanism(mol_weight, nasa7_blocks, reactions, A, beta=None, Ea=None, reversible=None,
                   t_split=1000.0):
    """reactions: list of dicts {species: nu} (nu < 0 reactant, > 0 product).

    nasa7_blocks: per species either one block (used for both ranges) or a
    pair (low, high)."""
    S, R = len(mol_weight), len(reactions)
    nasa7 = np.zeros((S, 2, 7))
    for i, b in enumerate(nasa7_blocks):
        b = np.asarray(b, dtype=np.float64)
        nasa7[i] = b if b.ndim == 2 else np.stack([b, b])
    ptr, sp, nu = [0], [], []
    for rx in reactions:
        for s in sorted(rx):
            sp.append(s)
            nu.append(float(rx[s]))
        ptr.append(len(sp))
    m = types.SimpleNamespace()
    m.mol_weight = np.asarray(mol_weight, dtype=np.float64)
    m.nasa7 = nasa7
    m.t_range = np.tile([200.0, t_split, 6000.0], (S, 1))
    m.rxn_ptr = np.array(ptr, dtype=np.int32)
    m.rxn_species = np.array(sp, dtype=np.int32)
    m.rxn_nu = np.array(nu, dtype=np.float64)
    m.A = np.asarray(A, dtype=np.float64)
    m.beta = np.zeros(R) if beta is None else np.asarray(beta, dtype=np.float64)
    m.Ea = np.zeros(R) if Ea is None else np.asarray(Ea, dtype=np.float64)
    m.reversible = (np.ones(R, dtype=np.uint8) if reversible is None
                    else np.asarray(reversible, dtype=np.uint8))
    m.n_species, m.n_reactions = S, R
    return m


def isomer_pair(A=1.0e3, K=3.0, W=0.028, cp_over_r=3.5, a6=-1000.0):
    """A <=> B with identical molar mass and enthalpy; K = exp(a7_B - a7_A)."""
    blkA = constant_cp_block(cp_over_r, a6=a6, a7=0.0)
    blkB = constant_cp_block(cp_over_r, a6=a6, a7=float(np.log(K)))
    return tiny_mechanism([W, W], [blkA, blkB], [{0: -1, 1: 1}], A=[A])
