"""The BFER mechanism the tests and the benchmark use (synth.bfer_mechanism)
against the paper's printed data (tests/golden/bfer_table1.json: Sec. 7.1,
Eqs. 26-29 and Table 1): stoichiometry, reaction orders, temperature
exponent, reversibility, and Table 1's k and Ea converted from cm-mol-s-cal
to SI here (k in (cm^3/mol)^(n-1)/s times 1e-6^(n-1) for a forward order n;
Ea times 4.184 J/cal)."""
import json
import os

import numpy as np
import pytest

from paper_1905_09395_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bfer_table1.json")


def _reactions(m):
    names = list(synth.BFER_SPECIES)
    out = []
    for r in range(len(m.A)):
        k0, k1 = int(m.rxn_ptr[r]), int(m.rxn_ptr[r + 1])
        nu = {names[m.rxn_species[k]]: float(m.rxn_nu[k]) for k in range(k0, k1)}
        order = {names[m.rxn_species[k]]: float(m.rxn_order[k]) for k in range(k0, k1)}
        out.append((nu, order))
    return out


def test_bfer_matches_the_papers_table():
    ref = json.load(open(GOLDEN))["reactions"]
    m = synth.bfer_mechanism()
    rx = _reactions(m)
    for r, name in enumerate(("MEPOX", "COROX")):
        g = ref[name]
        nu, order = rx[r]
        assert nu == g["nu"]
        for sp, o in g["forward_orders"].items():
            assert order[sp] == o
        for sp, o in g.get("reverse_orders", {}).items():
            assert order[sp] == o
        n = sum(g["forward_orders"].values())
        assert m.A[r] == pytest.approx(g["k"] * 1e-6 ** (n - 1.0), rel=1e-12)
        assert m.Ea[r] == pytest.approx(g["Ea_cal_per_mol"] * 4.184, rel=1e-12)
        assert m.beta[r] == g["T_exponent"]
        assert bool(m.reversible[r]) == g["reversible"]


def test_bfer_species_and_mass_balance():
    m = synth.bfer_mechanism()
    assert list(synth.BFER_SPECIES) == ["CH4", "O2", "CO", "H2O", "CO2", "N2"]
    for r in range(len(m.A)):
        k0, k1 = int(m.rxn_ptr[r]), int(m.rxn_ptr[r + 1])
        e = sum(m.rxn_nu[k] * m.elements[m.rxn_species[k]] for k in range(k0, k1))
        np.testing.assert_allclose(e, 0.0, atol=1e-12)
