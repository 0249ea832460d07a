"""The C ABI without a GPU: the library loads, exports every symbol that
include/stev.h declares, and rejects bad mechanisms before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1905_09395_b300 as stev
from paper_1905_09395_b300 import binding, synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "stev.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stev_[a-z0-9_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = stev.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_default_options():
    o = stev.default_options()
    assert o.y_step_max == 1e-3 and o.delta_max == 0.01 and o.alpha == 1e-5
    assert o.dft_n == 13 and o.dft_hi_first == 4
    assert o.tol_ring == 0.5 and o.tol_freq == 1e-6 and o.r_fac == 2.0
    assert o.precision == stev.FP64 and o.dft_on == 1


def _create(mech, **kw):
    """Calls stev_mechanism_create and returns its status code."""
    L = stev.lib()
    tables = dict(
        W=np.ascontiguousarray(mech.mol_weight, np.float64),
        nasa7=np.ascontiguousarray(mech.nasa7, np.float64),
        tr=np.ascontiguousarray(mech.t_range, np.float64),
        ptr=np.ascontiguousarray(mech.rxn_ptr, np.int32),
        sp=np.ascontiguousarray(mech.rxn_species, np.int32),
        nu=np.ascontiguousarray(mech.rxn_nu, np.float64),
        A=np.ascontiguousarray(mech.A, np.float64), beta=np.ascontiguousarray(mech.beta, np.float64),
        Ea=np.ascontiguousarray(mech.Ea, np.float64),
        rev=np.ascontiguousarray(mech.reversible, np.uint8))
    tables.update(kw)
    S = kw.get("S", len(tables["W"]))
    R = kw.get("R", len(tables["A"]))
    h = ctypes.c_void_p()
    p = lambda a: a.ctypes.data
    code = L.stev_mechanism_create(S, R, p(tables["W"]), p(tables["nasa7"]), p(tables["tr"]),
                                   p(tables["ptr"]), p(tables["sp"]), p(tables["nu"]),
                                   p(tables["A"]), p(tables["beta"]), p(tables["Ea"]),
                                   p(tables["rev"]), None, ctypes.byref(h))
    if code == 0:
        L.stev_destroy(h)
    return code, L.stev_last_error().decode()


@pytest.fixture(scope="module")
def mech():
    return synth.small_mechanism()


def test_rejects_bad_sizes(mech):
    assert _create(mech, S=0)[0] == binding.STEV_EINVAL
    assert _create(mech, S=65)[0] == binding.STEV_EINVAL
    assert _create(mech, R=0)[0] == binding.STEV_EINVAL


def test_rejects_nonfinite_and_negative_rates(mech):
    A = mech.A.copy()
    A[3] = np.nan
    assert _create(mech, A=A)[0] == binding.STEV_EINVAL
    A[3] = -1.0
    code, msg = _create(mech, A=A)
    assert code == binding.STEV_EINVAL and "A[3]" in msg


def test_rejects_unbalanced_reaction(mech):
    W = mech.mol_weight.copy()
    W[0] *= 1.5
    assert _create(mech, W=W)[0] == binding.STEV_EUNBALANCED


def test_rejects_non_elementary(mech):
    nu = mech.rxn_nu.copy()
    nu[0] = -0.5
    assert _create(mech, nu=nu)[0] == binding.STEV_EINVAL
    sp = mech.rxn_species.copy()
    sp[0] = 99
    assert _create(mech, sp=sp)[0] == binding.STEV_EINVAL


def test_global_rate_laws_need_create_orders():
    # the BFER mechanism (real nu, real orders) passes validation through
    # stev_mechanism_create_orders; an order <= 0 does not
    m = synth.bfer_mechanism()
    code, msg = _create(m)
    assert code == binding.STEV_EINVAL and "create_orders" in msg
    L = binding.lib()
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    arrs = dict(W=f64(m.mol_weight), n7=f64(m.nasa7), tr=f64(m.t_range),
                ptr=np.ascontiguousarray(m.rxn_ptr, dtype=np.int32),
                sp=np.ascontiguousarray(m.rxn_species, dtype=np.int32), nu=f64(m.rxn_nu),
                A=f64(m.A), beta=f64(m.beta), Ea=f64(m.Ea),
                rev=np.ascontiguousarray(m.reversible, dtype=np.uint8))

    def create(order):
        h = ctypes.c_void_p()
        o = f64(order)
        p = lambda a: a.ctypes.data
        code = L.stev_mechanism_create_orders(
            m.n_species, m.n_reactions, p(arrs["W"]), p(arrs["n7"]), p(arrs["tr"]),
            p(arrs["ptr"]), p(arrs["sp"]), p(arrs["nu"]), p(o), p(arrs["A"]), p(arrs["beta"]),
            p(arrs["Ea"]), p(arrs["rev"]), None, ctypes.byref(h))
        if code == binding.STEV_OK:
            L.stev_destroy(h)
        return code, L.stev_last_error().decode()

    code, msg = create(m.rxn_order)
    assert code in (binding.STEV_OK, binding.STEV_ECUDA), msg
    bad = m.rxn_order.copy()
    bad[1] = 0.0
    code, msg = create(bad)
    assert code == binding.STEV_EINVAL and "rxn_order[1]" in msg


def test_mechanism_validation_passes_the_synthetic_workloads():
    # a valid mechanism either succeeds (GPU) or fails only at the CUDA step
    for m in (synth.small_mechanism(), synth.scale_mechanism(), synth.large_mechanism()):
        code, msg = _create(m)
        assert code in (binding.STEV_OK, binding.STEV_ECUDA), msg
