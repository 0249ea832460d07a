"""stev_solve_host_noalloc: the solve entry point that allocates nothing.

It exists for callers that may not allocate device memory when they solve (a
CFD code whose device memory is owned by its own pool, a real-time or callback
context where cudaMalloc's implicit synchronisation is not acceptable).  It
stages through one fixed 16 MiB device array inside the library.  Checked here
through the C ABI against the allocating host entry point, stev_solve_host, on
the same inputs for two calls in a row (the array keeps the previous call's
contents, so the second call proves the reset), and for its size limit.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1905_09395_b300 import Mechanism, MIXED, binding, lib, synth

TOL_Y, TOL_T = 1e-8, 1e-6   # the FP64 bar of the other parity tests


def _call(fn, m, T, P, Y, dt):
    n, S = Y.shape
    To, Yo = np.empty(n), np.empty((n, S))
    it, st = np.empty(n, np.int32), np.empty(n, np.uint8)
    code = fn(m._h, n, T.ctypes.data, P.ctypes.data, Y.ctypes.data, float(dt), To.ctypes.data,
              Yo.ctypes.data, it.ctypes.data, st.ctypes.data, None)
    return code, (To, Yo, it, st)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, MIXED])
def test_noalloc_matches_allocating_entry_point(precision):
    L = lib()
    mech, T, P, Y, dt = synth.small_case(3000)
    m = Mechanism(mech, precision=precision)
    for half in (slice(0, 1500), slice(1500, 3000)):   # two calls in a row, different data
        Th, Ph, Yh = (np.ascontiguousarray(a[half]) for a in (T, P, Y))
        code, ref = _call(L.stev_solve_host, m, Th, Ph, Yh, dt)
        assert code == 0, L.stev_last_error().decode()
        code, got = _call(L.stev_solve_host_noalloc, m, Th, Ph, Yh, dt)
        assert code == 0, L.stev_last_error().decode()
        assert np.abs(got[1] - ref[1]).max() <= TOL_Y
        assert np.abs(got[0] - ref[0]).max() <= TOL_T
        np.testing.assert_array_equal(got[2], ref[2])
        np.testing.assert_array_equal(got[3], ref[3])
    m.close()


@pytest.mark.gpu
def test_noalloc_rejects_oversized_batches():
    L = lib()
    mech, T, P, Y, dt = synth.small_case(8)
    m = Mechanism(mech)
    n = 2_000_000                      # far beyond the 16 MiB array
    Tb = np.full(n, 1500.0)
    Pb = np.full(n, 101325.0)
    Yb = np.tile(Y[:1], (n, 1))
    code, _ = _call(L.stev_solve_host_noalloc, m, Tb, Pb, Yb, dt)
    assert code == binding.STEV_EINVAL
    msg = L.stev_last_error().decode()
    assert "at most" in msg and "16777216" in msg
    m.close()


@pytest.mark.gpu
def test_noalloc_rejects_a_cell_count_whose_byte_count_would_wrap():
    """A cell count so large that its byte count would overflow size_t is
    rejected on the host before any size is computed or any copy is queued
    (the arrays passed are tiny: nothing may read them)."""
    L = lib()
    mech, T, P, Y, dt = synth.small_case(8)
    m = Mechanism(mech)
    n = (1 << 62) // 8
    To, Yo = np.empty(8), np.empty((8, Y.shape[1]))
    it, st = np.empty(8, np.int32), np.empty(8, np.uint8)
    code = L.stev_solve_host_noalloc(m._h, n, T.ctypes.data, P.ctypes.data, Y.ctypes.data,
                                     float(dt), To.ctypes.data, Yo.ctypes.data, it.ctypes.data,
                                     st.ctypes.data, None)
    assert code == binding.STEV_EINVAL
    assert "at most" in L.stev_last_error().decode()
    m.close()
