"""Serving loop (stev_server_*): continuous batching of requests from two
mechanisms (8 species / 20 reactions and 32 / 150) into resident persistent
kernels.

Each cell's result depends only on the cell, its request's t_f and the
mechanism (Sec. 2.4: cells are integrated independently; a slot freed by a
finished cell takes the next cell), so a request's results in the mix must be
bit-for-bit those of the same request solved alone.  Also: admission by the
memory budget, requests that overlap on the device, relaunch after an idle
exit, empty requests, shutdown with work outstanding, and a prefix of the
solve against the oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_1905_09395_b300 import (FP64, MIXED, THERMO_MLP, THERMO_POLY, Mechanism, Server,
                                   StevError, synth)

pytestmark = pytest.mark.gpu

MODES = {"fp64": dict(precision=FP64), "mixed": dict(precision=MIXED),
         "mixed_mlp": dict(precision=MIXED, thermo=THERMO_MLP),
         # kernels compiled for each mechanism at run time (NVRTC)
         "mixed_mlp_spec": dict(precision=MIXED, thermo=THERMO_MLP, specialize=1)}


def _mechanisms(mode, **extra):
    opts = dict(MODES[mode], **extra)
    thermo = opts.pop("thermo", THERMO_POLY)
    ms = [Mechanism(synth.small_mechanism(), **opts), Mechanism(synth.scale_mechanism(), **opts)]
    if thermo != THERMO_POLY:
        Ts = np.linspace(300.0, 3000.0, 200_000)
        for m in ms:
            m.mlp_train(Ts, epochs=4, batch=4096, lr=2e-3, seed=1)
            m.set_options(thermo=thermo)
    if opts.get("specialize"):
        assert all(m.is_specialized for m in ms)
    return ms


def _requests(seed, n_req, lo=20, hi=1500):
    """Seeded requests alternating between the two mechanisms: (mech, T, P, Y, dt)."""
    rng = np.random.default_rng(seed)
    small, scale = synth.small_mechanism(), synth.scale_mechanism()
    reqs = []
    for k in range(n_req):
        mi = k % 2
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        mech = small if mi == 0 else scale
        T, P, Y = synth.make_cells(mech, n, seed=100 + k, T_range=(800, 2200),
                                   P_atm_range=(1, 5), dirichlet=0.5)
        dt = [1e-3, 5e-4][(k // 2) % 2]
        reqs.append((mi, T, P, Y, dt))
    return reqs


def _drain(srv, n, timeout=120.0):
    got, t_end = {}, time.time() + timeout
    while len(got) < n and time.time() < t_end:
        for d in srv.poll(timeout=0.5):
            got[d["id"]] = d
    assert len(got) == n, "only %d of %d requests finished" % (len(got), n)
    return got


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_mlp", "mixed_mlp_spec"])
def test_same_alone_and_in_the_mix(mode):
    ms = _mechanisms(mode)
    reqs = _requests(seed=5, n_req=12)
    alone = [ms[mi].solve_host(T, P, Y, dt) for mi, T, P, Y, dt in reqs]
    srv = Server(ms, sm_share=[40, 100], mem_budget=256 << 20)
    ids = []
    # half now, the rest once the first results are back: later requests are
    # admitted while earlier ones are still on the device
    for mi, T, P, Y, dt in reqs[:6]:
        ids.append(srv.submit(mi, T, P, Y, dt))
    first = srv.poll(timeout=60.0)
    assert first, "no request finished"
    for mi, T, P, Y, dt in reqs[6:]:
        ids.append(srv.submit(mi, T, P, Y, dt))
    got = {d["id"]: d for d in first}
    got.update(_drain(srv, len(reqs) - len(first)))
    for rid, ref in zip(ids, alone):
        d = got[rid]
        assert d["status"] == 0
        for a, b in zip(d["out"], ref):
            np.testing.assert_array_equal(a, b)
    st = srv.stats
    assert st["completed"] == len(reqs) and st["cells_completed"] == sum(len(r[1]) for r in reqs)
    assert st["resident_bytes"] == 0
    srv.close()
    for m in ms:
        m.close()


def _bytes(n, S):
    a = lambda b: (b + 255) // 256 * 256
    return 2 * a(8 * n) + a(8 * n * S) + a(4 * n) + a(n)


def test_admission_by_memory_budget():
    ms = _mechanisms("mixed")
    reqs = _requests(seed=6, n_req=10, lo=2000, hi=4000)
    need = [_bytes(len(T), ms[mi].S) for mi, T, _, _, _ in reqs]
    budget = 2 * max(need)                       # two requests at a time at most
    srv = Server(ms, sm_share=[40, 100], mem_budget=budget)
    with pytest.raises(StevError):               # larger than the whole budget
        n_big = budget // (8 * 34) + 1
        T, P, Y = synth.make_cells(synth.scale_mechanism(), n_big, seed=1)
        srv.submit(1, T, P, Y, 1e-3)
    ids = [srv.submit(mi, T, P, Y, dt) for mi, T, P, Y, dt in reqs]
    got = _drain(srv, len(ids))
    st = srv.stats
    assert st["peak_resident_bytes"] <= budget
    assert st["completed"] == len(ids) and st["resident_bytes"] == 0
    # first come, first served: admission order is submission order
    adm = [got[i]["t_admit"] for i in ids]
    assert adm == sorted(adm)
    # the budget held requests back: someone was admitted only after another finished
    done = sorted(got[i]["t_done"] for i in ids)
    assert any(a >= done[0] for a in adm[2:])
    for d in got.values():
        assert d["t_submit"] <= d["t_admit"] <= d["t_done"]
    srv.close()
    for m in ms:
        m.close()


def test_requests_overlap_on_the_device():
    ms = _mechanisms("mixed")
    reqs = _requests(seed=7, n_req=8, lo=3000, hi=6000)
    srv = Server(ms, sm_share=[30, 110], mem_budget=1 << 30)
    ids = [srv.submit(mi, T, P, Y, dt) for mi, T, P, Y, dt in reqs]
    got = _drain(srv, len(ids))
    iv = {mi: [(got[i]["t_admit"], got[i]["t_done"]) for i, r in zip(ids, reqs) if r[0] == mi]
          for mi in (0, 1)}
    # both mechanisms' kernels ran at the same time
    assert any(a0 < b1 and a1 < b0 for a0, b0 in iv[0] for a1, b1 in iv[1])
    srv.close()
    for m in ms:
        m.close()


def test_relaunch_after_idle_and_empty_requests():
    ms = _mechanisms("fp64")
    srv = Server(ms, sm_share=[20, 20], mem_budget=64 << 20)
    mech = synth.small_mechanism()
    T, P, Y = synth.make_cells(mech, 300, seed=3)
    ref = ms[0].solve_host(T, P, Y, 1e-3)
    e = np.zeros(0)
    rid0 = srv.submit(0, e, e, np.zeros((0, mech.n_species)), 1e-3)
    d0 = _drain(srv, 1)[rid0]
    assert d0["status"] == 0 and d0["n_cells"] == 0
    for k in range(3):
        rid = srv.submit(0, T, P, Y, 1e-3)
        d = _drain(srv, 1)[rid]
        for a, b in zip(d["out"], ref):
            np.testing.assert_array_equal(a, b)
        time.sleep(0.1)                          # past the kernel's idle exit
    assert srv.stats["kernel_launches"] >= 3
    srv.close()
    for m in ms:
        m.close()


def test_stop_with_work_outstanding():
    ms = _mechanisms("fp64")
    srv = Server(ms, sm_share=[8, 8], mem_budget=1 << 30)
    mech = synth.small_mechanism()
    Ts, Ps, Ys = synth.make_cells(mech, 500, seed=2)
    T, P, Y = synth.make_cells(synth.scale_mechanism(), 200_000, seed=9)
    small = srv.submit(0, Ts, Ps, Ys, 1e-3)
    big = srv.submit(1, T, P, Y, 1e-3)           # minutes of work on 8 SMs
    time.sleep(2.0)
    t0 = time.time()
    srv.stop(timeout=60.0)                       # cells in flight finish, nothing new starts
    assert time.time() - t0 < 30.0
    got = {}
    while True:
        more = srv.poll()
        if not more:
            break
        got.update({d["id"]: d for d in more})
    assert got[small]["status"] == 0 and got[small]["cells_done"] == 500
    b = got[big]
    assert b["status"] != 0 and 0 < b["cells_done"] < b["n_cells"]
    st = srv.stats
    assert st["completed"] == 1 and st["cancelled"] == 1
    assert st["cells_completed"] == 500 + b["cells_done"]
    with pytest.raises(StevError):
        srv.submit(0, Ts, Ps, Ys, 1e-3)
    srv.close()
    for m in ms:
        m.close()


def test_serving_prefix_against_oracle():
    # the first 25 steps of every cell through the server against the oracle
    ms = _mechanisms("fp64", max_iters=25)
    reqs = _requests(seed=8, n_req=4, lo=30, hi=80)
    srv = Server(ms, sm_share=[10, 10], mem_budget=64 << 20)
    ids = [srv.submit(mi, T, P, Y, dt) for mi, T, P, Y, dt in reqs]
    got = _drain(srv, len(ids))
    mechs = [synth.small_mechanism(), synth.scale_mechanism()]
    for rid, (mi, T, P, Y, dt) in zip(ids, reqs):
        To, Yo, it, _ = got[rid]["out"]
        ref = oracle.solve(mechs[mi], T, P, Y, dt, max_iters=25)
        assert (it == ref[2]).all()
        assert np.abs(Yo - ref[1]).max() <= 1e-8
        assert np.abs(To - ref[0]).max() <= 1e-6
    srv.close()
    for m in ms:
        m.close()


def test_global_rate_laws_in_the_mix():
    # the BFER mechanism (real orders, real stoichiometry) served beside the
    # 8/20 mechanism: each request's results equal its solve alone
    tabs = [synth.bfer_mechanism(), synth.small_mechanism()]
    ms = [Mechanism(t) for t in tabs]
    reqs = []
    for k in range(6):
        mi = k % 2
        n = [700, 1500, 300][k // 2]
        if mi == 0:
            T, P, Y = synth.bfer_cells(tabs[0], n, seed=20 + k)
        else:
            T, P, Y = synth.make_cells(tabs[1], n, seed=20 + k)
        reqs.append((mi, T, P, Y, 1e-3))
    alone = [ms[mi].solve_host(T, P, Y, dt) for mi, T, P, Y, dt in reqs]
    srv = Server(ms, sm_share=[60, 60], mem_budget=64 << 20)
    ids = [srv.submit(mi, T, P, Y, dt) for mi, T, P, Y, dt in reqs]
    got = _drain(srv, len(ids))
    for rid, ref in zip(ids, alone):
        assert got[rid]["status"] == 0
        for a, b in zip(got[rid]["out"], ref):
            np.testing.assert_array_equal(a, b)
    srv.close()
    for m in ms:
        m.close()
