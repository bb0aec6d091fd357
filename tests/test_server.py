"""Serving engine (sat_server_*): continuous batching on one GPU.

A request's result must be the same whether it runs alone or in a mix of
other requests of other sizes admitted while it runs, and the same as
sat_run on that one chain with resync_every = stages_per_tick: with the
windowed 4-warp group layout when its image size's classes share launches
(the default), with sat_run's size rules when every class runs its own
(SAT_SERVER_PER_CLASS)."""
import time

import numpy as np
import pytest

import oracle
from paper_1411_4622_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_4622_gb300 import api as a
    from paper_1411_4622_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)
    return a


TICK = 3


@pytest.fixture(params=["shared", "per_class"])
def mode(request, api):
    """Server flags of the two launch layouts, and the sat_run plan each matches."""
    if request.param == "shared":
        return dict(flags=0, plan=api.SAT_PLAN_WINDOW_G4)
    return dict(flags=api.SAT_SERVER_PER_CLASS, plan=api.SAT_PLAN_RULES)


def _requests():
    """Mixed sizes, precisions, K and schedule lengths (one with no stages);
    sizes 48 and 64 each with two angle counts, so one launch carries
    several tables."""
    shapes = [(32, 24, 0, None, 1, 7), (48, 40, 1, "disk", 4, 5), (64, 60, 0, "disk", 8, 4), (48, 40, 1, "disk", 4, 9),
              (32, 24, 0, None, 1, 0), (40, 30, 1, "disk", 4, 6), (64, 60, 0, "disk", 8, 2), (32, 24, 0, None, 1, 3),
              (48, 30, 1, "disk", 8, 5), (64, 44, 0, "disk", 1, 4)]
    reqs = []
    for i, (n, U, prec, m, K, S) in enumerate(shapes):
        B = synth.bins_for(n)
        mask = synth.disk_mask(n) if m else None
        ph = synth.phantom(n, 6, 300 + i) * (mask if mask is not None else 1.0)
        sino = oracle.drt(ph, U, B).astype(np.float32)
        reqs.append(dict(sino=sino, n=n, precision=prec, mask=mask, bome_k=K, n_sweeps=S, seed=900 + i,
                         t0=-1.0, tn=-1.0))
    return reqs


def _run_alone(api, reqs, flags=0):
    out = []
    with api.Server(stages_per_tick=TICK, flags=flags) as srv:
        for r in reqs:
            t = srv.submit(**r)
            out.append(srv.wait(t, 60000))
    return out


def test_server_same_alone_and_in_mix(api, mode):
    reqs = _requests()
    alone = _run_alone(api, reqs, mode["flags"])
    with api.Server(stages_per_tick=TICK, flags=mode["flags"]) as srv:
        # a first wave, then a second submitted while the first runs
        tickets = [srv.submit(**r) for r in reqs[:4]]
        first = srv.wait(tickets[0], 60000)
        tickets += [srv.submit(**r) for r in reqs[4:]]
        mixed = [first] + [srv.wait(t, 60000) for t in tickets[1:]]
        info = srv.info()
    assert info["completed"] == len(reqs) and info["failed"] == 0
    for (ia, sa), (im, sm), r in zip(alone, mixed, reqs):
        assert sa["status"] == 0 and sm["status"] == 0
        assert np.array_equal(ia, im)
        assert sa["accepted"] == sm["accepted"] and sa["final_cost"] == sm["final_cost"]
        assert sm["proposed"] == r["n_sweeps"] * (int(r["mask"].sum()) if r["mask"] is not None else r["n"] ** 2)


def test_server_matches_sat_run(api, mode):
    """Each request is sat_run on one chain with resync_every = stages_per_tick."""
    reqs = _requests()
    with api.Server(stages_per_tick=TICK, flags=mode["flags"]) as srv:
        tickets = [srv.submit(**r) for r in reqs]
        got = [srv.wait(t, 60000) for t in tickets]
    for (img, st), r in zip(got, reqs):
        n = r["n"]
        U, B = r["sino"].shape
        p = api.pila_build(n, U, B, r["precision"], mask=r["mask"])
        init = synth.initial_image(n, 0.5, r["mask"]).astype(np.float32)[None]
        ref = torch.tensor(init, device="cuda")
        kw = {k: v for k, v in r.items() if k not in ("sino", "n", "precision", "mask")}
        s1 = api.sat_run(p, torch.tensor(r["sino"][None], device="cuda"), ref, resync_every=TICK, plan=mode["plan"],
                         **kw)
        api.pila_free(p)
        assert np.array_equal(ref.cpu().numpy()[0], img)
        assert s1[0]["accepted"] == st["accepted"] and s1[0]["t0"] == st["t0"]
        assert abs(s1[0]["final_cost"] - st["final_cost"]) <= 1e-12 * max(1.0, st["final_cost"])


def test_server_memory_budget_bounds_residency(api):
    """A small budget admits a few chains at a time; every request still
    completes, with the result it has alone."""
    reqs = [r for r in _requests() if r["n"] == 48]
    reqs = [dict(r, seed=r["seed"] + 10 * k) for k in range(6) for r in reqs]
    alone = _run_alone(api, reqs[:3])
    budget = 1_100_000
    with api.Server(stages_per_tick=TICK, mem_budget=budget) as srv:
        tickets = [srv.submit(**r) for r in reqs]
        got = [srv.wait(t, 120000) for t in tickets]
        info = srv.info()
    assert info["completed"] == len(reqs)
    assert info["bytes_peak"] <= budget
    for (ia, sa), (im, sm) in zip(alone, got[:3]):
        assert np.array_equal(ia, im) and sa["accepted"] == sm["accepted"]


def test_server_busy_pending_not_found(api):
    r = _requests()[2]
    long = dict(r, n_sweeps=40)
    with api.Server(stages_per_tick=TICK, max_active=1, queue_limit=2) as srv:
        t1 = srv.submit(**long)
        while srv.info()["admitted"] < 1:
            time.sleep(0.001)
        assert srv.poll(t1) is None  # still running (PENDING)
        t2 = srv.submit(**long)
        t3 = srv.submit(**long)
        with pytest.raises(api.SatpilaError) as ei:
            srv.submit(**long)
        assert ei.value.code == api.ERR_BUSY
        with pytest.raises(api.SatpilaError) as ei:
            srv.poll(123456789)
        assert ei.value.code == api.ERR_NOT_FOUND
        for t in (t1, t2, t3):
            assert srv.wait(t, 120000) is not None
        with pytest.raises(api.SatpilaError) as ei:
            srv.poll(t1)  # already collected
        assert ei.value.code == api.ERR_NOT_FOUND
    with api.Server() as srv:
        with pytest.raises(api.SatpilaError) as ei:
            srv.submit(r["sino"], n=r["n"], bome_k=0)
        assert ei.value.code == api.ERR_INVALID_ARG


def test_served_chain_follows_oracle(api):
    """A request served in a mixed stream (FP16 table, Poisson noise, K = 8,
    the FP64-grade resync every tick), followed move by move by the oracle:
    the served image equals sat_run's on that chain with resync_every =
    stages_per_tick (bit for bit), and that run's trace is followed by the
    oracle over the same binary16 lengths (decisions, Eq. (7) sums, T0)."""
    n, U, K, S = 96, 72, 8, 6
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    ph = synth.phantom(n, 12, 321) * mask
    pm = synth.poisson_noise(oracle.drt(ph, U, B), 1e5, 654).astype(np.float32)
    target = dict(sino=pm, n=n, precision=api.PILA_F16, mask=mask, bome_k=K, n_sweeps=S, seed=4242, t0=-1.0, tn=-1.0)
    reqs = _requests()
    with api.Server(stages_per_tick=TICK) as srv:
        tickets = [srv.submit(**r) for r in reqs[:4]]
        tt = srv.submit(**target)
        tickets += [srv.submit(**r) for r in reqs[4:]]
        img, st = srv.wait(tt, 120000)
        for t in tickets:
            assert srv.wait(t, 120000) is not None
    assert st["status"] == 0
    M = int(mask.sum())
    img0 = synth.initial_image(n, 0.5, mask).astype(np.float32)
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    ref = torch.tensor(img0[None], device="cuda")
    trace = torch.zeros(S * M * api.TRACE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    s1 = api.sat_run(p, torch.tensor(pm[None], device="cuda"), ref, bome_k=K, n_sweeps=S, seed=4242, t0=-1.0,
                     tn=-1.0, resync_every=TICK, trace_chain=0, trace=trace, plan=api.SAT_PLAN_WINDOW_G4)
    api.pila_free(p)
    assert np.array_equal(ref.cpu().numpy()[0], img)
    assert s1[0]["accepted"] == st["accepted"] and s1[0]["t0"] == st["t0"]
    tr = np.frombuffer(trace.cpu().numpy().tobytes(), dtype=api.TRACE_DTYPE)
    t0, found = oracle.sat_t0(pm, img0, seed=4242, mask=mask, length_format=oracle.LEN_BINARY16)
    assert found == st["t0_found"] == 200 and abs(st["t0"] - t0) <= 1e-4 * t0
    _, rep = oracle.sat_lockstep(pm, img0, tr, t0=st["t0"], tn=st["tn"], bome_k=K, n_sweeps=S, seed=4242, mask=mask,
                                 length_format=oracle.LEN_BINARY16)
    assert rep["moves"] == S * M
    assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
    assert rep["max_err_dS"] <= 1e-5 and rep["max_err_f"] <= 1e-5, rep
    assert rep["near_ties"] <= 1e-3 * S * M, rep


def test_server_wide_tables_share_a_launch(api):
    """Tables of 200-400 angles (all three precisions) served together in one
    image size's launch: the records of a lane's second chunk pair are real
    angles here.  Each result equals sat_run's with the 4-warp group layout."""
    n = 64
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    shapes = [(300, api.PILA_F16, 4), (200, api.PILA_U8, 8), (400, api.PILA_F32, 1), (300, api.PILA_F16, 8)]
    reqs = []
    for i, (U, prec, K) in enumerate(shapes):
        ph = synth.phantom(n, 6, 700 + i) * mask
        sino = oracle.drt(ph, U, B).astype(np.float32)
        reqs.append(dict(sino=sino, n=n, precision=prec, mask=mask, bome_k=K, n_sweeps=4, seed=1300 + i,
                         t0=-1.0, tn=-1.0))
    with api.Server(stages_per_tick=2) as srv:
        tickets = [srv.submit(**r) for r in reqs]
        got = [srv.wait(t, 120000) for t in tickets]
    for (img, st), r in zip(got, reqs):
        assert st["status"] == 0
        U = r["sino"].shape[0]
        p = api.pila_build(n, U, B, r["precision"], mask=mask)
        ref = torch.tensor(synth.initial_image(n, 0.5, mask).astype(np.float32)[None], device="cuda")
        kw = {k: v for k, v in r.items() if k not in ("sino", "n", "precision", "mask")}
        s1 = api.sat_run(p, torch.tensor(r["sino"][None], device="cuda"), ref, resync_every=2,
                         plan=api.SAT_PLAN_WINDOW_G4, **kw)
        api.pila_free(p)
        assert np.array_equal(ref.cpu().numpy()[0], img)
        assert s1[0]["accepted"] == st["accepted"] and s1[0]["t0"] == st["t0"]
