"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on
the same seeded inputs.  Tolerances:
  * PILA bins bit-exact; FP32 lengths within 1e-6 relative (+1e-9 absolute,
    entries shorter than 1e-9 are edge grazes and may be absent on one side);
    FP16 lengths within half an FP16 ulp (2^-11 relative + 6e-8);
  * per-move Eq. (7) sums within 1e-5 of the magnitude of their terms
    (2|df| sum|r l| + df^2 sum l^2) in FP32 mode; accept decisions identical
    except recorded near-ties (the oracle's own margin below 2e-5 of the
    term magnitude);
  * final image RMSE against the phantom within 2% of the oracle's.
"""
import math

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


def dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda").contiguous()


def compact(bins, lens, floor):
    """Drop entries shorter than floor and left-align the two slots."""
    b = np.where(lens > floor, bins, -1).astype(np.int64)
    l = np.where(lens > floor, lens, 0.0).astype(np.float64)
    move = (b[..., 0] < 0) & (b[..., 1] >= 0)
    b[move, 0], l[move, 0] = b[move, 1], l[move, 1]
    b[move, 1], l[move, 1] = -1, 0.0
    return b, l


GEOMS = [(64, 90, 91, None), (37, 45, 53, None), (16, 7, 23, None), (5, 3, 7, None), (1, 4, 1, None),
         (24, 33, 35, "random")]


@pytest.mark.parametrize("n,U,B,ang", GEOMS)
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_pila_matches_oracle(api, n, U, B, ang, prec):
    angles = None
    if ang == "random":
        angles = np.sort(np.random.default_rng(3).uniform(0, np.pi, U))
    ob, ol = oracle.pila(n, U, B, angles)
    p = api.pila_build(n, U, B, prec, angles=angles)
    gb, gl = api.pila_export(p)
    info = api.pila_info(p)
    assert info["record_bytes"] == {0: 16, 1: 8, 2: 4}[prec]
    if prec == 2:
        # one-byte lengths (q / 180, Sec. II-B): entries longer than half a
        # unit are present, on the same bins, within half a unit; shorter ones
        # are absent (records holding an entry within 1e-7 of half a unit,
        # where rounding decides, are left out)
        half = 0.5 / 180.0
        amb = np.any(np.abs(ol - half) < 1e-7, axis=-1)
        ob2, ol2 = compact(ob, ol, half)
        gb2, gl2 = compact(gb, gl.astype(np.float64), half)
        assert np.array_equal(ob2[~amb], gb2[~amb])
        assert np.all(np.abs(gl2 - ol2)[~amb] <= half + 1e-7)
        assert info["entries"] == int((gl > 0).sum())
        api.pila_free(p)
        return
    ob_, ol_ = compact(ob, ol, 1e-9)
    gb_, gl_ = compact(gb, gl.astype(np.float64), 1e-9)
    if prec == 0:
        assert np.array_equal(ob_, gb_)
        assert np.all(np.abs(gl_ - ol_) <= 1e-6 * ol_ + 1e-9)
    else:
        # an FP16 length can flush to zero only below 2^-25
        ok = (ob_ == gb_) | ((gb_ < 0) & (ol_ < 3e-8))
        assert np.all(ok)
        assert np.all(np.abs(gl_ - ol_) <= 2.0**-11 * ol_ + 6e-8)
    assert info["entries"] == int((gl > 0).sum())
    api.pila_free(p)


@pytest.mark.parametrize("prec", [0, 1])
def test_pila_full_size_sampled_rays(api, prec):
    """512^2, 360 angles, 725 bins: sampled rays traversed by the oracle one
    by one against the device table (gathered on the device)."""
    n, U, B = 512, 360, 725
    p = api.pila_build(n, U, B, prec)
    P = n * n
    bins = torch.empty((P, U, 2), dtype=torch.int32, device="cuda")
    lens = torch.empty((P, U, 2), dtype=torch.float32, device="cuda")
    api.pila_export(p, bins, lens)
    rng = np.random.default_rng(11)
    for _ in range(120):
        u, k = int(rng.integers(U)), int(rng.integers(B))
        pix, ln = oracle.siddon_ray(n, math.pi * u / U, k - 0.5 * (B - 1))
        keep = ln > 1e-9
        pix, ln = pix[keep], ln[keep]
        if len(pix) == 0:
            continue
        pt = torch.tensor(pix, dtype=torch.long, device="cuda")
        gb = bins[pt, u].cpu().numpy()
        gl = lens[pt, u].cpu().numpy().astype(np.float64)
        hit = gb == k
        assert np.all(hit.sum(axis=1) == 1), (u, k)
        got = (gl * hit).sum(axis=1)
        tol = (1e-6 * ln + 1e-9) if prec == 0 else (2.0**-11 * ln + 6e-8)
        assert np.all(np.abs(got - ln) <= tol)
        # and no other pixel of this ray's angle claims bin k: total count check
    api.pila_free(p)
    del bins, lens
    torch.cuda.empty_cache()


def test_forward_projection(api):
    n, U, B = 64, 90, 91
    rng = np.random.default_rng(5)
    img = rng.random((2, n, n)).astype(np.float32)
    p = api.pila_build(n, U, B, api.PILA_F32)
    out = api.pila_forward(p, dev(img))
    got = out.cpu().numpy()
    gb, gl = api.pila_export(p)
    # exact FP64 sum over the stored lengths
    want = np.zeros((2, U, B))
    for s in range(2):
        ok = gl[:, :, s] > 0
        pp, uu = np.nonzero(ok)
        for i in range(2):
            np.add.at(want[i], (uu, gb[pp, uu, s]), img[i].reshape(-1)[pp].astype(np.float64) * gl[pp, uu, s])
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    # against the oracle's ray-driven DRT (FP32 length rounding only)
    for i in range(2):
        drt = oracle.drt(img[i].astype(np.float64), U, B)
        assert np.max(np.abs(got[i] - drt)) <= 2e-7 * np.max(np.abs(drt))
    # host input/output path
    h = api.pila_forward(p, img)
    assert np.array_equal(h, got)
    api.pila_free(p)


class _pixel_projector:
    """Selects the pixel-driven projector for the calls inside the block."""

    def __enter__(self):
        import os

        os.environ["SATPILA_PROJECTOR"] = "pixel"

    def __exit__(self, *exc):
        import os

        os.environ.pop("SATPILA_PROJECTOR", None)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("n,U,B,items", [(64, 90, 91, 1), (48, 40, 69, 3), (37, 45, 53, 24), (50, 33, 71, 45),
                                          (128, 120, 181, 64)])
def test_ray_projector_bit_identical_to_pixel_projector(api, prec, n, U, B, items):
    """The ray-driven projector (ray-major index, sums in registers) adds the
    same exact fixed-point terms as the pixel-driven one: projections equal
    to the bit, in the entry-lanes form (few images) and the image-lanes form
    (24 and more; ragged last group), with zero and negative pixels."""
    rng = np.random.default_rng(n + U + items)
    img = rng.random((items, n, n)).astype(np.float32)
    img[:, :3, :] = 0.0
    img[0, n // 2, :] = -0.25
    p = api.pila_build(n, U, B, prec)
    got = api.pila_forward(p, dev(img)).cpu().numpy()
    with _pixel_projector():
        ref = api.pila_forward(p, dev(img)).cpu().numpy()
    assert np.array_equal(got, ref)
    api.pila_free(p)


@pytest.mark.parametrize("chains", [5, 30])
def test_ray_projector_resync_and_sirt_bit_identical(api, chains):
    """Annealing with a resync after every stage, and SIRT, give bit-identical
    images, costs and drifts with either projector (the per-angle sums of
    squares are formed in the same fixed order)."""
    n, U = 48, 60
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    sinos = np.stack([oracle.drt(synth.phantom(n, 6, 70 + i) * mask, U, B) for i in range(chains)]).astype(np.float32)
    img0 = np.stack([synth.initial_image(n, 0.5, mask)] * chains).astype(np.float32)
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    kw = dict(bome_k=4, n_sweeps=4, t0=-1.0, tn=-1.0, seed=91, resync_every=1, flags=api.SAT_FLAG_NO_GRAPH)
    a = dev(img0)
    st_a = api.sat_run(p, dev(sinos), a, **kw)
    with _pixel_projector():
        b = dev(img0)
        st_b = api.sat_run(p, dev(sinos), b, **kw)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    for x, y in zip(st_a, st_b):
        for k in ("t0", "initial_cost", "final_cost", "final_cost_incremental", "max_resync_drift", "accepted"):
            assert x[k] == y[k], k
    sa, ca = dev(img0[:3]), torch.zeros((3, 5), dtype=torch.float64, device="cuda")
    api.sirt_run(p, dev(sinos[:3]), sa, n_iter=5, costs=ca)
    with _pixel_projector():
        sb, cb = dev(img0[:3]), torch.zeros((3, 5), dtype=torch.float64, device="cuda")
        api.sirt_run(p, dev(sinos[:3]), sb, n_iter=5, costs=cb)
    assert np.array_equal(sa.cpu().numpy(), sb.cpu().numpy())
    assert np.array_equal(ca.cpu().numpy(), cb.cpu().numpy())
    # the SIRT factor matrix of a fresh table, built either way
    q = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    w_ray = api.pila_sirt_factor(q)
    api.pila_free(q)
    with _pixel_projector():
        q = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
        w_pix = api.pila_sirt_factor(q)
        api.pila_free(q)
    assert np.array_equal(w_ray, w_pix)
    api.pila_free(p)


def test_sirt_factor(api):
    n, U = 48, 30
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    p = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    w = api.pila_sirt_factor(p)
    want = oracle.sirt_factor(n, U, B, mask)
    assert np.max(np.abs(w - want)) <= 1e-6 * np.max(want)
    api.pila_free(p)


def _plain64():
    cfg = synth.WORKLOADS["plain64"]
    n, U, B = cfg["n"], cfg["n_angles"], cfg["n_bins"]
    ph = synth.phantom(n, cfg["ellipses"], 1000)
    pm = oracle.drt(ph, U, B)
    return cfg, n, U, B, ph, pm


def _run_traced(api, p, pm, img0, S, M, **kw):
    U, B = pm.shape
    n = img0.shape[0]
    trace = torch.zeros(S * M * 32, dtype=torch.uint8, device="cuda")
    img = dev(img0).reshape(1, n, n)
    st = api.sat_run(p, dev(pm).reshape(1, U, B), img, n_sweeps=S, trace_chain=0, trace=trace, **kw)
    tr = np.frombuffer(trace.cpu().numpy().tobytes(), dtype=api.TRACE_DTYPE)
    return st[0], tr, img.cpu().numpy()[0]


@pytest.mark.parametrize("W", [1, 2, 4])
def test_sat_lockstep_plain64(api, W):
    """The plain 64^2 workload (90 angles, K=1, T0=1e-2 -> 0, 20 stages):
    every move compared with the oracle, for 1, 2 and 4 warps per chain."""
    cfg, n, U, B, ph, pm = _plain64()
    img0 = np.full((n, n), 0.5)
    p = api.pila_build(n, U, B, api.PILA_F32)
    S, M = cfg["n_sweeps"], n * n
    st, tr, img = _run_traced(api, p, pm, img0, S, M, bome_k=1, t0=cfg["t0"], tn=cfg["tn"], seed=3000,
                              resync_every=1, group_warps=W)
    assert st["status"] == 0 and st["proposed"] == S * M
    _, rep = oracle.sat_lockstep(pm, img0, tr, t0=st["t0"], tn=st["tn"], bome_k=1, n_sweeps=S, seed=3000)
    assert rep["moves"] == S * M
    assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
    assert rep["max_err_dS"] <= 1e-5 and rep["max_err_dC"] <= 1e-5, rep
    assert rep["near_ties"] <= 1e-3 * S * M, rep
    assert st["max_resync_drift"] <= 1e-4 * np.max(np.abs(pm))
    api.pila_free(p)


def test_near_tie_count_changes_no_result(api):
    """Counting near-ties (SAT_FLAG_NEAR_TIES) adds a reduction but changes no
    decision: images and costs equal a run without it, on the windowed
    layouts; other layouts report -1."""
    n, U = 48, 60
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    C = 6
    sinos = np.stack([oracle.drt(synth.phantom(n, 6, 90 + i) * mask, U, B) for i in range(C)]).astype(np.float32)
    img0 = np.stack([synth.initial_image(n, 0.5, mask)] * C).astype(np.float32)
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    for plan in (api.SAT_PLAN_WINDOW_SMEM, api.SAT_PLAN_WINDOW_GLOBAL, api.SAT_PLAN_WINDOW_G2, api.SAT_PLAN_PIPE_1):
        kw = dict(bome_k=4, n_sweeps=3, t0=-1.0, tn=-1.0, seed=5, plan=plan)
        a, b = dev(img0), dev(img0)
        sa = api.sat_run(p, dev(sinos), a, **kw)
        sb = api.sat_run(p, dev(sinos), b, flags=api.SAT_FLAG_NEAR_TIES, **kw)
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
        assert [x["final_cost"] for x in sa] == [x["final_cost"] for x in sb]
        assert all(x["near_ties"] == -1 for x in sa)
        if plan == api.SAT_PLAN_PIPE_1:
            assert all(x["near_ties"] == -1 for x in sb)
        else:
            assert all(0 <= x["near_ties"] <= x["proposed"] for x in sb)
    api.pila_free(p)


@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("layout", ["window", "pipelined2", "window_groups4"])
def test_sat_schedules_lockstep(api, schedule, layout):
    """The geometric (8b) and cubic (9) schedules of Sec. III-C on the plain
    64^2 workload (90 angles, K = 4): every move of 20 stages compared with
    the oracle, on the windowed, pipelined and grouped-window kernels."""
    cfg, n, U, B, ph, pm = _plain64()
    img0 = np.full((n, n), 0.5)
    p = api.pila_build(n, U, B, api.PILA_F32)
    S, M = cfg["n_sweeps"], n * n
    t0, tn = 1e-2, 1e-5
    kw = {"window": dict(residency=1), "pipelined2": dict(group_warps=2),
          "window_groups4": dict(group_warps=4, flags=api.SAT_FLAG_WINDOW_GROUPS)}[layout]
    st, tr, img = _run_traced(api, p, pm, img0, S, M, bome_k=4, t0=t0, tn=tn, seed=3100 + schedule,
                              schedule=schedule, resync_every=5, **kw)
    assert st["status"] == 0 and st["proposed"] == S * M
    assert st["plan"] == {"window": api.SAT_PLAN_WINDOW_SMEM, "pipelined2": api.SAT_PLAN_PIPE_2,
                          "window_groups4": api.SAT_PLAN_WINDOW_G4}[layout]
    _, rep = oracle.sat_lockstep(pm, img0, tr, t0=st["t0"], tn=st["tn"], bome_k=4, n_sweeps=S, seed=3100 + schedule,
                                 schedule=schedule)
    assert rep["moves"] == S * M
    assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
    assert rep["max_err_dS"] <= 1e-5 and rep["max_err_dC"] <= 1e-5, rep
    assert rep["near_ties"] <= 1e-3 * S * M, rep
    # uphill moves were decided at the stage temperatures (the oracle takes
    # them from its own closed forms, so a wrong temperature is a mismatch)
    assert np.count_nonzero((tr["accepted"] == 1) & (tr["dC"] > 0)) > 0
    api.pila_free(p)


@pytest.mark.parametrize("K,res,W", [(8, 0, 0), (8, 2, 1), (32, 2, 4), (3, 0, 2)])
def test_sat_lockstep_bome_with_mask(api, K, res, W):
    """256^2-geometry slice (180 angles, 363 bins) with the disk reconstruction
    space, Gaussian noise, BoME, T0 by Eq. (8): two stages in lockstep."""
    n, U, B = 256, 180, 363
    ph = synth.phantom(n, 20, 1001)
    mask = synth.disk_mask(n)
    pm = synth.gaussian_noise(oracle.drt(ph, U, B), 0.01, 2001)
    img0 = synth.initial_image(n, 0.5, mask)
    p = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    S, M = 2, 6000
    st, tr, img = _run_traced(api, p, pm, img0, S, M, bome_k=K, t0=-1.0, tn=-1.0, seed=3001, moves_per_sweep=M,
                              residency=res, group_warps=W)
    t0, found = oracle.sat_t0(pm, img0, seed=3001, mask=mask)
    assert found == st["t0_found"] == 200
    assert abs(st["t0"] - t0) <= 1e-4 * t0
    _, rep = oracle.sat_lockstep(pm, img0, tr, t0=st["t0"], tn=st["tn"], bome_k=K, n_sweeps=S, seed=3001,
                                 moves_per_sweep=M, mask=mask)
    assert rep["moves"] == S * M
    assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
    assert rep["max_err_dS"] <= 1e-5, rep
    api.pila_free(p)


def test_sat_batched_equals_single_and_residency_identical(api):
    n, U = 48, 40
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    sinos = np.stack([oracle.drt(synth.phantom(n, 6, 50 + i), U, B) for i in range(5)]).astype(np.float32)
    img0 = np.stack([synth.initial_image(n, 0.5, mask)] * 5).astype(np.float32)
    p = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    kw = dict(bome_k=4, n_sweeps=6, t0=-1.0, tn=-1.0, resync_every=2, group_warps=2)
    outs = {}
    for res in (1, 2):
        imgs = dev(img0)
        st = api.sat_run(p, dev(sinos), imgs, seed=77, residency=res, **kw)
        outs[res] = (imgs.cpu().numpy(), [s["accepted"] for s in st], [s["final_cost"] for s in st])
    assert np.array_equal(outs[1][0], outs[2][0]) and outs[1][1] == outs[2][1]
    for c in (0, 3):
        one = dev(img0[c:c + 1])
        st = api.sat_run(p, dev(sinos[c:c + 1]), one, seed=77 + c, **kw)
        assert np.array_equal(one.cpu().numpy()[0], outs[1][0][c])
        assert st[0]["accepted"] == outs[1][1][c]
    api.pila_free(p)


def test_sat_final_rmse_plain64_vs_oracle(api):
    cfg, n, U, B, ph, pm = _plain64()
    img0 = np.full((n, n), 0.5)
    p = api.pila_build(n, U, B, api.PILA_F32)
    img = dev(img0).reshape(1, n, n)
    st = api.sat_run(p, dev(pm).reshape(1, U, B), img, bome_k=1, n_sweeps=cfg["n_sweeps"], t0=cfg["t0"],
                     tn=cfg["tn"], seed=3000)
    oimg, ost, _ = oracle.sat_run(pm, img0, bome_k=1, n_sweeps=cfg["n_sweeps"], t0=cfg["t0"], tn=cfg["tn"],
                                  seed=3000)
    r_gpu = synth.rmse(img.cpu().numpy()[0], ph)
    r_orc = synth.rmse(oimg, ph)
    assert abs(r_gpu - r_orc) <= 0.02 * r_orc, (r_gpu, r_orc)
    assert abs(st[0]["final_cost"] - ost["final_cost_fresh"]) <= 0.02 * ost["final_cost_fresh"]
    api.pila_free(p)


def test_sat256_free_running_rmse_vs_oracle(api):
    """The 256^2 SAT configuration in full (180 angles, 363 bins, disk space,
    Gaussian noise at 1%, K = 8, T0 by Eq. (8), 100 stages of the whole
    reconstruction space, FP32 table), free running on both sides: final RMSE
    against the phantom and final Eq. (4) cost within 2% of the oracle's."""
    cfg = synth.WORKLOADS["sat256"]
    n, U, B, K, S = cfg["n"], cfg["n_angles"], cfg["n_bins"], cfg["bome_k"], cfg["n_sweeps"]
    mask = synth.disk_mask(n)
    ph = synth.phantom(n, cfg["ellipses"], synth.slice_seeds(0)[0]) * mask
    pm = synth.gaussian_noise(oracle.drt(ph, U, B), cfg["noise"][1], synth.slice_seeds(0)[1]).astype(np.float32)
    img0 = synth.initial_image(n, 0.5, mask)
    seed = synth.slice_seeds(0)[2]
    p = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    img = dev(img0).reshape(1, n, n)
    st = api.sat_run(p, dev(pm).reshape(1, U, B), img, bome_k=K, n_sweeps=S, t0=-1.0, tn=-1.0, seed=seed)
    api.pila_free(p)
    assert st[0]["status"] == 0
    oimg, ost, _ = oracle.sat_run(pm, img0, bome_k=K, n_sweeps=S, seed=seed, mask=mask)
    r_gpu, r_orc = synth.rmse(img.cpu().numpy()[0], ph, mask), synth.rmse(oimg, ph, mask)
    assert abs(r_gpu - r_orc) <= 0.02 * r_orc, (r_gpu, r_orc)
    assert abs(st[0]["final_cost"] - ost["final_cost_fresh"]) <= 0.02 * ost["final_cost_fresh"]


def test_sat_u8_table(api):
    """The one-byte table of Sec. II-B (lengths q / 180): its forward
    projection is the exact sum of its stored lengths, the windowed kernel
    gives the same chain whichever memory holds the residual, follows the
    oracle move by move over the same one-byte lengths, and the final
    RMSE of the 128^2 / 120-angle slice stays within 5% of the FP64 oracle's
    (exact lengths); the FP16 table's is within 2% (next test)."""
    n, U, B = 128, 120, 181
    ph = synth.phantom(n, 20, 1002)
    mask = synth.disk_mask(n)
    pm = oracle.drt(ph, U, B)
    img0 = synth.initial_image(n, 0.5, mask)
    p = api.pila_build(n, U, B, api.PILA_U8, mask=mask)
    bins, lens = api.pila_export(p)
    x = np.random.default_rng(8).random((n, n)).astype(np.float32)
    fwd = api.pila_forward(p, dev(x).reshape(1, n, n)).cpu().numpy()[0]
    ref = np.zeros((U, B))
    P = n * n
    pix = np.repeat(np.arange(P), U * 2).reshape(P, U, 2)
    ang = np.tile(np.repeat(np.arange(U), 2).reshape(U, 2), (P, 1, 1))
    ok = bins >= 0
    np.add.at(ref, (ang[ok], bins[ok]), lens[ok].astype(np.float64) * x.ravel()[pix[ok]])
    assert np.max(np.abs(fwd - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))
    kw = dict(bome_k=4, n_sweeps=8, t0=-1.0, tn=-1.0, seed=3002)
    outs = []
    for res in (api.SAT_RESIDENT_SMEM, api.SAT_RESIDENT_GLOBAL):
        img = dev(img0).reshape(1, n, n)
        st = api.sat_run(p, dev(pm).reshape(1, U, B), img, residency=res, **kw)
        assert st[0]["status"] == 0
        outs.append(img.cpu().numpy()[0])
    assert np.array_equal(outs[0], outs[1])
    # move by move against the oracle over the same one-byte lengths
    S, M = kw["n_sweeps"], int(mask.sum())
    st, tr, img = _run_traced(api, p, pm.astype(np.float32), img0, S, M, residency=api.SAT_RESIDENT_SMEM, **{
        k: v for k, v in kw.items() if k != "n_sweeps"})
    assert np.array_equal(img, outs[0])
    t0, found = oracle.sat_t0(pm.astype(np.float32), img0, seed=kw["seed"], mask=mask,
                              length_format=oracle.LEN_BYTE180)
    assert found == st["t0_found"] == 200 and abs(st["t0"] - t0) <= 1e-4 * t0
    _, rep = oracle.sat_lockstep(pm.astype(np.float32), img0, tr, t0=st["t0"], tn=st["tn"], bome_k=4, n_sweeps=S,
                                 seed=kw["seed"], mask=mask, length_format=oracle.LEN_BYTE180)
    assert rep["moves"] == S * M
    assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
    assert rep["max_err_dS"] <= 1e-5, rep
    oimg, ost, _ = oracle.sat_run(pm, img0, mask=mask, **kw)
    r_gpu, r_orc = synth.rmse(outs[0], ph, mask), synth.rmse(oimg, ph, mask)
    assert abs(r_gpu - r_orc) <= 0.05 * r_orc, (r_gpu, r_orc)
    with pytest.raises(api.SatpilaError):
        api.sat_run(p, dev(pm).reshape(1, U, B), dev(img0).reshape(1, n, n), pipeline_depth=4, **kw)
    api.pila_free(p)


def test_sat_f16_rmse_vs_oracle(api):
    """128^2 slice of the batched workload shape with the FP16 PILA: final
    RMSE within 2% of the FP64 oracle's (which uses exact lengths)."""
    n, U, B = 128, 120, 181
    ph = synth.phantom(n, 20, 1002)
    mask = synth.disk_mask(n)
    pm = oracle.drt(ph, U, B)
    img0 = synth.initial_image(n, 0.5, mask)
    kw = dict(bome_k=4, n_sweeps=8, t0=-1.0, tn=-1.0, seed=3002)
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    img = dev(img0).reshape(1, n, n)
    api.sat_run(p, dev(pm).reshape(1, U, B), img, **kw)
    oimg, ost, _ = oracle.sat_run(pm, img0, mask=mask, **kw)
    r_gpu, r_orc = synth.rmse(img.cpu().numpy()[0], ph, mask), synth.rmse(oimg, ph, mask)
    assert abs(r_gpu - r_orc) <= 0.02 * r_orc, (r_gpu, r_orc)
    api.pila_free(p)


def test_sat_edge_cases(api):
    n, U = 9, 7
    B = synth.bins_for(n)
    pm = oracle.drt(synth.phantom(n, 3, 9), U, B)
    p = api.pila_build(n, U, B, api.PILA_F32)
    img0 = np.full((n, n), 0.5)
    # no stages: image unchanged, final cost = initial cost
    img = dev(img0).reshape(1, n, n)
    st = api.sat_run(p, dev(pm).reshape(1, U, B), img, n_sweeps=0)
    assert np.array_equal(img.cpu().numpy()[0], img0.astype(np.float32))
    assert st[0]["final_cost"] == st[0]["initial_cost"] and st[0]["proposed"] == 0
    # one move per stage, K = 32, in lockstep
    st, tr, _ = _run_traced(api, p, pm, img0, 3, 1, bome_k=32, t0=1e-3, tn=1e-5, seed=5, moves_per_sweep=1)
    _, rep = oracle.sat_lockstep(pm, img0, tr, t0=st["t0"], tn=st["tn"], bome_k=32, n_sweeps=3, seed=5,
                                 moves_per_sweep=1)
    assert rep["moves"] == 3 and rep["hard_mismatch"] == -1 and rep["pixel_mismatch"] == -1
    # empty reconstruction space: nothing moves
    q = api.pila_build(n, U, B, api.PILA_F32, mask=np.zeros((n, n), np.uint8))
    img = dev(img0).reshape(1, n, n)
    st = api.sat_run(q, dev(pm).reshape(1, U, B), img, n_sweeps=2, t0=-1.0)
    assert st[0]["proposed"] == 0 and st[0]["t0_found"] == 0
    assert np.array_equal(img.cpu().numpy()[0], img0.astype(np.float32))
    # invalid arguments come back as errors
    with pytest.raises(api.SatpilaError):
        api.sat_run(p, dev(pm).reshape(1, U, B), dev(img0).reshape(1, n, n), bome_k=33)
    with pytest.raises(api.SatpilaError):
        api.sat_run(p, dev(pm).reshape(1, U, B), dev(img0).reshape(1, n, n), beta=0.0)
    # 1x1 image
    one = api.pila_build(1, 5, 1, api.PILA_F32)
    pm1 = oracle.drt(np.full((1, 1), 0.3), 5, 1)
    st, tr, im = _run_traced(api, one, pm1, np.full((1, 1), 0.9), 4, 50, bome_k=2, t0=1e-3, tn=1e-4, seed=1,
                             moves_per_sweep=50)
    _, rep = oracle.sat_lockstep(pm1, np.full((1, 1), 0.9), tr, t0=st["t0"], tn=st["tn"], bome_k=2, n_sweeps=4,
                                 seed=1, moves_per_sweep=50)
    assert rep["hard_mismatch"] == -1 and abs(im[0, 0] - 0.3) < 0.05
    for h in (p, q, one):
        api.pila_free(h)


def test_sat_host_buffers_match_device(api):
    n, U = 32, 30
    B = synth.bins_for(n)
    pm = oracle.drt(synth.phantom(n, 5, 4), U, B).astype(np.float32).reshape(1, U, B)
    img0 = np.full((1, n, n), 0.5, dtype=np.float32)
    p = api.pila_build(n, U, B, api.PILA_F16)
    kw = dict(bome_k=4, n_sweeps=3, seed=9)
    h = img0.copy()
    api.sat_run(p, pm, h, **kw)
    d = dev(img0)
    api.sat_run(p, dev(pm), d, **kw)
    assert np.array_equal(h, d.cpu().numpy())
    api.pila_free(p)


@pytest.mark.parametrize("mode", [0, 1])
def test_sirt_vs_oracle(api, mode):
    n, U = 32, 45
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    ph = synth.phantom(n, 6, 21) * mask
    pm = oracle.drt(ph, U, B)
    img0 = synth.initial_image(n, 0.5, mask)
    p = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    img = dev(img0).reshape(1, n, n)
    costs = torch.zeros((1, 6), dtype=torch.float64, device="cuda")
    api.sirt_run(p, dev(pm).reshape(1, U, B), img, n_iter=6, mode=mode, costs=costs)
    oimg, oc = oracle.sirt_run(pm, img0, 6, mode=mode, mask=mask)
    assert np.max(np.abs(img.cpu().numpy()[0] - oimg)) <= 2e-5 * max(1.0, np.max(np.abs(oimg)))
    assert np.allclose(costs.cpu().numpy()[0], oc, rtol=1e-4)
    api.pila_free(p)


@pytest.mark.parametrize("mode", [0, 1])
def test_sirt_full_size_256(api, mode):
    """SIRT on the 256^2 SAT+SIRT configuration (180 angles, 363 bins, disk
    space, Gaussian noise at 1%): one slice, so the simultaneous mode's
    projections run split into pixel chunks; four iterations against the
    oracle, images within 2e-5 and per-iteration costs within 1e-4."""
    cfg = synth.WORKLOADS["sat256"]
    n, U, B = cfg["n"], cfg["n_angles"], cfg["n_bins"]
    mask = synth.disk_mask(n)
    ph = synth.phantom(n, cfg["ellipses"], synth.slice_seeds(0)[0]) * mask
    pm = synth.gaussian_noise(oracle.drt(ph, U, B), cfg["noise"][1], synth.slice_seeds(0)[1]).astype(np.float32)
    img0 = synth.initial_image(n, 0.5, mask)
    p = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    img = dev(img0).reshape(1, n, n)
    it = 4
    costs = torch.zeros((1, it), dtype=torch.float64, device="cuda")
    api.sirt_run(p, dev(pm).reshape(1, U, B), img, n_iter=it, mode=mode, costs=costs)
    oimg, oc = oracle.sirt_run(pm, img0, it, mode=mode, mask=mask)
    assert np.max(np.abs(img.cpu().numpy()[0] - oimg)) <= 2e-5 * max(1.0, np.max(np.abs(oimg)))
    assert np.allclose(costs.cpu().numpy()[0], oc, rtol=1e-4)
    api.pila_free(p)


def test_batched_workload_full_size_sampled_chains(api):
    """The batched workload at full size, in the launch the benchmark times:
    512 chains of 128^2 slices (disk space, 120 angles, 181 bins), K = 4,
    T0 by Eq. (8), the 50-stage linear schedule, the FP16 table and the
    autotuned layout.  A sampled chain is traced and followed move by move,
    all 644,600 moves, by the oracle over the same binary16 lengths, with T0
    checked against the oracle's Eq. (8); for sampled chains the reported
    final cost equals the oracle's Eq. (4) cost of the returned image through
    the rounded table, and the running FP32 cost stays within 1e-4 of it."""
    cfg = synth.WORKLOADS["batch128x512"]
    n, U, B, K, S, C = cfg["n"], cfg["n_angles"], cfg["n_bins"], cfg["bome_k"], cfg["n_sweeps"], cfg["slices"]
    mask = synth.disk_mask(n)
    M = int(mask.sum())
    distinct = 8
    phs = [synth.phantom(n, cfg["ellipses"], synth.slice_seeds(i)[0]) * mask for i in range(distinct)]
    sinos = np.stack([oracle.drt(ph, U, B) for ph in phs]).astype(np.float32)
    img0 = synth.initial_image(n, 0.5, mask).astype(np.float32)
    seed0 = synth.slice_seeds(0)[2]
    traced = int(np.random.default_rng(11).integers(C))
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    imgs = dev(np.broadcast_to(img0, (C, n, n)))
    trace = torch.zeros(S * M * api.TRACE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    st = api.sat_run(p, dev(sinos[np.arange(C) % distinct]), imgs, bome_k=K, n_sweeps=S, t0=cfg["t0"],
                     tn=cfg["tn"], beta=cfg["beta"], seed=seed0, resync_every=0, plan=api.SAT_PLAN_WINDOW_SMEM,
                     flags=api.SAT_FLAG_NEAR_TIES, trace_chain=traced, trace=trace)
    api.pila_free(p)
    assert all(s["status"] == 0 and s["proposed"] == S * M for s in st)
    # the layout the benchmark pins (the autotuner's pick for this shape)
    assert st[0]["plan"] == api.SAT_PLAN_WINDOW_SMEM
    final = imgs.cpu().numpy()
    tr = np.frombuffer(trace.cpu().numpy().tobytes(), dtype=api.TRACE_DTYPE)
    pm = sinos[traced % distinct]
    t0, found = oracle.sat_t0(pm, img0, seed=seed0 + traced, mask=mask, length_format=oracle.LEN_BINARY16)
    assert found == st[traced]["t0_found"] == 200
    assert abs(st[traced]["t0"] - t0) <= 1e-4 * t0
    _, rep = oracle.sat_lockstep(pm, img0, tr, t0=st[traced]["t0"], tn=st[traced]["tn"], bome_k=K, n_sweeps=S,
                                 seed=seed0 + traced, mask=mask, length_format=oracle.LEN_BINARY16)
    assert rep["moves"] == S * M
    assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
    assert rep["max_err_dS"] <= 1e-5, rep
    assert rep["near_ties"] <= 1e-3 * S * M, rep
    # the device's own count of near-tie decisions: rare, and it includes the
    # decisions where the oracle's FP64 evaluation went the other way
    assert all(0 <= s["near_ties"] <= 1e-3 * S * M for s in st)
    assert rep["near_ties"] <= st[traced]["near_ties"], (rep["near_ties"], st[traced]["near_ties"])
    bins, lens = oracle.pila(n, U, B)
    l16 = lens.astype(np.float16).astype(np.float64)
    ok = l16 > 0
    pix = np.broadcast_to(np.arange(n * n)[:, None, None], l16.shape)[ok]
    ang = np.broadcast_to(np.arange(U)[None, :, None], l16.shape)[ok]
    for c in sorted({0, C // 2, C - 1, traced}):
        proj = np.zeros((U, B))
        np.add.at(proj, (ang, bins[ok]), final[c].astype(np.float64).ravel()[pix] * l16[ok])
        cost = math.sqrt(np.mean((proj - sinos[c % distinct]) ** 2))
        assert abs(st[c]["final_cost"] - cost) <= 1e-9 * cost, (c, st[c]["final_cost"], cost)
        assert abs(st[c]["final_cost_incremental"] - cost) <= 1e-4 * cost
        assert np.all(final[c][mask == 0] == 0.0) and final[c].min() >= 0.0 and final[c].max() <= cfg["beta"]


def test_precision_workload_full_size_sampled_chain(api):
    """The 512^2 workload at full size, in the launch the benchmark times: 304
    chains (2 distinct phantoms, Poisson noise at 1e5 photons), 360 angles,
    725 bins, K = 8, T0 by Eq. (8), 200 stages of 2,058 moves with a resync
    every 20, the FP16 table and the layout the benchmark pins (the windowed
    move on 4 warps per chain).  A sampled chain is followed move by move (all
    411,600 moves) by the oracle over the same binary16 lengths: decisions,
    Eq. (7) sums and the new pixel values, and T0."""
    cfg = synth.WORKLOADS["precision512"]
    n, U, B, K, S = cfg["n"], cfg["n_angles"], cfg["n_bins"], cfg["bome_k"], cfg["n_sweeps"]
    C, distinct = 304, 2
    mask = synth.disk_mask(n)
    M = int(mask.sum()) // 100
    sinos = []
    for i in range(distinct):
        clean = oracle.drt(synth.phantom(n, cfg["ellipses"], synth.slice_seeds(i)[0]) * mask, U, B)
        sinos.append(synth.poisson_noise(clean, cfg["noise"][1], synth.slice_seeds(i)[1]).astype(np.float32))
    sinos = np.stack(sinos)
    img0 = synth.initial_image(n, 0.5, mask).astype(np.float32)
    seed0 = synth.slice_seeds(0)[2]
    traced = int(np.random.default_rng(12).integers(C))
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    imgs = dev(np.broadcast_to(img0, (C, n, n)))
    trace = torch.zeros(S * M * api.TRACE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    st = api.sat_run(p, dev(sinos[np.arange(C) % distinct]), imgs, bome_k=K, n_sweeps=S, moves_per_sweep=M,
                     t0=cfg["t0"], tn=cfg["tn"], beta=cfg["beta"], seed=seed0, plan=api.SAT_PLAN_WINDOW_G4,
                     resync_every=20, flags=api.SAT_FLAG_NEAR_TIES, trace_chain=traced, trace=trace)
    api.pila_free(p)
    assert all(s["status"] == 0 and s["proposed"] == S * M for s in st)
    assert st[0]["plan"] == api.SAT_PLAN_WINDOW_G4
    assert max(s["max_resync_drift"] for s in st) <= 1e-4 * float(np.max(np.abs(sinos)))
    tr = np.frombuffer(trace.cpu().numpy().tobytes(), dtype=api.TRACE_DTYPE)
    pm = sinos[traced % distinct]
    t0, found = oracle.sat_t0(pm, img0, seed=seed0 + traced, mask=mask, length_format=oracle.LEN_BINARY16)
    assert found == st[traced]["t0_found"] == 200
    assert abs(st[traced]["t0"] - t0) <= 1e-4 * t0
    _, rep = oracle.sat_lockstep(pm, img0, tr, t0=st[traced]["t0"], tn=st[traced]["tn"], bome_k=K, n_sweeps=S,
                                 moves_per_sweep=M, seed=seed0 + traced, mask=mask,
                                 length_format=oracle.LEN_BINARY16)
    assert rep["moves"] == S * M
    assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
    assert rep["max_err_dS"] <= 1e-5 and rep["max_err_f"] <= 1e-5, rep
    assert rep["near_ties"] <= 1e-3 * S * M, rep
    # the device's count of decisions within 2e-5 of their term scale: with
    # ~720 terms per sum and 8 estimates more of them sit in that margin, but
    # it still includes every decision the oracle saw go the other way
    ties = [s["near_ties"] for s in st]
    assert min(ties) >= 0 and max(ties) <= 0.02 * S * M, (min(ties), max(ties))
    assert rep["near_ties"] <= st[traced]["near_ties"], (rep["near_ties"], st[traced]["near_ties"])
    final = imgs[traced].cpu().numpy()
    assert np.all(final[mask == 0] == 0.0) and final.min() >= 0.0 and final.max() <= cfg["beta"]


def test_resync_drift_bound_512(api):
    """One stage of the 512^2 precision workload shape (360 angles, 725
    bins, Poisson noise) with the residual in global memory: the
    incremental residual stays within 1e-4 * max|P_m| of a fresh one."""
    n, U, B = 512, 360, 725
    mask = synth.disk_mask(n)
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    ph = synth.phantom(n, 40, 1003)
    clean = api.pila_forward(p, dev(ph[None])).cpu().numpy()[0]
    pm = synth.poisson_noise(clean, 1e5, 2003).astype(np.float32)
    img = dev(synth.initial_image(n, 0.5, mask)).reshape(1, n, n)
    st = api.sat_run(p, dev(pm).reshape(1, U, B), img, bome_k=8, n_sweeps=1, moves_per_sweep=100000, seed=3003,
                     resync_every=1)
    assert st[0]["status"] == 0
    assert st[0]["max_resync_drift"] <= 1e-4 * float(np.max(np.abs(pm)))
    assert abs(st[0]["final_cost_incremental"] - st[0]["final_cost"]) <= 1e-4 * st[0]["final_cost"]
    assert st[0]["final_cost"] < st[0]["initial_cost"]
    api.pila_free(p)


def test_window_kernel_identical_in_shared_and_global_memory(api):
    """The windowed move runs the same arithmetic whichever memory holds the
    residual, so both residencies give bit-identical chains."""
    n, U = 40, 36
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    sinos = np.stack([oracle.drt(synth.phantom(n, 6, 70 + i), U, B) for i in range(3)]).astype(np.float32)
    img0 = np.stack([synth.initial_image(n, 0.5, mask)] * 3).astype(np.float32)
    for prec in (0, 1):
        p = api.pila_build(n, U, B, prec, mask=mask)
        outs = []
        for res in (1, 2):
            imgs = dev(img0)
            st = api.sat_run(p, dev(sinos), imgs, bome_k=4, n_sweeps=4, seed=5, residency=res, group_warps=1)
            outs.append((imgs.cpu().numpy(), [s["accepted"] for s in st]))
        assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
        api.pila_free(p)


def test_window_band_residual_off_centre_mask(api):
    """A shared-memory windowed warp keeps only the band of bins that moves
    can touch.  With an off-centre rectangular reconstruction space the band
    is narrow and starts off a 16-byte boundary: the chain must still follow
    the oracle move by move and equal its run with the residual in global
    memory."""
    n, U = 40, 36
    B = synth.bins_for(n)
    mask = np.zeros((n, n), np.uint8)
    mask[5:21, 23:36] = 1
    ph = synth.phantom(n, 6, 1003) * (0.5 + 0.5 * mask)
    pm = oracle.drt(ph, U, B)
    img0 = np.where(mask > 0, 0.5, 0.0)
    M, S = int(mask.sum()) * 2, 3
    for prec in (0, 1):
        p = api.pila_build(n, U, B, prec, mask=mask)
        outs = []
        for res in (api.SAT_RESIDENT_SMEM, api.SAT_RESIDENT_GLOBAL):
            st, tr, img = _run_traced(api, p, pm, img0, S, M, bome_k=4, t0=1e-3, tn=1e-5, seed=3003,
                                      moves_per_sweep=M, residency=res, group_warps=1)
            assert st["status"] == 0
            outs.append((img, st["accepted"], tr))
        assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
        assert np.all(outs[0][0][mask == 0] == 0.0)
        if prec == 0:
            _, rep = oracle.sat_lockstep(pm, img0, outs[0][2], t0=1e-3, tn=1e-5, bome_k=4, n_sweeps=S, seed=3003,
                                         moves_per_sweep=M, mask=mask)
            assert rep["moves"] == S * M
            assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
            assert rep["max_err_dS"] <= 1e-5, rep
        api.pila_free(p)


@pytest.mark.parametrize("prec", [0, 1])
def test_window_pixel_repeats_and_ragged_last_window(api, prec):
    """A reconstruction space of two adjacent pixels makes the two moves of a
    window draw the same pixel about half the time (the windowed kernel then
    recomputes the later move's candidates after the earlier decision) and
    their footprints share cells at every angle; an odd number of moves per
    stage leaves a ragged last window.  Both residencies follow the oracle
    move by move (the FP16 table over binary16 lengths)."""
    n, U = 24, 30
    B = synth.bins_for(n)
    mask = np.zeros((n, n), np.uint8)
    mask[11, 12] = mask[12, 12] = 1
    pm = oracle.drt(synth.phantom(n, 4, 1004), U, B).astype(np.float32)
    img0 = np.where(mask > 0, 0.5, 0.0)
    S, M = 3, 401
    fmt = oracle.LEN_EXACT if prec == api.PILA_F32 else oracle.LEN_BINARY16
    p = api.pila_build(n, U, B, prec, mask=mask)
    imgs = []
    for res in (api.SAT_RESIDENT_SMEM, api.SAT_RESIDENT_GLOBAL):
        st, tr, img = _run_traced(api, p, pm, img0, S, M, bome_k=4, t0=1e-3, tn=1e-5, seed=3004,
                                  moves_per_sweep=M, residency=res, group_warps=1)
        assert st["status"] == 0 and st["proposed"] == S * M
        pix = tr["pixel"].reshape(S, M)[:, :M - 1].reshape(S, -1, 2)
        assert np.mean(pix[..., 0] == pix[..., 1]) > 0.3
        _, rep = oracle.sat_lockstep(pm, img0, tr, t0=st["t0"], tn=st["tn"], bome_k=4, n_sweeps=S, seed=3004,
                                     moves_per_sweep=M, mask=mask, length_format=fmt)
        assert rep["moves"] == S * M
        assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
        assert rep["max_err_dS"] <= 1e-5, rep
        imgs.append(img)
    assert np.array_equal(imgs[0], imgs[1])
    assert np.all(imgs[0][mask == 0] == 0.0)
    api.pila_free(p)


@pytest.mark.parametrize("U", [128, 129])
def test_window_angle_limit(api, U):
    """128 angles fill every record slot of a windowed warp's lanes (4 per
    lane); at 129 the rules fall back to the pipelined kernel.  Both follow
    the oracle move by move."""
    n = 32
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    pm = oracle.drt(synth.phantom(n, 5, 1005), U, B).astype(np.float32)
    img0 = synth.initial_image(n, 0.5, mask)
    S, M = 2, int(mask.sum())
    p = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    st, tr, img = _run_traced(api, p, pm, img0, S, M, bome_k=4, t0=-1.0, tn=-1.0, seed=3005, group_warps=1)
    assert st["status"] == 0 and st["proposed"] == S * M
    _, rep = oracle.sat_lockstep(pm, img0, tr, t0=st["t0"], tn=st["tn"], bome_k=4, n_sweeps=S, seed=3005,
                                 mask=mask)
    assert rep["moves"] == S * M
    assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
    assert rep["max_err_dS"] <= 1e-5, rep
    api.pila_free(p)


@pytest.mark.parametrize("W,U,prec", [(2, 180, 0), (4, 180, 1), (4, 360, 1), (2, 90, 1), (2, 180, 2), (4, 360, 2)])
def test_window_groups_lockstep(api, W, U, prec):
    """The windowed move on groups of 2 or 4 warps per chain (residual in
    global memory; the warps exchange window sums): move by move against the
    oracle (FP16 tables over binary16 lengths, one-byte tables over the
    lengths q/180 of Sec. II-B at 180 and 360 angles), with 2 and 4 record
    slots per lane, and a chain in a batch equal to its run alone."""
    n = 48
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    pm = synth.gaussian_noise(oracle.drt(synth.phantom(n, 8, 1006), U, B), 0.01, 2006).astype(np.float32)
    img0 = synth.initial_image(n, 0.5, mask)
    S, M = 2, 1500
    fmt = {api.PILA_F32: oracle.LEN_EXACT, api.PILA_F16: oracle.LEN_BINARY16, api.PILA_U8: oracle.LEN_BYTE180}[prec]
    p = api.pila_build(n, U, B, prec, mask=mask)
    kw = dict(bome_k=8, t0=-1.0, tn=-1.0, seed=3006, moves_per_sweep=M, group_warps=W,
              flags=api.SAT_FLAG_WINDOW_GROUPS)
    st, tr, img = _run_traced(api, p, pm, img0, S, M, **kw)
    assert st["status"] == 0 and st["proposed"] == S * M
    _, rep = oracle.sat_lockstep(pm, img0, tr, t0=st["t0"], tn=st["tn"], bome_k=8, n_sweeps=S, seed=3006,
                                 moves_per_sweep=M, mask=mask, length_format=fmt)
    assert rep["moves"] == S * M
    assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
    assert rep["max_err_dS"] <= 1e-5, rep
    # batch of 5 chains: chain 3 equals its run alone
    sinos = np.stack([pm] * 5)
    imgs = dev(np.stack([img0] * 5))
    kwb = {k: v for k, v in kw.items() if k != "seed"}
    stb = api.sat_run(p, dev(sinos), imgs, n_sweeps=S, seed=500, **kwb)
    one = dev(img0[None])
    st1 = api.sat_run(p, dev(pm[None]), one, n_sweeps=S, seed=503, **kwb)
    assert np.array_equal(imgs.cpu().numpy()[3], one.cpu().numpy()[0])
    assert stb[3]["accepted"] == st1[0]["accepted"]
    api.pila_free(p)


@pytest.mark.parametrize("plan,n,U,prec", [(9, 128, 120, 1), (10, 128, 120, 1), (9, 64, 90, 0), (10, 96, 180, 1)])
def test_window_smem_groups_lockstep(api, plan, n, U, prec):
    """The windowed move on groups of 2 or 4 warps per chain with the residual
    band in shared memory (each warp owning the rows of its angles): move by
    move against the oracle, the same image as the one-warp windowed kernel
    for the same chain, and batched chains equal to their runs alone."""
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    pm = synth.gaussian_noise(oracle.drt(synth.phantom(n, 8, 1010 + n), U, B), 0.01, 2010).astype(np.float32)
    img0 = synth.initial_image(n, 0.5, mask)
    S, M = 2, 1500
    fmt = oracle.LEN_EXACT if prec == api.PILA_F32 else oracle.LEN_BINARY16
    p = api.pila_build(n, U, B, prec, mask=mask)
    kw = dict(bome_k=4, t0=-1.0, tn=-1.0, seed=3010, moves_per_sweep=M)
    st, tr, img = _run_traced(api, p, pm, img0, S, M, plan=plan, **kw)
    assert st["status"] == 0 and st["proposed"] == S * M and st["plan"] == plan
    _, rep = oracle.sat_lockstep(pm, img0, tr, t0=st["t0"], tn=st["tn"], bome_k=4, n_sweeps=S, seed=3010,
                                 moves_per_sweep=M, mask=mask, length_format=fmt)
    assert rep["moves"] == S * M
    assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
    assert rep["max_err_dS"] <= 1e-5, rep
    # batch of 7 chains: chain 5 equals its run alone
    kwb = {k: v for k, v in kw.items() if k != "seed"}
    imgs = dev(np.stack([img0] * 7))
    stb = api.sat_run(p, dev(np.stack([pm] * 7)), imgs, n_sweeps=S, seed=700, plan=plan, **kwb)
    one = dev(img0[None])
    st1 = api.sat_run(p, dev(pm[None]), one, n_sweeps=S, seed=705, plan=plan, **kwb)
    assert np.array_equal(imgs.cpu().numpy()[5], one.cpu().numpy()[0])
    assert stb[5]["accepted"] == st1[0]["accepted"]
    api.pila_free(p)


def test_hybrid_batch_matches_single_chains(api):
    """More chains than shared-memory slots: the batch runs on shared-memory
    and global-memory warps side by side, with chains moving between them
    stage by stage; every chain must still equal its run alone."""
    n, U = 128, 120
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    C = 600
    base = [oracle.drt(synth.phantom(n, 8, 90 + i), U, B).astype(np.float32) for i in range(5)]
    sinos = np.stack([base[i % 5] for i in range(C)])
    img0 = np.stack([synth.initial_image(n, 0.5, mask)] * C).astype(np.float32)
    kw = dict(bome_k=4, n_sweeps=3, moves_per_sweep=400, t0=2e-3, tn=2e-5)
    imgs = dev(img0)
    st = api.sat_run(p, dev(sinos), imgs, seed=100, flags=api.SAT_FLAG_HYBRID, **kw)
    out = imgs.cpu().numpy()
    for c in (0, 7, 200, C - 1):
        one = dev(img0[c:c + 1])
        s1 = api.sat_run(p, dev(sinos[c:c + 1]), one, seed=100 + c, **kw)
        assert np.array_equal(one.cpu().numpy()[0], out[c]), c
        assert s1[0]["accepted"] == st[c]["accepted"]
    api.pila_free(p)


def test_graph_replay_matches_direct_launches(api):
    """A repeated call with the same table, buffers and parameters replays a
    cached CUDA graph; it must give what direct launches give."""
    n, U = 48, 40
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    sinos = np.stack([oracle.drt(synth.phantom(n, 6, 120 + i), U, B) for i in range(6)]).astype(np.float32)
    img0 = np.stack([synth.initial_image(n, 0.5, mask)] * 6).astype(np.float32)
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    kw = dict(bome_k=4, n_sweeps=5, t0=-1.0, tn=-1.0, resync_every=2, seed=11)
    sino_d = dev(sinos)
    ref = dev(img0)
    st_ref = api.sat_run(p, sino_d, ref, flags=api.SAT_FLAG_NO_GRAPH, **kw)
    work = dev(img0)
    init = dev(img0)
    for _ in range(3):  # capture, then two replays on the same buffers
        work.copy_(init)
        st = api.sat_run(p, sino_d, work, **kw)
        assert torch.equal(work, ref)
        assert [s["accepted"] for s in st] == [s["accepted"] for s in st_ref]
        assert [s["final_cost"] for s in st] == [s["final_cost"] for s in st_ref]
        assert all(s["sweep_ms"] > 0.0 for s in st)
    api.pila_free(p)


def test_sat_run_asynchronous_without_stats(api):
    """With no stats and device buffers sat_run returns once its graph is
    enqueued; the images, once the stream has run, equal a synchronous call's;
    two such calls of one problem on two streams share the cached graph and
    workspace, the second waiting for the first."""
    n, U = 48, 40
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    C = 4
    sinos = dev(np.stack([oracle.drt(synth.phantom(n, 6, 60 + i) * mask, U, B) for i in range(C)]).astype(np.float32))
    img0 = np.stack([synth.initial_image(n, 0.5, mask)] * C).astype(np.float32)
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    kw = dict(bome_k=4, n_sweeps=3, t0=-1.0, tn=-1.0, seed=8)
    ref = dev(img0)
    api.sat_run(p, sinos, ref, **kw)
    a, b = dev(img0), dev(img0)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    assert api.sat_run(p, sinos, a, stream=s1, sync=False, **kw) is None
    s1.synchronize()
    assert np.array_equal(a.cpu().numpy(), ref.cpu().numpy())
    # the same call twice (same buffers: the same cached graph and workspace),
    # on two streams: the second must start from the first's result
    api.sat_run(p, sinos, ref, **kw)  # ref = two synchronous calls in a row
    a.copy_(dev(img0))
    torch.cuda.synchronize()
    api.sat_run(p, sinos, a, stream=s1, sync=False, **kw)
    api.sat_run(p, sinos, a, stream=s2, sync=False, **kw)
    torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy(), ref.cpu().numpy())
    del b
    api.pila_free(p)


def test_sat_run_ptrs_matches_the_stacked_batch(api):
    """sat_run_ptrs over one buffer per chain (separate device tensors and a
    host array, mixed) gives sat_run's results on the stacked batch, bit for
    bit, and without stats it is asynchronous for device buffers."""
    n, U = 48, 40
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    C = 3
    sinos = np.stack([oracle.drt(synth.phantom(n, 6, 80 + i) * mask, U, B) for i in range(C)]).astype(np.float32)
    img0 = np.stack([synth.initial_image(n, 0.5, mask)] * C).astype(np.float32)
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    kw = dict(bome_k=4, n_sweeps=4, t0=-1.0, tn=-1.0, resync_every=2, seed=31)
    ref = dev(img0)
    s_ref = api.sat_run(p, dev(sinos), ref, **kw)
    ref = ref.cpu().numpy()
    imgs = [dev(img0[0]), img0[1].copy(), dev(img0[2])]
    ins = [dev(sinos[0]), sinos[1].copy(), dev(sinos[2])]
    st = api.sat_run_ptrs(p, ins, imgs, **kw)
    for c in range(C):
        got = imgs[c].cpu().numpy() if hasattr(imgs[c], "cpu") else imgs[c]
        assert np.array_equal(got, ref[c]), c
        assert st[c]["accepted"] == s_ref[c]["accepted"] and st[c]["final_cost"] == s_ref[c]["final_cost"]
        assert st[c]["plan"] == s_ref[c]["plan"]
    # device buffers, no stats: enqueued on the stream, the same images
    dimgs = [dev(img0[c]) for c in range(C)]
    dins = [dev(sinos[c]) for c in range(C)]
    s1 = torch.cuda.Stream()
    torch.cuda.synchronize()
    assert api.sat_run_ptrs(p, dins, dimgs, stream=s1, sync=False, **kw) is None
    s1.synchronize()
    for c in range(C):
        assert np.array_equal(dimgs[c].cpu().numpy(), ref[c]), c
    with pytest.raises(api.SatpilaError):
        api.sat_run_ptrs(p, dins, dimgs[:2] + [None], **kw)
    api.pila_free(p)


def test_autotune_picks_a_layout_and_is_repeatable(api):
    """SAT_FLAG_AUTOTUNE times the launch layouts once per shape: the chosen
    layout is reported, a second call reuses it with identical results, and
    the results agree with the rule-chosen layout to the stated tolerance."""
    n, U = 64, 60
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    C = 40
    sinos = np.stack([oracle.drt(synth.phantom(n, 8, 140 + i % 4), U, B) for i in range(C)]).astype(np.float32)
    img0 = np.stack([synth.initial_image(n, 0.5, mask)] * C).astype(np.float32)
    ph = np.stack([synth.phantom(n, 8, 140 + i % 4) for i in range(C)])
    p = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    kw = dict(bome_k=4, n_sweeps=12, t0=-1.0, tn=-1.0, resync_every=4, seed=21)
    outs = []
    for _ in range(2):
        imgs = dev(img0)
        st = api.sat_run(p, dev(sinos), imgs, flags=api.SAT_FLAG_AUTOTUNE, **kw)
        assert all(s["status"] == 0 for s in st)
        assert 1 <= st[0]["plan"] <= 10
        outs.append((imgs.cpu().numpy(), [s["plan"] for s in st], [s["accepted"] for s in st]))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1:] == outs[1][1:]
    # the pick passed back as sat_params.plan reproduces the autotuned run exactly
    pinned = dev(img0)
    st_p = api.sat_run(p, dev(sinos), pinned, plan=outs[0][1][0], **kw)
    assert st_p[0]["plan"] == outs[0][1][0]
    assert np.array_equal(pinned.cpu().numpy(), outs[0][0])
    rule = dev(img0)
    st_r = api.sat_run(p, dev(sinos), rule, **kw)
    assert 1 <= st_r[0]["plan"] <= 10  # the layout the size rules chose
    r_tuned = np.mean([synth.rmse(outs[0][0][c], ph[c]) for c in range(C)])
    r_rule = np.mean([synth.rmse(rule.cpu().numpy()[c], ph[c]) for c in range(C)])
    assert abs(r_tuned - r_rule) <= 0.02 * r_rule
    api.pila_free(p)


@pytest.mark.parametrize("K,prec", [(1, 0), (4, 0), (16, 0), (8, 1)])
def test_bome_independent_lockstep(api, K, prec):
    """BoME as Sec. III-B words it (each estimate its own random pixel):
    every move against the oracle's independent-pixel reading, with the
    disk reconstruction space and Gaussian noise."""
    n, U = 48, 40
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    ph = synth.phantom(n, 8, 1005) * mask
    pm = synth.gaussian_noise(oracle.drt(ph, U, B), 0.01, 2005)
    img0 = synth.initial_image(n, 0.5, mask)
    p = api.pila_build(n, U, B, prec, mask=mask)
    S, M = 3, 1500
    st, tr, img = _run_traced(api, p, pm, img0, S, M, bome_k=K, t0=2e-3, tn=2e-5, seed=3005, moves_per_sweep=M,
                              flags=api.SAT_FLAG_BOME_INDEPENDENT)
    assert st["status"] == 0 and st["proposed"] == S * M
    if K > 1:
        assert np.mean(tr["cstar"] > 0) > 0.3  # estimates other than the first are chosen
    if prec == 0:
        _, rep = oracle.sat_lockstep(pm, img0, tr, t0=2e-3, tn=2e-5, bome_k=K, n_sweeps=S, seed=3005,
                                     moves_per_sweep=M, mask=mask, bome_mode=oracle.BOME_INDEPENDENT)
        assert rep["moves"] == S * M
        assert rep["pixel_mismatch"] == -1 and rep["hard_mismatch"] == -1, rep
        assert rep["max_err_dS"] <= 1e-5, rep
        assert rep["near_ties"] <= 1e-3 * S * M, rep
    assert st["max_resync_drift"] <= 1e-4 * np.max(np.abs(pm))
    api.pila_free(p)


def test_bome_independent_batched_equals_single(api):
    n, U = 40, 30
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    sinos = np.stack([oracle.drt(synth.phantom(n, 6, 160 + i), U, B) for i in range(5)]).astype(np.float32)
    img0 = np.stack([synth.initial_image(n, 0.5, mask)] * 5).astype(np.float32)
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    kw = dict(bome_k=8, n_sweeps=4, t0=-1.0, tn=-1.0, resync_every=2, flags=api.SAT_FLAG_BOME_INDEPENDENT)
    imgs = dev(img0)
    st = api.sat_run(p, dev(sinos), imgs, seed=31, **kw)
    out = imgs.cpu().numpy()
    for c in (0, 4):
        one = dev(img0[c:c + 1])
        s1 = api.sat_run(p, dev(sinos[c:c + 1]), one, seed=31 + c, **kw)
        assert np.array_equal(one.cpu().numpy()[0], out[c]) and s1[0]["accepted"] == st[c]["accepted"]
    api.pila_free(p)


@pytest.mark.parametrize("n,U", [(24, 18), (64, 90)])
def test_drt_bilinear_vs_oracle(api, n, U):
    """The conventional forward model (bilinear interpolation, unit steps) in
    FP32 against the oracle's FP64."""
    B = synth.bins_for(n)
    rng = np.random.default_rng(n)
    imgs = rng.random((3, n, n))
    got = api.drt_bilinear(dev(imgs), U, B).cpu().numpy()
    for i in range(3):
        ref = oracle.drt_bilinear(imgs[i], U, B)
        assert np.max(np.abs(got[i] - ref)) <= 2e-6 * B * max(1.0, np.max(np.abs(ref)))


def test_sat_drt_follows_oracle(api):
    """SAT with a full bilinear DRT per estimate: the GPU chain and the oracle
    draw the same moves; their decisions agree (FP32 vs FP64 costs) until a
    near-tie, and the costs agree to FP32 accuracy."""
    n, U, K, S, M = 16, 12, 2, 2, 60
    B = synth.bins_for(n)
    ph = synth.phantom(n, 4, 33)
    pm = oracle.drt_bilinear(ph, U, B)
    img0 = np.full((n, n), 0.5)
    kw = dict(t0=2e-3, tn=2e-5, bome_k=K, n_sweeps=S, moves_per_sweep=M, seed=44)
    _, st_o, tr_o = oracle.sat_drt_run(pm, img0, trace=True, **kw)
    trace = torch.zeros(S * M * 32, dtype=torch.uint8, device="cuda")
    img = dev(img0).reshape(1, n, n)
    st = api.sat_drt_run(dev(pm).reshape(1, U, B), img, trace=trace, trace_chain=0, **kw)[0]
    tr = np.frombuffer(trace.cpu().numpy().tobytes(), dtype=api.TRACE_DTYPE)
    assert st["proposed"] == S * M
    cref = st_o["initial_cost"]
    first_diff = S * M
    for i in range(S * M):
        assert tr["pixel"][i] == tr_o["pixel"][i]
        if tr["cstar"][i] != tr_o["cstar"][i] or tr["accepted"][i] != tr_o["accepted"][i]:
            first_diff = i
            break
        assert abs(float(tr["dC"][i]) - tr_o["dC"][i]) <= 1e-4 * cref, i
        assert abs(float(tr["fnew"][i]) - tr_o["fnew"][i]) <= 1e-6, i
    if first_diff < S * M:  # only a near-tie may separate them
        i = first_diff
        T = oracle.schedule_temp(oracle.SCHED_LINEAR, 2e-3, 2e-5, i // M, S)
        thr = -T * np.log(tr_o["u_acc"][i])
        assert abs(tr_o["dC"][i] - thr) <= 1e-4 * cref or abs(tr_o["dC"][i]) <= 1e-4 * cref
    assert first_diff >= 0.5 * S * M


def test_fbp_and_prior_vs_oracle(api):
    """FBP (Ram-Lak) in FP32 against the oracle's FP64, and the prior (beta,
    threshold mask, clipped start image) against its definition applied to
    the GPU's own FBP image."""
    from oracle import fbp as F

    n, U = 64, 90
    B = synth.bins_for(n)
    phs = [synth.phantom(n, 8, 500 + i) for i in range(3)]
    sinos = np.stack([oracle.drt(ph, U, B) for ph in phs])
    rec = api.fbp(dev(sinos), n)
    got = rec.cpu().numpy()
    for i in range(3):
        ref = F.fbp(sinos[i], n)
        assert np.max(np.abs(got[i] - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))
    init, mask, beta = api.fbp_prior(rec, 0.1)
    init, mask, beta = init.cpu().numpy(), mask.cpu().numpy(), beta.cpu().numpy()
    for i in range(3):
        mx = max(float(got[i].max()), 0.0)
        assert beta[i] == np.float32(mx)
        m = got[i] > np.float32(0.1) * np.float32(mx)
        assert np.array_equal(mask[i].astype(bool), m)
        assert np.array_equal(init[i], np.where(m, np.clip(got[i], 0.0, mx), 0.0).astype(np.float32))
