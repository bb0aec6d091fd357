"""Pins for the CPU reference oracle: each checks the oracle against something
other than itself (published vectors, closed forms, invariants, brute force,
a stationary distribution), chosen so that a dropped term, a wrong sign, a
swapped index or a transposed operand fails at least one of them."""
import math
import os

import numpy as np
import pytest

from paper_1411_4622_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _snap(v):
    return 0.0 if abs(v) < 1e-12 else v


def chord_closed_form(n, theta, s_k, i, j):
    """Chord length of the line x cos + y sin = s_k in pixel (i, j): the unit
    square's projection is a trapezoid of half-width (|c|+|s|)/2, plateau
    half-width ||c|-|s||/2 and height 1/max(|c|,|s|); membership is
    half-open, [s_p - w/2, s_p + w/2)."""
    c, s = _snap(math.cos(theta)), _snap(math.sin(theta))
    a, b = abs(c), abs(s)
    x, y = j - 0.5 * (n - 1), 0.5 * (n - 1) - i
    d = s_k - (x * c + y * s)
    w = a + b
    if d < -0.5 * w or d >= 0.5 * w:
        return 0.0
    t = abs(d)
    if t <= 0.5 * abs(a - b):
        return 1.0 / max(a, b)
    return (0.5 * w - t) / (a * b)


def clip_length(n, theta, s):
    """Liang-Barsky: length of the line x cos + y sin = s inside [-n/2, n/2]^2.
    An axis-aligned line on the square's edge counts only on the +s side."""
    c, sn = _snap(math.cos(theta)), _snap(math.sin(theta))
    h = 0.5 * n
    qx, qy, dx, dy = s * c, s * sn, -sn, c
    lo, hi = -math.inf, math.inf
    for q, d in ((qx, dx), (qy, dy)):
        if d == 0.0:
            # Half-open: the line's +s side must overlap the square.
            along = c if (dx == 0.0 and q is qx) else sn
            inside = (-h <= q < h) if along > 0 else (-h < q <= h)
            if not inside:
                return 0.0
        else:
            t1, t2 = (-h - q) / d, (h - q) / d
            lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
    return max(0.0, hi - lo)


def test_philox_known_answers(orc):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if ln[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


@pytest.mark.parametrize("n,U", [(4, 4), (5, 6), (8, 12), (7, 9)])
def test_pila_matches_trapezoid_closed_form(orc, n, U):
    B = synth.bins_for(n)
    bins, lens = orc.pila(n, U, B)
    for p in range(n * n):
        i, j = divmod(p, n)
        for u in range(U):
            theta = math.pi * u / U
            want = {}
            for k in range(B):
                l = chord_closed_form(n, theta, k - 0.5 * (B - 1), i, j)
                if l > 1e-9:
                    want[k] = l
            got = {int(bins[p, u, s]): lens[p, u, s] for s in range(2) if lens[p, u, s] > 1e-9}
            assert set(got) == set(want), (p, u, got, want)
            for k in want:
                assert abs(got[k] - want[k]) <= 1e-12 * max(1.0, want[k])
            # two slots are sorted, the second one is the next bin
            if lens[p, u, 1] > 0:
                assert bins[p, u, 1] == bins[p, u, 0] + 1


@pytest.mark.parametrize("n", [4, 5, 64])
def test_pila_axis_aligned_and_diagonal(orc, n):
    U = 4  # 0, 45, 90, 135 degrees
    B = synth.bins_for(n)
    bins, lens = orc.pila(n, U, B)
    for p in range(n * n):
        i, j = divmod(p, n)
        # 0 degrees: one entry of length 1 at bin j + (B-1-n)/2 (exact for even n;
        # for odd n the ray passes through the centre column).
        k0 = j + (B - 1 - n) / 2
        if float(k0).is_integer():
            assert bins[p, 0, 0] == int(k0) and lens[p, 0, 0] == 1.0 and lens[p, 0, 1] == 0.0
        else:
            assert lens[p, 0, 0] == 1.0 and bins[p, 0, 0] == math.ceil(k0) and lens[p, 0, 1] == 0.0
        # 90 degrees: bin (B-1+n)/2 - 1 - i.
        k90 = (B - 1 + n) / 2 - 1 - i
        assert bins[p, 2, 0] == math.ceil(k90) and lens[p, 2, 0] == 1.0 and lens[p, 2, 1] == 0.0
        # 45 degrees: l = sqrt(2) - 2 t, t the distance to the pixel centre.
        x, y = j - 0.5 * (n - 1), 0.5 * (n - 1) - i
        sp = (x + y) / math.sqrt(2.0)
        for s in range(2):
            if lens[p, 1, s] > 1e-9:
                t = abs(bins[p, 1, s] - 0.5 * (B - 1) - sp)
                assert abs(lens[p, 1, s] - (math.sqrt(2.0) - 2.0 * t)) < 1e-12


@pytest.mark.parametrize("n,U", [(6, 7), (9, 10), (32, 13)])
def test_pila_ray_sums_equal_clipped_chords(orc, n, U):
    """The pixels tile the square, so every ray's lengths add up to its
    chord through the whole image."""
    B = synth.bins_for(n) + 2  # also rays that miss the square
    bins, lens = orc.pila(n, U, B)
    sums = np.zeros((U, B))
    for s in range(2):
        ok = lens[:, :, s] > 0
        pp, uu = np.nonzero(ok)
        np.add.at(sums, (uu, bins[pp, uu, s]), lens[pp, uu, s])
    for u in range(U):
        for k in range(B):
            want = clip_length(n, math.pi * u / U, k - 0.5 * (B - 1))
            assert abs(sums[u, k] - want) < 1e-9, (u, k, sums[u, k], want)


def test_drt_of_constant_and_unit_images(orc):
    n, U = 8, 11
    B = synth.bins_for(n)
    ones = orc.drt(np.ones((n, n)), U, B)
    for u in range(U):
        for k in range(B):
            assert abs(ones[u, k] - clip_length(n, math.pi * u / U, k - 0.5 * (B - 1))) < 1e-9
    bins, lens = orc.pila(n, U, B)
    for p in (0, 9, 27, 63):
        e = np.zeros((n, n))
        e.flat[p] = 1.0
        s = orc.drt(e, U, B)
        want = np.zeros((U, B))
        for u in range(U):
            for slot in range(2):
                if lens[p, u, slot] > 0:
                    want[u, bins[p, u, slot]] += lens[p, u, slot]
        assert np.allclose(s, want, atol=1e-12)
    rng = np.random.default_rng(5)
    a, b = rng.random((n, n)), rng.random((n, n))
    assert np.allclose(orc.drt(2 * a - 3 * b, U, B), 2 * orc.drt(a, U, B) - 3 * orc.drt(b, U, B), atol=1e-11)


def test_drt_equals_closed_form_chord_sum(orc):
    n, U = 7, 5
    B = synth.bins_for(n)
    rng = np.random.default_rng(3)
    img = rng.random((n, n))
    s = orc.drt(img, U, B)
    for u in range(U):
        for k in range(B):
            want = sum(img[i, j] * chord_closed_form(n, math.pi * u / U, k - 0.5 * (B - 1), i, j)
                       for i in range(n) for j in range(n))
            assert abs(s[u, k] - want) < 1e-12


def test_cost_eq4(orc):
    rng = np.random.default_rng(1)
    a, b = rng.random((5, 7)), rng.random((5, 7))
    assert orc.cost(a, a) == 0.0
    assert abs(orc.cost(a, b) - np.sqrt(np.mean((a - b) ** 2))) < 1e-15
    assert abs(orc.cost(a, b) - np.linalg.norm(a - b) / np.sqrt(35)) < 1e-14


def _small_problem(n=8, U=9, seed=11, noise=0.0):
    B = synth.bins_for(n)
    ph = synth.phantom(n, 4, seed)
    return ph, B, U


def _draw(orc, seed, c0, c1, stream, nblk):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    w = []
    for b in range(nblk):
        w += orc.philox4x32_10([c0, c1, b, stream], key).tolist()
    return w


def _u01(x):
    return ((x >> 9) * 2 + 1) * 2.0**-24


def test_eq7_and_bome_against_brute_force(orc):
    """Every move's dC (Eq. (7)) equals C' - C recomputed from scratch with
    the DRT and Eq. (4), and the chosen estimate is the exhaustive argmin."""
    n, U, K, seed, beta = 8, 9, 5, 77, 1.0
    ph, B, _ = _small_problem(n, U)
    pm = orc.drt(ph, U, B)
    img0 = np.full((n, n), 0.5)
    M = 40
    img, st, tr = orc.sat_run(pm, img0, bome_k=K, n_sweeps=2, moves_per_sweep=M, t0=1e-3, tn=1e-4,
                              seed=seed, trace=True)
    cur = img0.copy()
    nblk = (K + 2 + 3) // 4
    for idx, rec in enumerate(tr):
        s, m = divmod(idx, M)
        w = _draw(orc, seed, s, m, 1, nblk)
        p = (w[0] * n * n) >> 32
        assert rec["pixel"] == p
        c_now = orc.cost(orc.drt(cur, U, B), pm)
        f = cur.flat[p]
        lo, hi = max(0.0, f - beta), min(beta, f + beta)
        costs = []
        for c in range(K):
            trial = cur.copy()
            trial.flat[p] = lo + _u01(w[2 + c]) * (hi - lo)
            costs.append(orc.cost(orc.drt(trial, U, B), pm))
        best = int(np.argmin(costs))
        assert rec["cstar"] == best
        assert abs(rec["dC"] - (costs[best] - c_now)) < 1e-12
        assert rec["u_acc"] == _u01(w[1])
        if rec["accepted"]:
            cur.flat[p] = lo + _u01(w[2 + best]) * (hi - lo)
    assert np.allclose(cur, img, atol=1e-15)


def test_bome_independent_pixels_against_brute_force(orc):
    """Sec. III-B as written: each estimate is a random pixel with a random
    value.  Every move's chosen estimate is the exhaustive argmin of C' over
    the N_e (pixel, value) pairs, each C' recomputed from scratch with the DRT
    and Eq. (4); draw 2 + c is estimate c's value and draw 2 + N_e + c - 1 its
    pixel (estimate 0 takes draw 0)."""
    n, U, K, seed, beta = 8, 9, 4, 78, 1.0
    ph, B, _ = _small_problem(n, U)
    pm = orc.drt(ph, U, B)
    img0 = np.full((n, n), 0.5)
    M = 40
    img, st, tr = orc.sat_run(pm, img0, bome_k=K, n_sweeps=2, moves_per_sweep=M, t0=1e-3, tn=1e-4,
                              seed=seed, trace=True, bome_mode=orc.BOME_INDEPENDENT)
    cur = img0.copy()
    nblk = (2 * K + 1 + 3) // 4
    distinct = 0
    for idx, rec in enumerate(tr):
        s, m = divmod(idx, M)
        w = _draw(orc, seed, s, m, 1, nblk)
        pix = [(w[0] * n * n) >> 32] + [(w[2 + K + c - 1] * n * n) >> 32 for c in range(1, K)]
        distinct += len(set(pix)) > 1
        c_now = orc.cost(orc.drt(cur, U, B), pm)
        costs, vals = [], []
        for c in range(K):
            f = cur.flat[pix[c]]
            lo, hi = max(0.0, f - beta), min(beta, f + beta)
            vals.append(lo + _u01(w[2 + c]) * (hi - lo))
            trial = cur.copy()
            trial.flat[pix[c]] = vals[c]
            costs.append(orc.cost(orc.drt(trial, U, B), pm))
        best = int(np.argmin(costs))
        assert rec["cstar"] == best and rec["pixel"] == pix[best]
        assert abs(rec["dC"] - (costs[best] - c_now)) < 1e-12
        if rec["accepted"]:
            cur.flat[pix[best]] = vals[best]
    assert distinct > 0.9 * len(tr)
    assert np.allclose(cur, img, atol=1e-15)


def test_bome_modes_agree_for_one_estimate(orc):
    """With N_e = 1 both BoME readings draw the same single (pixel, value)
    proposal, so the chains are identical."""
    n, U = 12, 10
    ph, B, _ = _small_problem(n, U)
    pm = synth.gaussian_noise(orc.drt(ph, U, B), 0.01, 5)
    a, sa, _ = orc.sat_run(pm, np.full((n, n), 0.5), bome_k=1, n_sweeps=3, seed=12)
    b, sb, _ = orc.sat_run(pm, np.full((n, n), 0.5), bome_k=1, n_sweeps=3, seed=12,
                           bome_mode=orc.BOME_INDEPENDENT)
    assert np.array_equal(a, b) and sa["accepted"] == sb["accepted"]


def test_incremental_state_matches_fresh_drt(orc):
    n, U = 16, 20
    ph, B, _ = _small_problem(n, U)
    pm = synth.gaussian_noise(orc.drt(ph, U, B), 0.01, 4)
    img, st, _ = orc.sat_run(pm, np.full((n, n), 0.5), bome_k=4, n_sweeps=5, seed=9)
    assert st["proposed"] == 5 * n * n and 0 < st["accepted"] < st["proposed"]
    assert abs(st["final_cost"] - st["final_cost_fresh"]) <= 1e-10 * st["final_cost_fresh"]
    assert abs(st["final_cost_fresh"] - orc.cost(orc.drt(img, U, B), pm)) < 1e-13
    assert img.min() >= 0.0 and img.max() <= 1.0


def test_stored_length_formats(orc):
    """Sec. II-B stores the PILA's lengths in reduced precision.  binary16
    rounding equals numpy's float64 -> float16 cast (ties to even, the
    subnormal range included); one-byte lengths are the nearest multiple of
    1/180.  A run over a rounded table keeps its projections as sums over
    that table: its initial and final Eq. (4) costs equal numpy's sums over
    the numpy-rounded lengths."""
    n, U = 16, 20
    ph, B, _ = _small_problem(n, U)
    bins, lens = orc.pila(n, U, B)
    special = [0.0, 2.0 ** -25, 2.0 ** -24, 3 * 2.0 ** -25, 5 * 2.0 ** -25, 2.0 ** -14 - 2.0 ** -25,
               2.0 ** -14, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, math.sqrt(2.0), 1e-7, 0.123456789]
    vals = np.concatenate([lens.ravel()[::7], np.array(special),
                           np.random.default_rng(5).uniform(0.0, 1.5, 2000)])
    got16 = np.array([orc.round_length(orc.LEN_BINARY16, v) for v in vals])
    assert np.array_equal(got16, vals.astype(np.float16).astype(np.float64))
    got8 = np.array([orc.round_length(orc.LEN_BYTE180, v) for v in vals])
    q = got8 * 180.0
    assert np.all(np.abs(q - np.round(q)) < 1e-9) and np.all(np.abs(got8 - vals) <= 0.5 / 180 + 1e-12)
    assert orc.round_length(orc.LEN_EXACT, 0.3) == 0.3
    pm = synth.gaussian_noise(orc.drt(ph, U, B), 0.01, 4)
    img0 = np.full((n, n), 0.5)
    for fmt, cast in ((orc.LEN_BINARY16, lambda a: a.astype(np.float16).astype(np.float64)),
                      (orc.LEN_BYTE180, lambda a: np.round(a * 180.0) / 180.0)):
        rl = cast(lens)

        def project(x):
            out = np.zeros((U, B))
            ok = rl > 0
            pix = np.broadcast_to(np.arange(n * n)[:, None, None], rl.shape)
            ang = np.broadcast_to(np.arange(U)[None, :, None], rl.shape)
            np.add.at(out, (ang[ok], bins[ok]), x.ravel()[pix[ok]] * rl[ok])
            return out

        img, st, _ = orc.sat_run(pm, img0, bome_k=4, n_sweeps=3, seed=9, length_format=fmt)
        c0 = math.sqrt(np.mean((project(img0) - pm) ** 2))
        c1 = math.sqrt(np.mean((project(img) - pm) ** 2))
        assert abs(st["initial_cost"] - c0) <= 1e-12 * c0
        assert abs(st["final_cost_fresh"] - c1) <= 1e-12 * c1
        assert abs(st["final_cost"] - c1) <= 1e-10 * c1
        assert 0 < st["accepted"] < st["proposed"]


def test_metropolis_stationary_distribution(orc):
    """One pixel, fixed T, one estimate: proposals are uniform on [0, beta]
    and independent of the state, so Step 4 makes the chain sample the
    density proportional to exp(-C(f)/T) on [0, beta]."""
    n, U, B = 1, 6, 1
    fstar, beta, T = 0.3, 1.0, 0.02
    pm = orc.drt(np.full((1, 1), fstar), U, B)
    M = 60000
    img, st, tr = orc.sat_run(pm, np.full((1, 1), 0.9), bome_k=1, n_sweeps=1, moves_per_sweep=M,
                              t0=T, tn=T, seed=123, trace=True, beta=beta)
    samples = tr["fnew"][1000::3]
    lam = math.sqrt(np.mean(pm[:, 0] ** 2)) / fstar  # C(f) = lam * |f - f*|
    grid = np.linspace(0.0, beta, 20001)
    dens = np.exp(-lam * np.abs(grid - fstar) / T)
    cdf = np.cumsum(dens)
    cdf /= cdf[-1]
    emp = np.searchsorted(np.sort(samples), grid, side="right") / len(samples)
    assert np.max(np.abs(emp - cdf)) < 0.03
    mean_theory = float(np.sum(grid * dens) / np.sum(dens))
    assert abs(samples.mean() - mean_theory) < 0.01


def test_schedules_closed_forms(orc):
    t0, tn, S = 2.0, 0.002, 50
    lin = [orc.schedule_temp(orc.SCHED_LINEAR, t0, tn, s, S) for s in range(S + 1)]
    geo = [orc.schedule_temp(orc.SCHED_GEOMETRIC, t0, tn, s, S) for s in range(S + 1)]
    cub = [orc.schedule_temp(orc.SCHED_CUBIC, t0, tn, s, S) for s in range(S + 1)]
    for seq in (lin, geo, cub):
        assert seq[0] == t0 and abs(seq[S] - tn) < 1e-15
        assert all(a > b for a, b in zip(seq, seq[1:]))
    assert np.allclose(np.diff(lin), (tn - t0) / S, rtol=1e-12)
    assert np.allclose(np.array(geo[1:]) / np.array(geo[:-1]), (tn / t0) ** (1 / S), rtol=1e-12)
    ss = np.arange(S + 1)
    assert np.allclose(t0 - np.array(cub), (t0 - tn) * (ss / S) ** 3, rtol=1e-12, atol=1e-15)
    # cubic stays hotter than linear, geometric colder
    assert all(c > l > g for c, l, g in list(zip(cub, lin, geo))[1:-1])


def test_t0_rule_brute_force(orc):
    """Eq. (8): T0 makes exp(-mean uphill dC / T0) = 0.9, averaging the first
    Q proposals from the initial image that raise the cost."""
    n, U, beta, seed, Q = 8, 7, 1.0, 31, 25
    ph, B, _ = _small_problem(n, U)
    pm = orc.drt(ph, U, B)
    img0 = np.full((n, n), 0.5)
    t0, found = orc.sat_t0(pm, img0, seed=seed, t0_samples=Q)
    assert found == Q
    c0 = orc.cost(orc.drt(img0, U, B), pm)
    ups = []
    t = 0
    while len(ups) < Q:
        w = _draw(orc, seed, t, 0, 2, 1)
        p = (w[0] * n * n) >> 32
        trial = img0.copy()
        trial.flat[p] = _u01(w[2]) * beta  # f = 0.5 lies in [0, beta]
        d = orc.cost(orc.drt(trial, U, B), pm) - c0
        if d > 0:
            ups.append(d)
        t += 1
    assert abs(math.exp(-np.mean(ups) / t0) - 0.9) < 1e-12


def test_sat_reconstructs_small_noiseless_phantom(orc):
    n, U = 8, 12
    ph, B, _ = _small_problem(n, U, seed=2)
    pm = orc.drt(ph, U, B)
    img, st, _ = orc.sat_run(pm, np.full((n, n), 0.5), bome_k=8, n_sweeps=200, t0=-1, tn=-1, seed=4)
    assert st["final_cost_fresh"] < 0.08 * st["initial_cost"]
    assert synth.rmse(img, ph) < 0.08


def test_lockstep_follows_own_trace_and_flags_planted_error(orc):
    n, U, K = 8, 9, 4
    ph, B, _ = _small_problem(n, U)
    pm = synth.gaussian_noise(orc.drt(ph, U, B), 0.02, 1)
    img0 = np.full((n, n), 0.5)
    kw = dict(bome_k=K, n_sweeps=3, seed=5)
    img, st, tr = orc.sat_run(pm, img0, trace=True, t0=2e-3, tn=2e-6, **kw)
    g = np.zeros(len(tr), dtype=orc.GPU_TRACE_DTYPE)
    for f in ("pixel", "cstar", "accepted"):
        g[f] = tr[f]
    g["dS"], g["dC"], g["fnew"] = tr["dS"], tr["dC"], tr["fnew"]
    out, rep = orc.sat_lockstep(pm, img0, g, t0=st["t0"], tn=st["tn"], **kw)
    assert rep["moves"] == len(tr) and rep["near_ties"] == 0
    assert rep["hard_mismatch"] == -1 and rep["pixel_mismatch"] == -1
    assert rep["max_err_dS"] < 1e-6 and rep["max_err_dC"] < 1e-5
    assert np.allclose(out, img, atol=1e-6)
    # plant a decision flip on a clear-cut move: it must be reported
    clear = np.nonzero((tr["accepted"] == 0) & (tr["dC"] > 10 * tr["temp"]))[0]
    assert len(clear) > 0
    bad = g.copy()
    bad["accepted"][clear[0]] = 1
    _, rep2 = orc.sat_lockstep(pm, img0, bad, t0=st["t0"], tn=st["tn"], **kw)
    assert rep2["hard_mismatch"] == clear[0]


def test_sirt_factor_matrix_closed_form(orc):
    n, U = 6, 4
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    w = orc.sirt_factor(n, U, B, mask)
    # 0 degrees: ray k covers column j = k - (B-1-n)/2 with l = 1: W = mask pixels in it.
    for k in range(B):
        j = k - (B - 1 - n) // 2
        want = int(mask[:, j].sum()) if 0 <= j < n else 0
        assert w[0, k] == want
    # 45 degrees: l^2 summed from the closed form
    for k in range(B):
        want = sum(chord_closed_form(n, math.pi / 4, k - 0.5 * (B - 1), i, j) ** 2
                   for i in range(n) for j in range(n) if mask[i, j])
        assert abs(w[1, k] - want) < 1e-12


@pytest.mark.parametrize("mode", [0, 1])
def test_sirt_fixed_point_and_convergence(orc, mode):
    n, U = 8, 10
    ph, B, _ = _small_problem(n, U, seed=6)
    mask = synth.disk_mask(n)
    ph = ph * mask
    pm = orc.drt(ph, U, B)
    same, c = orc.sirt_run(pm, ph, 3, mode=mode, mask=mask)
    assert np.allclose(same, ph, atol=1e-13) and np.all(c < 1e-13)
    img, costs = orc.sirt_run(pm, synth.initial_image(n, 0.5, mask), 60, mode=mode, mask=mask)
    assert costs[-1] < 0.1 * costs[0]
    assert np.all(np.diff(costs[5:]) <= 1e-12)
    # pixels outside the reconstruction space are never touched
    assert np.all(img[mask == 0] == 0.0)


def test_sirt_single_update_by_hand(orc):
    """One simultaneous step from zero on a 1-pixel image: each angle's ray
    gives (P_m/W) * l with W = l^2, so the update is f* exactly."""
    n, U, B = 1, 5, 1
    pm = orc.drt(np.full((1, 1), 0.7), U, B)
    img, costs = orc.sirt_run(pm, np.zeros((1, 1)), 1, mode=0)
    assert abs(img[0, 0] - 0.7) < 1e-14 and costs[0] < 1e-14


def test_bilinear_drt_against_scipy_interpolation(orc):
    """The conventional forward model of Sec. III-A: every ray is the sum of B
    unit-step samples of the bilinear interpolant.  Checked against scipy's
    linear interpolation (zero beyond the grid) at the same sample points."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    for n, U in ((9, 7), (16, 12)):
        B = synth.bins_for(n)
        img = rng.random((n, n))
        got = orc.drt_bilinear(img, U, B)
        ks = np.arange(B) - 0.5 * (B - 1)
        ts = np.arange(B) - 0.5 * (B - 1)
        for u in range(U):
            th = np.pi * u / U
            c, s = np.cos(th), np.sin(th)
            c = 0.0 if abs(c) < 1e-12 else c
            s = 0.0 if abs(s) < 1e-12 else s
            x = ks[:, None] * c - ts[None, :] * s
            y = ks[:, None] * s + ts[None, :] * c
            rows, cols = 0.5 * (n - 1) - y, x + 0.5 * (n - 1)
            vals = ndimage.map_coordinates(img, [rows.ravel(), cols.ravel()], order=1, mode="grid-constant", cval=0.0)
            np.testing.assert_allclose(got[u], vals.reshape(B, B).sum(axis=1), rtol=1e-12, atol=1e-12)


def test_sat_with_full_drt_against_recomputation(orc):
    """SAT without the PILA: each move's dC is C' - C of a fresh bilinear DRT,
    the best of the estimates is kept, and the chain follows Step 4."""
    n, U, K, seed = 8, 7, 3, 21
    B = synth.bins_for(n)
    ph = synth.phantom(n, 3, 5)
    pm = orc.drt_bilinear(ph, U, B)
    img0 = np.full((n, n), 0.5)
    M = 30
    img, st, tr = orc.sat_drt_run(pm, img0, t0=1e-3, tn=1e-5, bome_k=K, n_sweeps=2, moves_per_sweep=M, seed=seed,
                                  trace=True)
    cur = img0.copy()
    cost = lambda im: float(np.sqrt(np.mean((orc.drt_bilinear(im, U, B) - pm) ** 2)))
    nblk = (K + 2 + 3) // 4
    for idx, rec in enumerate(tr):
        s, m = divmod(idx, M)
        w = _draw(orc, seed, s, m, 1, nblk)
        p = (w[0] * n * n) >> 32
        assert rec["pixel"] == p
        f = cur.flat[p]
        lo, hi = max(0.0, f - 1.0), min(1.0, f + 1.0)
        vals = [lo + _u01(w[2 + e]) * (hi - lo) for e in range(K)]
        costs = []
        for v in vals:
            t = cur.copy()
            t.flat[p] = v
            costs.append(cost(t))
        best = int(np.argmin(costs))
        assert rec["cstar"] == best
        assert abs(rec["dC"] - (costs[best] - cost(cur))) < 1e-12
        T = orc.schedule_temp(orc.SCHED_LINEAR, 1e-3, 1e-5, s, 2)
        dC = rec["dC"]
        assert bool(rec["accepted"]) == (dC <= 0 or _u01(w[1]) < np.exp(-dC / T))
        if rec["accepted"]:
            cur.flat[p] = vals[best]
    assert np.allclose(cur, img, atol=1e-15)
    assert abs(st["final_cost"] - st["final_cost_fresh"]) < 1e-12


def test_fbp_ramlak_and_reconstruction(orc):
    """FBP (the start image and spatial constraint of Step 1 / Fig. 9; filter
    read as Ram-Lak): the taps sum to zero up to the truncation bound
    1/(pi^2 (B - 1)), FBP is linear, and it reconstructs a uniform disk from
    exact line integrals: ~1 inside, ~0 outside, peak at an isolated pixel."""
    from oracle import fbp as F

    for B in (91, 363, 725):
        assert abs(F.ramlak(B).sum()) <= 1.0 / (np.pi ** 2 * (B - 1)) + 1e-12
    n, U = 64, 100
    B = synth.bins_for(n)
    disk = synth.disk_mask(n, 20.0).astype(np.float64)
    rec = F.fbp(orc.drt(disk, U, B), n)
    j = np.arange(n) - 0.5 * (n - 1)
    r = np.sqrt(j[None, :] ** 2 + j[:, None] ** 2)
    assert np.all(np.abs(rec[r < 17] - 1.0) < 0.06)
    ring = (r > 24) & (r < 31)  # just outside the disk: ringing of the pixelised edge only
    assert np.max(np.abs(rec[ring])) < 0.1 and np.mean(np.abs(rec[ring])) < 0.03
    assert np.mean(np.abs(rec[r > 23])) < 0.02
    a, b = np.random.default_rng(1).random((2, U, B))
    np.testing.assert_allclose(F.fbp(2.0 * a - 3.0 * b, n), 2.0 * F.fbp(a, n) - 3.0 * F.fbp(b, n), atol=1e-12)
    dot = np.zeros((n, n))
    dot[20, 41] = 1.0
    rd = F.fbp(orc.drt(dot, U, B), n)
    assert np.unravel_index(np.argmax(rd), rd.shape) == (20, 41)


def test_exhaustive_search_on_4x4_grid_images(orc):
    """Brute force on 4x4 images: every image with pixels in {0, 0.5, 1}
    (3^16 = 43 M) is scored by Eq. (4) through a Gray-ordered sinogram
    update.  With noiseless data of a grid phantom the least cost is 0, the
    phantom attains it, and SAT restricted to grid values (Steps 1-4 with
    Eq. (7), a slow schedule) ends at a global minimiser."""
    n, U, L = 4, 4, 3
    B = synth.bins_for(n)
    ph = np.array([[0.0, 0.5, 1.0, 0.5], [1.0, 0.0, 0.5, 0.0], [0.5, 1.0, 0.0, 1.0], [0.0, 0.5, 0.5, 1.0]])
    pm = orc.drt(ph, U, B)
    cmin, count, arg = orc.exhaustive_grid(pm, n, L, 1.0)
    assert cmin < 1e-9 and count >= 1
    assert orc.cost(orc.drt(arg, U, B), pm) < 1e-9
    # a wrong image is measurably worse: the grid search is not degenerate
    worse = ph.copy()
    worse[0, 0] = 1.0
    assert orc.cost(orc.drt(worse, U, B), pm) > 1e-3
    # SAT never beats the exhaustive minimum and, being stochastic, reaches
    # it in most runs (single-pixel moves can stall in a local minimum)
    reached = 0
    for seed in range(16):
        img, st, _ = orc.sat_run(pm, np.full((n, n), 0.5), bome_k=1, n_sweeps=2000, moves_per_sweep=16, t0=5e-2,
                                 tn=1e-5, seed=seed, grid_levels=L)
        assert st["final_cost_fresh"] >= cmin - 1e-9
        assert set(np.round(img.ravel() * 2).astype(int)) <= {0, 1, 2}
        reached += st["final_cost_fresh"] <= cmin + 1e-9
    assert reached >= 8
