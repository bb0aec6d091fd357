#!/usr/bin/env python
"""Benchmark: SAT pixel-moves/s on the batched workload.

Workload (per GPU): 512 independent 128x128 slices (20 seeded random
ellipses each, disk reconstruction space, uniform 0.5 start), 120 angles over
[0, 180), 181 bins, noiseless sinograms, BoME with 4 estimates, 50 linear
stages with T0 from Eq. (8), FP16 PILA, all chains in one persistent launch.
A step is one pass of the whole path over that batch: PILA build, FP64-grade
resync, Eq. (8) temperatures, 50 stages of moves, final resync and cost.
Metric: pixel-moves/s (one BoME selection + Metropolis decision = one move),
whole job.  Also reported: the plain single-chain FP32 form on a sample of
the same slices at equal final RMSE, the roofline of the sweep kernel, the
CPU reference oracle on a bounded sample, and the end-to-end rate through the
C-ABI with host buffers.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1411_4622_gb300 import shard, synth  # noqa: E402

WORKLOAD = "batch128x512"
PLAN_NAMES = {0: "independent-pixel BoME kernel", 1: "windowed, band residual in shared memory",
              2: "windowed, residual in global memory", 3: "windowed hybrid",
              4: "pipelined, 1 warp per chain", 5: "pipelined, 2 warps per chain",
              6: "pipelined, 4 warps per chain", 7: "windowed, 2 warps per chain, residual in global memory",
              8: "windowed, 4 warps per chain, residual in global memory",
              9: "windowed, 2 warps per chain, residual band in shared memory",
              10: "windowed, 4 warps per chain, residual band in shared memory"}
METRIC = "SAT pixel-moves/s at equal final RMSE (batched vs plain); slice p50/p99 ms"
UNIT = "pixel-moves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--slices", type=int, default=None, help="override slices per GPU (testing)")
    ap.add_argument("--sweeps", type=int, default=None, help="override stages (testing)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--residency", type=int, default=0, help="0 auto, 1 shared memory, 2 global memory")
    ap.add_argument("--group-warps", type=int, default=0, help="warps per chain (0: chosen by size)")
    ap.add_argument("--flags", type=int, default=0,
                    help="SAT_FLAG_* bits for the batched run (2: the autotuner picks the launch layout; --plan 0)")
    ap.add_argument("--plan", type=int, default=1,
                    help="SAT_PLAN_* launch layout of the batched run (default 1, the windowed kernel with its "
                         "residual band in shared memory: the autotuner's pick for this shape); 0: rules/autotuner")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "precision512", "precision512-rmse", "serve", "bome", "drt", "fbp", "rows",
                             "chain512"],
                    help="batch128x512 (default); precision512: 512^2 gather throughput; serve: request stream; "
                         "bome: convergence vs estimates, equal evaluations and schedules (Sec. III-B, III-C); "
                         "drt: speed of SAT with the PILA against SAT with a full DRT per move (Sec. III-A); "
                         "fbp: FBP against SAT with and without the FBP spatial constraint (Fig. 9); "
                         "rows: the other steps of the path (table build, forward projection, SIRT, one chain), "
                         "each timed alone")
    ap.add_argument("--requests", type=int, default=2000, help="serve: requests in the stream")
    ap.add_argument("--rate", type=float, default=None,
                    help="serve: arrival rate in requests/s (default: 80%% of the capacity measured on a burst)")
    ap.add_argument("--pila", default="f16", choices=["f16", "u8", "f32"],
                    help="table precision of the batched run (f16: 8-byte records; u8: the paper's one-byte lengths)")
    ap.add_argument("--tables", default="f16,f32,u8", help="precision512: table precisions, comma separated")
    ap.add_argument("--part", default="both", choices=["both", "gpu", "oracle"],
                    help="precision512-rmse: run the GPU side, the oracle side (no GPU needed) or both")
    ap.add_argument("--oracle-chains", type=int, default=4, help="precision512-rmse: chains the oracle follows")
    ap.add_argument("--no-c4", action="store_true", help="default run: skip the 512^2 sub-object")
    ap.add_argument("--no-serve", action="store_true", help="default run: skip the serving sub-object")
    ap.add_argument("--serve-requests", type=int, default=200, help="default run: requests of the serving sub-object")
    ap.add_argument("--serve-rate", type=float, default=7.0,
                    help="default run: arrival rate of the serving sub-object (requests/s)")
    return ap.parse_args()


def workload(args):
    cfg = dict(synth.WORKLOADS[WORKLOAD])
    if args.slices:
        cfg["slices"] = args.slices
    if args.sweeps:
        cfg["n_sweeps"] = args.sweeps
    return cfg


def make_slices(cfg, first, count):
    n = cfg["n"]
    mask = synth.disk_mask(n)
    phantoms = np.stack([synth.phantom(n, cfg["ellipses"], synth.slice_seeds(first + i)[0]) * mask
                         for i in range(count)])
    return phantoms, mask


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = {
    "sat_window_kernel": ["common.cuh", "sat_sweep.cuh", "sat_window.cuh", "sat_window_inst.cuh", "sat_window.cu"],
    "sat_hybrid_kernel": ["common.cuh", "sat_sweep.cuh", "sat_window.cuh", "sat_window_inst.cuh", "sat_window.cu"],
    "sat_window_group_kernel": ["common.cuh", "sat_sweep.cuh", "sat_window.cuh", "sat_window_inst.cuh",
                                "sat_window_group.cu", "sat_window_gsmem.cu"],
    "sat_sweep_kernel": ["common.cuh", "sat_sweep.cuh", "sat_f16_glob.cu", "sat_f16_smem.cu", "sat_f32_glob.cu",
                         "sat_f32_smem.cu"],
}


def launch_name(plan, flags, pinned=0):
    """The launch layout a run used, and who chose it."""
    who = ("pinned: " if pinned else "autotuned: " if flags & 2 else "requested: " if flags & 16
           else "size rules: ")
    return who + PLAN_NAMES.get(plan, str(plan))


# the sweep kernel each launch layout (sat_stats.plan) runs
PLAN_KERNEL = {1: "sat_window_kernel", 2: "sat_window_kernel", 3: "sat_hybrid_kernel", 4: "sat_sweep_kernel",
               5: "sat_sweep_kernel", 6: "sat_sweep_kernel", 7: "sat_window_group_kernel",
               8: "sat_window_group_kernel", 9: "sat_window_group_kernel", 10: "sat_window_group_kernel"}


def kernel_source_hash(kernel):
    """Hash of the device sources of `kernel`; a stored DRAM-traffic figure
    only applies to them."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1411_4622_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(f.encode())
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def stored_profile(kernel, workload=WORKLOAD, key="dram_bytes_per_move"):
    """A per-move figure of `kernel` (DRAM bytes, warp instructions) from the
    committed ncu summary, or None when the summary is missing, lacks it, or
    was taken on different sources."""
    path = os.path.join(ROOT, "profiles", f"{kernel}__{workload}.md")
    try:
        kv = {}
        for ln in open(path):
            if ":" in ln and ln.startswith("- "):
                k, v = ln[2:].split(":", 1)
                kv[k.strip()] = v.strip().strip("`")
        if kv.get("source_sha") != kernel_source_hash(kernel):
            return None
        return float(kv[key])
    except (OSError, KeyError, ValueError):
        return None


def stored_traffic(kernel, workload=WORKLOAD):
    return stored_profile(kernel, workload, "dram_bytes_per_move")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measure_peaks(api):
    """Read rates of each memory level on this GPU, from the library's probes
    (satpila_probe_read / satpila_probe_smem): the denominators of the
    gathers' rooflines.  The PILA row is read as consecutive 16-byte chunks
    (stream), the residual cells as one 32-byte sector per record at
    scattered places (sector) or as scattered 4-byte shared-memory words.
    L2: a 64 MB buffer (inside the 126 MB L2); HBM: a 4 GB buffer (32x L2),
    sectors gathered by each warp inside its own 1 MiB region (as a chain's
    warps gather inside its residual) and, for comparison, over the whole
    buffer (then bound by address translation).  The HBM copy figure is
    MEASURED_PEAKS.json's."""
    import torch

    copy, kind = peaks()
    out = {"hbm_copy_gbs": copy, "hbm_copy_kind": kind}
    buf = torch.ones(64 << 20, dtype=torch.uint8, device="cuda")
    out["l2_stream_gbs"] = api.probe_read(buf, api.PROBE_STREAM, loads=1 << 30)
    out["l2_sector_gbs"] = api.probe_read(buf, api.PROBE_SECTOR, loads=1 << 28)
    del buf
    buf = torch.ones(4 << 30, dtype=torch.uint8, device="cuda")
    out["hbm_stream_gbs"] = api.probe_read(buf, api.PROBE_STREAM, loads=1 << 29)
    # sectors gathered inside 1 MiB regions, one per warp: the residual of a
    # 512^2 chain (360 rows of 728 cells) is 1.05 MB and its warps gather in it
    out["hbm_sector_gbs"] = api.probe_read(buf, api.PROBE_SECTOR, loads=1 << 28, region_bytes=1 << 20)
    out["hbm_sector_scatter_gbs"] = api.probe_read(buf, api.PROBE_SECTOR, loads=1 << 26)
    del buf
    torch.cuda.empty_cache()
    out["smem_gbs"] = api.probe_smem(0, loads=1 << 33)
    out["smem_random_gbs"] = api.probe_smem(1, loads=1 << 32)
    out["how"] = ("satpila_probe_read/_smem: one untimed and one timed launch of 8 CTAs x 256 threads per SM, "
                  "8 independent loads in flight per thread, L1 bypassed; CUDA events")
    return out


def issue_peak(clk):
    """Warp instructions per second the SMs can issue: 4 schedulers per SM,
    one instruction each per cycle, at the sampled SM clock (else the maximum,
    2070 MHz)."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    return sms * 4 * mhz * 1e6, sms, mhz


_ORACLE_SLICES = {}


def _oracle_problem(cfg, idx):
    import oracle

    if idx not in _ORACLE_SLICES:
        n, U, B = cfg["n"], cfg["n_angles"], cfg["n_bins"]
        ph, mask = make_slices(cfg, idx, 1)
        _ORACLE_SLICES[idx] = (oracle.drt(ph[0], U, B), synth.initial_image(n, 0.5, mask), mask)
    return _ORACLE_SLICES[idx]


def _oracle_slice(job):
    """Worker of the CPU oracle pool: run slice idx for a number of stages with
    the FP64 oracle as it stands; returns (moves, seconds)."""
    import oracle

    cfg, idx, stages = job
    pm, img0, mask = _oracle_problem(cfg, idx)
    if stages <= 0:
        return 0, 0.0
    t = time.perf_counter()
    _, st, _ = oracle.sat_run(pm, img0, n_sweeps=stages, bome_k=cfg["bome_k"], mask=mask,
                              seed=synth.slice_seeds(idx)[2], beta=cfg["beta"])
    return st["proposed"], time.perf_counter() - t


class OraclePool:
    """One single-threaded oracle process per host core, each on its own slice
    (spawned, so no CUDA state is inherited)."""

    def __init__(self, cfg, procs=None):
        import multiprocessing as mp

        import oracle

        oracle.build()
        self.cfg = cfg
        self.procs = procs or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.procs)
        self.run(0)  # import the oracle and set up every worker's slice

    def run(self, stages, per_proc=1):
        """per_proc x procs slices, each run for `stages` stages; (moves, wall s)."""
        jobs = [(self.cfg, i, stages) for i in range(self.procs * per_proc)]
        t = time.perf_counter()
        res = self.pool.map(_oracle_slice, jobs, chunksize=1)
        return sum(r[0] for r in res), time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_slices_for(cfg, budget_s):
    """Whole-schedule slices per core that take the oracle about budget_s:
    per-stage time from a 1-stage and a 3-stage run (setup cancels)."""
    t1 = _oracle_slice((cfg, 0, 1))[1]
    t3 = _oracle_slice((cfg, 0, 3))[1]
    per = max((t3 - t1) / 2.0, 1e-4)
    return int(max(1, min(16, round(budget_s / (per * cfg["n_sweeps"])))))


def cpu_baseline(cfg, budget_s=12.0):
    """The FP64 oracle as it stands (single-threaded per process), one process
    per host core, on distinct slices of the workload, each annealed over the
    workload's whole schedule, about budget_s in all."""
    per_proc = oracle_slices_for(cfg, budget_s)
    stages = cfg["n_sweeps"]
    pool = OraclePool(cfg)
    try:
        moves, wall = pool.run(stages, per_proc)
    finally:
        pool.close()
    count = pool.procs * per_proc
    return {"value": moves / wall, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
            "sample": f"{count} slices of {WORKLOAD} ({per_proc} per process), {stages} stages x "
                      f"{moves // max(1, stages * count)} moves each, K={cfg['bome_k']}, FP64, "
                      f"{wall:.1f} s wall"}


def run_reference(args, cfg):
    """The reference arm: the FP64 oracle on the host cores, one process per
    core; a step is every process running the workload's whole schedule on
    its own slice."""
    stages = cfg["n_sweeps"]
    pool = OraclePool(cfg)
    times, moves = [], 0
    try:
        for it in range(args.warmup + args.steps):
            mv, dt = pool.run(stages)
            if it >= args.warmup:
                times.append(dt)
                moves = mv
    finally:
        pool.close()
    ms = 1e3 * statistics.mean(times)
    value = moves / (ms / 1e3)
    sample = (f"{pool.procs} slices of {WORKLOAD} (one process per core), {stages} stages per step, "
              f"K={cfg['bome_k']}, FP64 oracle")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "sample": sample},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def timed_steps(args, step, stream, dist, local):
    """W warm-up steps, then K timed steps (L2 flushed between them, outside
    the events); returns (per-step ms, per-step stats, clocks)."""
    import torch

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, stats = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stats.append(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return step_ms, stats, clocks.stop()


def precision_phantoms(cfg, distinct):
    """Seeded 512^2 phantoms (40 ellipses, disk reconstruction space) and
    their measured sinograms: the discrete model's projection through an FP32
    table (FP64-grade sums), then Poisson noise at 1e5 photons per bin."""
    import torch

    from paper_1411_4622_gb300 import api

    n, U, B = cfg["n"], cfg["n_angles"], cfg["n_bins"]
    mask = synth.disk_mask(n)
    ph = np.stack([synth.phantom(n, cfg["ellipses"], synth.slice_seeds(i)[0]) * mask for i in range(distinct)])
    pf = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    clean = api.pila_forward(pf, torch.tensor(ph, dtype=torch.float32, device="cuda")).cpu().numpy()
    api.pila_free(pf)
    noisy = np.stack([synth.poisson_noise(clean[i], cfg["noise"][1], synth.slice_seeds(i)[1])
                      for i in range(distinct)]).astype(np.float32)
    return ph, noisy, mask


def precision_sample(pk, *, chains=304, stages=2, tables=("f16", "f32", "u8"), steps=2, warmup=1, flags=0,
                     residency=0, group_warps=0, plan=8):
    """The 512^2 configuration as configured, on a bounded sample of its
    schedule: C chains of 512x512 slices (8 distinct phantoms, each chain its
    own seed), 360 angles, 725 bins, K = 8, M = every reconstruction-space
    pixel per stage (205,887 moves), the FP64-grade resync after every stage
    (a fresh forward projection replaces the incremental residual and the
    drift is recorded), T0 by Eq. (8); `stages` stages of a linear schedule of
    that length.  One step: table build, resync, Eq. (8), the stages with
    their resyncs, final cost.  Per table precision: moves/s over the step
    and in the sweep kernel, the sweep's bytes per move against the measured
    HBM stream and sector-gather rates, the drift bound."""
    import types

    import torch

    from paper_1411_4622_gb300 import api

    cfg = dict(synth.WORKLOADS["precision512"])
    n, U, B, K = cfg["n"], cfg["n_angles"], cfg["n_bins"], cfg["bome_k"]
    distinct = min(8, chains)
    ph, noisy, mask = precision_phantoms(cfg, distinct)
    M = int(mask.sum())
    idx = np.arange(chains) % distinct
    sino = torch.tensor(noisy[idx], device="cuda").contiguous()
    pm_max = float(np.max(np.abs(noisy)))
    init = torch.tensor(np.stack([synth.initial_image(n, 0.5, mask)] * chains), dtype=torch.float32, device="cuda")
    images = init.clone()
    stream = torch.cuda.current_stream()
    moves = chains * stages * M
    # the sector-gather rate of this working set: one region per chain the
    # size of its residual (U rows of B + 1 cells padded to 4, plus the
    # lanes' dummy cells), all chains' residuals at once (partly L2-resident)
    resid_bytes = (U * ((B + 1 + 3) // 4 * 4) + 256) * 4 // 32 * 32
    buf = torch.ones(chains * resid_bytes, dtype=torch.uint8, device="cuda")
    from paper_1411_4622_gb300 import api as _api

    pk = dict(pk, ws_sector_gbs=_api.probe_read(buf, _api.PROBE_SECTOR, loads=1 << 27, region_bytes=resid_bytes),
              ws_bytes=chains * resid_bytes)
    del buf
    torch.cuda.empty_cache()
    out = {"workload": "precision512", "chains": chains, "distinct_slices": distinct, "n": n, "angles": U,
           "bins": B, "bome_k": K, "moves_per_stage": M, "stages": stages, "resync_every": 1,
           "sample": f"{stages} stages of full M (a linear schedule of {stages} stages from Eq. (8)'s T0; the "
                     f"configured schedule has {cfg['n_sweeps']})",
           "l2": "flushed between timed steps (256 MB write)", "steps": steps, "warmup": warmup, "tables": {}}
    for t in tables:
        prec = {"f16": api.PILA_F16, "f32": api.PILA_F32, "u8": api.PILA_U8}[t]
        kw = dict(bome_k=K, n_sweeps=stages, moves_per_sweep=M, t0=-1.0, tn=-1.0, seed=synth.slice_seeds(0)[2],
                  resync_every=1, residency=residency, group_warps=group_warps, flags=flags, plan=plan)
        info = {}

        def step():
            images.copy_(init)
            p = api.pila_build(n, U, B, prec, mask=mask)
            st = api.sat_run(p, sino, images, **kw)
            if not info:
                info.update(api.pila_info(p))
            api.pila_free(p)
            return st

        step_ms, stats, clk = timed_steps(types.SimpleNamespace(warmup=warmup, steps=steps), step, stream, None, 0)
        ms = statistics.mean(step_ms)
        st = stats[-1]
        acc = sum(x["accepted"] for x in st) / max(1, sum(x["proposed"] for x in st))
        sweep_ms = statistics.mean(x[0]["sweep_ms"] for x in stats)
        rate = moves / (sweep_ms / 1e3)
        E = info["entries"] / (n * n)
        row_bytes = info["row_records"] * info["record_bytes"]
        # one 32-byte sector per angle, two when a record's entries straddle a
        # sector boundary (k0 = 7 mod 8: 1/8 of the records with two entries)
        sectors = U * (1.0 + (E / U - 1.0) / 8.0)
        # sectors read (the gather) and written back (the scatter: the same
        # sectors, just read, written when the move is accepted)
        sector_resid = 32.0 * sectors + 8.0
        sector_write = (32.0 * sectors + 8.0) * acc
        useful = row_bytes + 4.0 * E * (1.0 + acc) + 4.0 * (1.0 + acc)
        # seconds of memory time per move at the probe rates: rows streamed
        # from HBM (the table is 6-12x L2), residual sectors gathered from the
        # chains' residuals (the probe over the same footprint)
        t_row = row_bytes / (pk["hbm_stream_gbs"] * 1e9)
        t_sec = sector_resid / (pk["ws_sector_gbs"] * 1e9)
        kernel = PLAN_KERNEL.get(st[0]["plan"], "sat_sweep_kernel")
        tpm = stored_traffic(kernel, "precision512")
        achieved = (row_bytes + sector_resid) * rate / 1e9
        peak_eff = (row_bytes + sector_resid) / (t_row + t_sec) / 1e9
        out["tables"][t] = {
            "moves_per_s": moves / (ms / 1e3), "sweep_moves_per_s": rate, "ms_per_step": ms, "sweep_ms": sweep_ms,
            "other_ms": ms - sweep_ms, "acceptance": acc, "table_bytes": info["table_bytes"],
            "launch": launch_name(st[0]["plan"], flags, plan),
            "drift_max_rel": max(x["max_resync_drift"] for x in st) / pm_max,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak_eff, "unit": "GB/s",
                         "frac": achieved / peak_eff, "kernel": kernel,
                         "bytes_per_move": row_bytes + sector_resid, "row_bytes": row_bytes,
                         "sector_bytes": sector_resid, "sector_write_bytes": sector_write,
                         "useful_bytes_per_move": useful,
                         "peak_rule": "bytes read: rows at the HBM stream rate, residual sectors at the sector-gather "
                                      "rate of the chains' residual footprint (one 1.05 MB region per chain; the "
                                      "probe's random sectors move 64 bytes of DRAM each, the residual's paired rows "
                                      "put two needed sectors in most 64-byte blocks); every byte class, the "
                                      "scatter's write-back included, against the HBM copy rate in frac_all_vs_hbm",
                         "frac_all_vs_hbm": (row_bytes + sector_resid + sector_write) * rate / 1e9 / pk["hbm_copy_gbs"],
                         "frac_rows": row_bytes * rate / 1e9 / pk["hbm_stream_gbs"],
                         "frac_sectors": sector_resid * rate / 1e9 / pk["ws_sector_gbs"],
                         "frac_sectors_vs_hbm_probe": sector_resid * rate / 1e9 / pk["hbm_sector_gbs"],
                         "ws_sector_gbs": pk["ws_sector_gbs"],
                         "traffic": tpm * chains * stages * M if tpm is not None else None,
                         "traffic_over_sector_bytes": (tpm / (row_bytes + sector_resid + sector_write)
                                                       if tpm is not None else None)},
            "clocks": clk}
    return out


def run_precision(args):
    """--workload precision512: the 512^2 configuration as configured
    (resync every stage, full M), FP16 and FP32 tables; one JSON line."""
    import torch

    from paper_1411_4622_gb300 import api
    from paper_1411_4622_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    pk = measure_peaks(api)
    sub = precision_sample(pk, chains=args.slices or 304, stages=args.sweeps or 2, steps=args.steps,
                           warmup=args.warmup, flags=args.flags, residency=args.residency,
                           group_warps=args.group_warps, tables=tuple(args.tables.split(",")),
                           plan=8 if args.plan == 1 else args.plan)
    main = sub["tables"][sub_first(sub)]
    out = {"metric": "SAT pixel-moves/s, 512x512 slices, resync every stage", "value": main["moves_per_s"],
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {k: v for k, v in sub.items() if k != "tables"}, "tables": sub["tables"],
           "roofline": main["roofline"], "peaks": pk, "clocks": main["clocks"]}
    print(json.dumps(out))


def _c4_problem(i):
    """Slice i of the 512^2 configuration for the oracle comparison: phantom
    (40 ellipses, disk reconstruction space), the oracle's FP64 Siddon DRT of
    it, Poisson noise at 1e5 photons, rounded to float32 (the values both
    sides read)."""
    import oracle

    cfg = synth.WORKLOADS["precision512"]
    n, U, B = cfg["n"], cfg["n_angles"], cfg["n_bins"]
    mask = synth.disk_mask(n)
    ph = synth.phantom(n, cfg["ellipses"], synth.slice_seeds(i)[0]) * mask
    pm = synth.poisson_noise(oracle.drt(ph, U, B), cfg["noise"][1], synth.slice_seeds(i)[1]).astype(np.float32)
    return ph, pm, mask


def _c4_oracle_chain(job):
    """Worker: the FP64 oracle over chain c's whole schedule (lengths exact or
    rounded to binary16 as the FP16 table stores them); final RMSE against
    the phantom on the reconstruction space."""
    import oracle

    c, slice_idx, seed, stages, fmt = job
    ph, pm, mask = _c4_problem(slice_idx)
    cfg = synth.WORKLOADS["precision512"]
    t = time.perf_counter()
    img, st, _ = oracle.sat_run(pm.astype(np.float64), synth.initial_image(cfg["n"], 0.5, mask), n_sweeps=stages,
                                bome_k=cfg["bome_k"], mask=mask, seed=seed, beta=cfg["beta"], length_format=fmt)
    return {"chain": c, "slice": slice_idx, "length_format": ["exact", "binary16", "byte180"][fmt],
            "rmse": float(synth.rmse(img, ph, mask)), "final_cost": st["final_cost_fresh"], "t0": st["t0"],
            "accepted": st["accepted"], "seconds": time.perf_counter() - t}


def run_precision_rmse(args):
    """The 512^2 configuration in full, with its errors against the FP64
    oracle: C chains (slice c mod 8, seed 3000 + c), 200 stages of full M,
    K = 8, resync after every stage, T0 by Eq. (8), on the FP16 and the FP32
    table; final RMSE against the phantom per chain, drift per resync.  The
    oracle runs the first chains over the same schedule with exact lengths
    and with the binary16 lengths of the FP16 table (one process per chain).
    --part gpu / oracle runs one side (the oracle needs no GPU)."""
    cfg = synth.WORKLOADS["precision512"]
    n, K = cfg["n"], cfg["bome_k"]
    S = args.sweeps or cfg["n_sweeps"]
    C = args.slices or 16
    n_or = min(C, args.oracle_chains)
    seed0 = synth.slice_seeds(0)[2]
    out = {"metric": "final RMSE against the phantom, 512x512, GPU (FP16 / FP32 table) and FP64 oracle",
           "unit": "rmse", "higher_is_better": False, "data": "synthetic",
           "config": {"workload": "precision512-rmse", "chains": C, "distinct_slices": min(8, C), "n": n,
                      "angles": cfg["n_angles"], "bins": cfg["n_bins"], "bome_k": K, "stages": S,
                      "moves_per_stage": "all reconstruction-space pixels", "resync_every": 1,
                      "oracle_chains": n_or, "sinogram": "oracle FP64 Siddon DRT + Poisson 1e5, as float32"}}
    import multiprocessing as mp

    pool = None
    if args.part in ("both", "oracle") and n_or > 0:
        import oracle

        oracle.build()
        jobs = [(c, c % 8, seed0 + c, S, fmt) for fmt in (0, 1) for c in range(n_or)]
        pool = mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1))
        pending = pool.map_async(_c4_oracle_chain, jobs, chunksize=1)
    if args.part in ("both", "gpu"):
        import torch

        from paper_1411_4622_gb300 import api
        from paper_1411_4622_gb300 import build as libbuild

        libbuild.build()
        torch.cuda.set_device(0)
        distinct = min(8, C)
        probs = [_c4_problem(i) for i in range(distinct)]
        mask = probs[0][2]
        M = int(mask.sum())
        sino = torch.tensor(np.stack([probs[c % distinct][1] for c in range(C)]), device="cuda").contiguous()
        init = torch.tensor(np.stack([synth.initial_image(n, 0.5, mask)] * C), dtype=torch.float32, device="cuda")
        pm_max = max(float(np.max(np.abs(p[1]))) for p in probs)
        out["gpu"] = {}
        for name, prec in (("f16", api.PILA_F16), ("f32", api.PILA_F32)):
            p = api.pila_build(n, cfg["n_angles"], cfg["n_bins"], prec, mask=mask)
            img = init.clone()
            torch.cuda.synchronize()
            t = time.perf_counter()
            st = api.sat_run(p, sino, img, bome_k=K, n_sweeps=S, t0=-1.0, tn=-1.0, seed=seed0, resync_every=1,
                             flags=api.SAT_FLAG_AUTOTUNE)
            wall = time.perf_counter() - t
            api.pila_free(p)
            final = img.cpu().numpy()
            rm = [float(synth.rmse(final[c], probs[c % distinct][0], mask)) for c in range(C)]
            out["gpu"][name] = {"rmse": rm, "rmse_mean": float(np.mean(rm)),
                                "final_cost": [x["final_cost"] for x in st], "t0": [x["t0"] for x in st],
                                "drift_max_rel": max(x["max_resync_drift"] for x in st) / pm_max,
                                "moves_per_s": C * S * M / wall, "sweep_ms": st[0]["sweep_ms"], "wall_s": wall,
                                "launch": launch_name(st[0]["plan"], api.SAT_FLAG_AUTOTUNE)}
        g16, g32 = out["gpu"]["f16"]["rmse"], out["gpu"]["f32"]["rmse"]
        out["f16_vs_f32_rel"] = [abs(a - b) / b for a, b in zip(g16, g32)]
    if pool is not None:
        res = pending.get()
        pool.close()
        pool.join()
        out["oracle"] = res
        ex = {r["chain"]: r["rmse"] for r in res if r["length_format"] == "exact"}
        b16 = {r["chain"]: r["rmse"] for r in res if r["length_format"] == "binary16"}
        out["oracle_rmse_exact"] = [ex[c] for c in sorted(ex)]
        out["oracle_rmse_binary16"] = [b16[c] for c in sorted(b16)]
        if "gpu" in out:
            for name in ("f16", "f32"):
                g = out["gpu"][name]["rmse"]
                out["gpu"][name]["vs_oracle_exact_rel"] = [abs(g[c] - ex[c]) / ex[c] for c in sorted(ex)]
                out["gpu"][name]["vs_oracle_binary16_rel"] = [abs(g[c] - b16[c]) / b16[c] for c in sorted(b16)]
    print(json.dumps(out))


def sub_first(sub):
    return next(iter(sub["tables"]))


def serve_stream(nreq, rate=None, burst=400, seed=7):
    """The serving workload: a Poisson stream of nreq requests, sizes uniform
    over {64, 128, 256, 512}^2, angles uniform in [N/2, N], 2 floor(N/sqrt 2)
    + 1 bins, Gaussian (1% of max) or Poisson (1e5) noise with probability
    1/2, K uniform over {1, 4, 8}, 50 stages each, FP16 PILA, disk
    reconstruction space, under a 120 GB (1.2e11 bytes) device budget.  The
    arrival rate is `rate` requests/s, else 80% of the capacity measured on a
    closed burst of the first `burst` requests.  Returns moves/s over the
    stream and per-request latency (submit to result) p50/p99."""
    import torch

    from paper_1411_4622_gb300 import api

    rng = np.random.default_rng(seed)
    sizes = rng.choice([64, 128, 256, 512], size=nreq)
    angles = np.array([rng.integers(s // 2, s + 1) for s in sizes])
    noise = rng.integers(0, 2, size=nreq)
    ks = rng.choice([1, 4, 8], size=nreq)
    pool = 8  # distinct phantoms per size
    phid = rng.integers(0, pool, size=nreq)
    masks = {s: synth.disk_mask(s) for s in (64, 128, 256, 512)}
    phantoms = {s: np.stack([synth.phantom(s, 20, 5000 + 100 * i + s) * masks[s] for i in range(pool)])
                for s in (64, 128, 256, 512)}
    # sinograms: one FP32 table per (size, angles), all phantoms of that size
    sinos = {}
    for s, u in sorted(set(zip(sizes.tolist(), angles.tolist()))):
        pf = api.pila_build(s, u, synth.bins_for(s), api.PILA_F32, mask=masks[s])
        sinos[(s, u)] = api.pila_forward(pf, torch.tensor(phantoms[s], dtype=torch.float32,
                                                          device="cuda")).cpu().numpy()
        api.pila_free(pf)
    reqs = []
    for i in range(nreq):
        s, u = int(sizes[i]), int(angles[i])
        clean = sinos[(s, u)][phid[i]]
        sn = (synth.gaussian_noise(clean, 0.01, 9000 + i) if noise[i] == 0
              else synth.poisson_noise(clean, 1e5, 9000 + i)).astype(np.float32)
        reqs.append(dict(sino=sn, n=s, precision=api.PILA_F16, mask=masks[s], bome_k=int(ks[i]), n_sweeps=50,
                         seed=20000 + i, t0=-1.0, tn=-1.0))
    moves_of = [50 * int(masks[r["n"]].sum()) for r in reqs]
    budget = 120 * 10**9
    cap = None
    with api.Server(stages_per_tick=5, mem_budget=budget) as srv:
        if rate is None:
            # capacity: a closed burst of the first requests
            nb = min(burst, nreq)
            t = time.perf_counter()
            tk = [srv.submit(**reqs[i]) for i in range(nb)]
            for x in tk:
                srv.wait(x)
            cap = sum(moves_of[:nb]) / (time.perf_counter() - t)
            rate = 0.8 * cap / float(np.mean(moves_of))  # requests per second
        gaps = rng.exponential(1.0 / rate, size=nreq)
        clocks = ClockSampler(0)
        clocks.start()
        t0 = time.perf_counter()
        due = t0
        tickets = []
        for i in range(nreq):
            due += gaps[i]
            while time.perf_counter() < due:
                time.sleep(min(0.001, max(0.0, due - time.perf_counter())))
            tickets.append(srv.submit(**reqs[i]))
        lat, done_moves, failed = [], 0, 0
        by_size = {s: [] for s in (64, 128, 256, 512)}
        for i, x in enumerate(tickets):
            img, st = srv.wait(x)
            lat.append(st["done_ms"] - st["submit_ms"])
            by_size[int(sizes[i])].append(lat[-1])
            done_moves += st["proposed"]
            failed += int(st["status"] != 0)
        wall = time.perf_counter() - t0
        clk = clocks.stop()
        info = srv.info()
    return {"moves_per_s": done_moves / wall, "wall_ms": wall * 1e3, "requests": nreq,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "latency_p50_ms_by_size": {str(s): float(np.percentile(v, 50)) for s, v in by_size.items() if v},
            "rate_per_s": rate, "capacity_moves_per_s": cap, "failed": failed,
            "config": {"sizes": [64, 128, 256, 512], "stages": 50, "k": [1, 4, 8], "pila": "f16",
                       "budget_bytes": budget, "arrival": "poisson", "geometries": len(sinos),
                       "launches": "one per window for each image size's classes (windowed kernel, 4-warp groups)"},
            "server": {k: info[k] for k in ("ticks", "bytes_peak", "geometries", "classes")}, "clocks": clk}


def run_serve(args):
    """--workload serve: the whole request stream (default 2000 requests),
    arrival rate given or 80% of the burst capacity; one JSON line."""
    import torch

    from paper_1411_4622_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    r = serve_stream(args.requests, args.rate)
    out = {"metric": "SAT pixel-moves/s, served request stream; request p50/p99 ms", "value": r["moves_per_s"],
           "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": r["wall_ms"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": dict(workload="serve", requests=args.requests, rate_per_s=r["rate_per_s"],
                          rate_rule="given" if args.rate else "80% of burst capacity",
                          capacity_moves_per_s=r["capacity_moves_per_s"], **r["config"]),
           "latency_ms": r["latency_ms"], "latency_p50_ms_by_size": r["latency_p50_ms_by_size"], "failed": r["failed"],
           "server": r["server"], "clocks": r["clocks"]}
    print(json.dumps(out))


def nrmse(img, ref):
    """Root mean square of (img - ref) divided by the mean of ref (Sec. III-B)."""
    d = np.asarray(img, np.float64) - np.asarray(ref, np.float64)
    return float(np.sqrt(np.mean(d * d)) / np.mean(ref))


def run_bome(args):
    """The experiments of Sec. III-B and III-C on synthetic phantoms: final
    NRMSE against N_e (both readings of BoME), N_e = 1 with the evaluations of
    N_e = 4 spread over more stages or moves, and the three cooling
    schedules at N_e = 1 and 16.  64x64 slices (10 random ellipses, the disk
    reconstruction space), 60 angles, beta = 0.9, T0 by Eq. (8), T_N = T0/1000;
    each configuration runs C chains (C phantoms) in one launch."""
    import torch

    from paper_1411_4622_gb300 import api
    from paper_1411_4622_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    n, U, C = 64, 60, args.slices or 16
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    N, M = (args.sweeps or 200), 2000
    ph = np.stack([synth.phantom(n, 10, synth.slice_seeds(i)[0]) * mask for i in range(C)])
    p = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    sino = api.pila_forward(p, torch.tensor(ph, dtype=torch.float32, device="cuda")).float().contiguous()
    init = torch.tensor(np.stack([synth.initial_image(n, 0.5, mask)] * C), dtype=torch.float32, device="cuda")

    def run(K, flags=0, sweeps=N, moves=M, schedule=api.SAT_SCHED_LINEAR):
        imgs = init.clone()
        t = time.perf_counter()
        st = api.sat_run(p, sino, imgs, bome_k=K, n_sweeps=sweeps, moves_per_sweep=moves, beta=0.9, t0=-1.0,
                         tn=-1.0, schedule=schedule, seed=synth.slice_seeds(0)[2], resync_every=max(1, sweeps // 10),
                         flags=flags)
        dt = time.perf_counter() - t
        out = imgs.cpu().numpy()
        return {"nrmse": float(np.mean([nrmse(out[i], ph[i]) for i in range(C)])),
                "moves_per_s": C * sweeps * moves / dt, "cost": float(np.mean([x["final_cost"] for x in st]))}

    ks = [1, 2, 4, 8, 16, 32]
    vs_k = {"independent": {k: run(k, api.SAT_FLAG_BOME_INDEPENDENT) for k in ks},
            "one_pixel": {k: run(k) for k in ks}}
    equal_eval = {f"N={N * f}, M={M * 4 // f}": run(1, 0, N * f, M * 4 // f) for f in (1, 2, 4)}
    scheds = {}
    for k in (1, 16):
        for name, sc in (("linear", api.SAT_SCHED_LINEAR), ("geometric", api.SAT_SCHED_GEOMETRIC),
                         ("cubic", api.SAT_SCHED_CUBIC)):
            scheds[f"N_e={k} {name}"] = run(k, api.SAT_FLAG_BOME_INDEPENDENT, schedule=sc)
    api.pila_free(p)
    out = {"metric": "final NRMSE (mean over slices)", "unit": "nrmse", "higher_is_better": False,
           "data": "synthetic",
           "config": {"workload": "bome", "n": n, "angles": U, "bins": B, "slices": C, "stages": N,
                      "moves_per_stage": M, "beta": 0.9, "pila": "f32"},
           "vs_estimates": vs_k, "equal_evaluations_Ne1": equal_eval,
           "equal_evaluations_Ne4": vs_k["independent"][4], "schedules": scheds}
    print(json.dumps(out))


def run_drt(args):
    """Sec. III-A's speed comparison (Fig. 3) on this GPU: SAT with the PILA
    against SAT with a full bilinear-interpolation DRT per move, for 64, 128
    and 256 pixel slices at 90, 180 and 360 angles, N = 1 stage of M = 200
    moves, one estimate, T0 = 1e-3.  Both on the GPU, one chain and 152
    chains (one CTA per SM for the DRT form); and both single-threaded on
    the host (the oracle), the paper's own setting, on a subset."""
    import torch

    from paper_1411_4622_gb300 import api
    from paper_1411_4622_gb300 import build as libbuild
    import oracle

    libbuild.build()
    oracle.build()
    torch.cuda.set_device(0)
    M = 200
    kw = dict(bome_k=1, n_sweeps=1, moves_per_sweep=M, t0=1e-3, tn=1e-6, seed=777)
    rows = []
    for n in (64, 128, 256):
        B = synth.bins_for(n)
        mask = synth.disk_mask(n)
        ph = synth.phantom(n, 10, synth.slice_seeds(0)[0]) * mask
        for U in (90, 180, 360):
            pm = oracle.drt(ph, U, B) if n <= 128 else None
            pf = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
            pm_d = api.pila_forward(pf, torch.tensor(ph[None], dtype=torch.float32, device="cuda")).float()
            api.pila_free(pf)
            row = {"n": n, "angles": U}
            for C in (1, 152):
                sino = pm_d.expand(C, U, B).contiguous()
                init = torch.tensor(np.stack([synth.initial_image(n, 0.5, mask)] * C), dtype=torch.float32,
                                    device="cuda")
                p = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
                img = init.clone()
                api.sat_run(p, sino, img, **kw)
                img = init.clone()
                st = api.sat_run(p, sino, img, **kw)
                pila_rate = C * M / (st[0]["sweep_ms"] / 1e3)
                api.pila_free(p)
                img = init.clone()
                st = api.sat_drt_run(sino, img, mask=mask, **kw)
                drt_rate = C * M / (st[0]["sweep_ms"] / 1e3)
                row[f"gpu_chains{C}"] = {"pila_moves_per_s": pila_rate, "drt_moves_per_s": drt_rate,
                                         "speedup": pila_rate / drt_rate}
            if pm is not None and U == 90:
                # the paper's setting: one CPU thread, both forms
                # per-move time as the difference of two run lengths (the setup cancels)
                def per_move(fn, m1, m2):
                    ts = []
                    for mm in (m1, m2):
                        t = time.perf_counter()
                        fn(pm, synth.initial_image(n, 0.5, mask), t0=1e-3, tn=1e-6, n_sweeps=1, moves_per_sweep=mm,
                           seed=777, mask=mask)
                        ts.append(time.perf_counter() - t)
                    return (ts[1] - ts[0]) / (m2 - m1)

                m_drt = (10, 30) if n == 128 else (20, 80)
                t_drt = per_move(oracle.sat_drt_run, *m_drt)
                t_pila = per_move(oracle.sat_run, 2000, 42000)
                row["cpu_one_thread"] = {"pila_s_per_move": t_pila, "drt_s_per_move": t_drt,
                                         "speedup": t_drt / t_pila, "note": "oracle FP64, single thread"}
            rows.append(row)
    out = {"metric": "SAT moves/s with the PILA over SAT with a full DRT per move", "unit": "ratio",
           "higher_is_better": True, "data": "synthetic",
           "config": {"workload": "drt", "moves": M, "stages": 1, "bome_k": 1, "pila": "f32",
                      "drt": "bilinear interpolation, B unit steps per ray"},
           "rows": rows}
    print(json.dumps(out))


def _timed_call(fn, reps, flush):
    """Mean ms of fn() over reps calls, CUDA events on the current stream, L2
    flushed (256 MB write) before each; one untimed call first."""
    import torch

    stream = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.mean(ts)


def run_rows(args):
    """The steps of the path besides the move, each timed alone through its
    C-ABI call (inputs resident in HBM, L2 flushed before each call), with the
    algorithmic bytes each must move against the measured HBM copy bandwidth:
      a0 PILA build: the table, the per-pixel sums and the band written once;
      a7 forward projection (the resync): the table read once, the images read
         and the FP64 projections written;
      a9 SIRT, simultaneous: per iteration the table read twice (forward and
         back projection) plus the sinogram, the factor matrix, the correction
         and the image;
      one 256^2 chain (K = 8) and one 512^2 chain (360 angles, K = 8, FP16
         table): a single chain is sequential, so each is reported as time per
         stage (a sweep of every reconstruction-space pixel) and moves/s."""
    import torch

    from paper_1411_4622_gb300 import api
    from paper_1411_4622_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    peak, peak_kind = peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    reps = max(1, args.steps)
    rows = []

    def add(row, cfg, ms, algo_bytes, unit_count=None, unit=None):
        gbs = algo_bytes / (ms / 1e3) / 1e9
        r = {"row": row, "config": cfg, "ms": ms, "algorithmic_bytes": algo_bytes, "achieved_gbs": gbs,
             "peak_gbs": peak, "frac": gbs / peak}
        if unit_count is not None:
            r["rate"] = unit_count / (ms / 1e3)
            r["rate_unit"] = unit
        rows.append(r)

    geoms = {"batch128x512": (128, 120, 181, 512), "precision512": (512, 360, 725, 304)}
    for name, (n, U, B, C) in geoms.items():
        C = args.slices or C
        mask = synth.disk_mask(n)
        holder = {}

        def build():
            if "p" in holder:
                api.pila_free(holder.pop("p"))
            holder["p"] = api.pila_build(n, U, B, api.PILA_F16, mask=mask)

        ms = _timed_call(build, reps, flush)
        info = api.pila_info(holder["p"])
        P = n * n
        table = info["table_bytes"]
        add("a0 PILA build (FP16)", f"{name}: {n}^2, {U} angles, {B} bins", ms, table + 4 * P,
            P * U, "records/s")
        ph = np.stack([synth.phantom(n, 20, synth.slice_seeds(i)[0]) * mask for i in range(8)])
        imgs = torch.tensor(ph[np.arange(C) % 8], dtype=torch.float32, device="cuda").contiguous()
        out = torch.empty((C, U, B), dtype=torch.float64, device="cuda")
        ms = _timed_call(lambda: api.pila_forward(holder["p"], imgs, out=out), reps, flush)
        terms = C * info["entries"]
        add("a7 forward projection (FP16 table, exact fixed-point sums)", f"{name}: {C} images", ms,
            table + C * (4 * P + 8 * U * B), terms, "terms/s")
        api.pila_free(holder.pop("p"))
        del imgs, out

    # a9 SIRT and one chain at 256^2, 180 angles, 363 bins (the SAT+SIRT configuration)
    cfg = synth.WORKLOADS["sat256"]
    n, U, B = cfg["n"], cfg["n_angles"], cfg["n_bins"]
    mask = synth.disk_mask(n)
    ph = synth.phantom(n, cfg["ellipses"], synth.slice_seeds(0)[0]) * mask
    pf = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    clean = api.pila_forward(pf, torch.tensor(ph[None], dtype=torch.float32, device="cuda")).cpu().numpy()[0]
    sino = torch.tensor(synth.gaussian_noise(clean, cfg["noise"][1], synth.slice_seeds(0)[1])[None],
                        dtype=torch.float32, device="cuda").contiguous()
    init = torch.tensor(synth.initial_image(n, 0.5, mask)[None], dtype=torch.float32, device="cuda")
    iters = cfg["sirt_iters"]
    sirt = {}
    for prec, label in ((api.PILA_F32, "FP32"), (api.PILA_F16, "FP16")):
        p = pf if prec == api.PILA_F32 else api.pila_build(n, U, B, prec, mask=mask)
        info = api.pila_info(p)
        img = init.clone()
        api.sirt_run(p, sino, img, n_iter=1)  # the factor matrix, cached with the table
        ms = _timed_call(lambda: (img.copy_(init), api.sirt_run(p, sino, img, n_iter=iters)), reps, flush)
        table = info["table_bytes"]
        per_iter = 2 * table + U * B * (4 + 4 + 4) + 8 * n * n
        add(f"a9 SIRT, simultaneous ({label} table)", f"sat256: {n}^2, {U} angles, {B} bins, {iters} iterations",
            ms, iters * per_iter, iters, "iterations/s")
        sirt[label] = iters / (ms / 1e3)
        if p is not pf:
            api.pila_free(p)
    stages = args.sweeps or 10
    p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
    img = init.clone()
    kw = dict(bome_k=cfg["bome_k"], n_sweeps=stages, t0=-1.0, tn=-1.0, seed=synth.slice_seeds(0)[2],
              flags=api.SAT_FLAG_AUTOTUNE)
    st = api.sat_run(p, sino, img, **kw)
    M = int(mask.sum())
    chain = {"stages": stages, "moves_per_stage": M, "sweep_ms": st[0]["sweep_ms"],
             "ms_per_stage": st[0]["sweep_ms"] / stages, "moves_per_s": stages * M / (st[0]["sweep_ms"] / 1e3),
             "launch": launch_name(st[0]["plan"], kw["flags"]), "bome_k": cfg["bome_k"], "pila": "f16"}
    api.pila_free(p)
    api.pila_free(pf)
    chain512 = single_chain_512(api, stages=2)
    out = {"metric": "SIRT-PILA iterations/s, 256x256 slice (180 angles, FP32 table)", "value": sirt["FP32"],
           "unit": "iterations/s", "n_gpus": 1, "steps": reps, "warmup": 1, "ms_per_step": 1e3 / sirt["FP32"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "rows", "l2": "flushed before each timed call (256 MB write)",
                      "peak_kind": peak_kind},
           "rows": rows, "chain256": chain, "chain512": chain512}
    print(json.dumps(out))


def single_chain_512(api, stages):
    """One chain of the 512^2 configuration (360 angles, K = 8, FP16 table,
    Poisson noise, resync every stage) on the 4-warp windowed layout, the
    autotuner's pick for one chain of this table: time per stage."""
    import torch

    c4 = synth.WORKLOADS["precision512"]
    n4, U4, B4, K4 = c4["n"], c4["n_angles"], c4["n_bins"], c4["bome_k"]
    mask4 = synth.disk_mask(n4)
    ph4 = synth.phantom(n4, c4["ellipses"], synth.slice_seeds(0)[0]) * mask4
    pf4 = api.pila_build(n4, U4, B4, api.PILA_F32, mask=mask4)
    clean4 = api.pila_forward(pf4, torch.tensor(ph4[None], dtype=torch.float32, device="cuda")).cpu().numpy()[0]
    sino4 = torch.tensor(synth.poisson_noise(clean4, c4["noise"][1], synth.slice_seeds(0)[1])[None],
                         dtype=torch.float32, device="cuda").contiguous()
    api.pila_free(pf4)
    p4 = api.pila_build(n4, U4, B4, api.PILA_F16, mask=mask4)
    st4 = api.sat_run(p4, sino4, torch.tensor(synth.initial_image(n4, 0.5, mask4)[None], dtype=torch.float32,
                                              device="cuda"),
                      bome_k=K4, n_sweeps=stages, t0=-1.0, tn=-1.0, seed=synth.slice_seeds(0)[2], resync_every=1,
                      plan=api.SAT_PLAN_WINDOW_G4)
    api.pila_free(p4)
    M4 = int(mask4.sum())
    return {"stages": stages, "moves_per_stage": M4, "sweep_ms": st4[0]["sweep_ms"],
            "ms_per_stage": st4[0]["sweep_ms"] / stages, "moves_per_s": stages * M4 / (st4[0]["sweep_ms"] / 1e3),
            "us_per_move": st4[0]["sweep_ms"] * 1e3 / (stages * M4), "launch": launch_name(st4[0]["plan"], 0, 8),
            "bome_k": K4, "pila": "f16", "resync_every": 1}


def run_chain512(args):
    """--workload chain512: one chain of the 512^2 configuration alone (a single
    chain is sequential: reported as time per stage); one JSON line."""
    import torch

    from paper_1411_4622_gb300 import api
    from paper_1411_4622_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    c = single_chain_512(api, stages=args.sweeps or 2)
    out = {"metric": "SAT ms per stage, one 512x512 chain (360 angles, K = 8)", "value": c["ms_per_stage"],
           "unit": "ms/stage", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": c["sweep_ms"],
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "chain512"}, "chain512": c}
    print(json.dumps(out))


def run_fbp(args):
    """Fig. 9 on synthetic phantoms: 16 slices of 128x128 whose ellipses sit
    off the centre of rotation, noiseless; FBP (Ram-Lak) at 90 and 200
    angles; SAT at 90 angles with the spatial constraint (FBP thresholded at
    10% of its maximum, FBP start image, beta = FBP maximum) and without it
    (every pixel, uniform 0.5 start, beta = 1); 8 estimates, 100 stages,
    T0 by Eq. (8).  Reported: mean NRMSE (RMS error over the phantom's mean)."""
    import torch

    from paper_1411_4622_gb300 import api
    from paper_1411_4622_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    n, C, S, K = 128, args.slices or 16, args.sweeps or 100, 8
    ph = []
    for i in range(C):
        base = synth.phantom(n, 10, synth.slice_seeds(i)[0]) * synth.disk_mask(n, 0.3 * n)
        shifted = np.zeros_like(base)
        shifted[n // 6:, n // 5:] = base[: n - n // 6, : n - n // 5]  # off the centre of rotation
        ph.append(shifted)
    ph = np.stack(ph)
    out = {}
    sinos = {}
    for U in (90, 200):
        B = synth.bins_for(n)
        pf = api.pila_build(n, U, B, api.PILA_F32)
        sinos[U] = api.pila_forward(pf, torch.tensor(ph, dtype=torch.float32, device="cuda")).float().contiguous()
        api.pila_free(pf)
        rec = api.fbp(sinos[U], n).cpu().numpy()
        out[f"fbp_U{U}"] = float(np.mean([nrmse(rec[i], ph[i]) for i in range(C)]))
    U, B = 90, synth.bins_for(n)
    rec = api.fbp(sinos[U], n)
    init, mask, beta = api.fbp_prior(rec, 0.1)
    masks, inits = mask.cpu().numpy(), init
    constrained = []
    for i in range(C):
        p = api.pila_build(n, U, B, api.PILA_F16, mask=masks[i])
        img = inits[i:i + 1].clone()
        api.sat_run(p, sinos[U][i:i + 1], img, bome_k=K, n_sweeps=S, beta=float(beta[i]), t0=-1.0, tn=-1.0,
                    seed=synth.slice_seeds(i)[2])
        constrained.append(nrmse(img.cpu().numpy()[0], ph[i]))
        api.pila_free(p)
    out["sat_U90_constrained"] = float(np.mean(constrained))
    p = api.pila_build(n, U, B, api.PILA_F16)
    img = torch.full((C, n, n), 0.5, dtype=torch.float32, device="cuda")
    api.sat_run(p, sinos[U], img, bome_k=K, n_sweeps=S, beta=1.0, t0=-1.0, tn=-1.0, seed=synth.slice_seeds(0)[2])
    api.pila_free(p)
    img = img.cpu().numpy()
    out["sat_U90_unconstrained"] = float(np.mean([nrmse(img[i], ph[i]) for i in range(C)]))
    print(json.dumps({"metric": "mean NRMSE", "unit": "nrmse", "higher_is_better": False, "data": "synthetic",
                      "config": {"workload": "fbp", "n": n, "slices": C, "stages": S, "bome_k": K,
                                 "mask_threshold": 0.1, "filter": "Ram-Lak"}, "results": out}))


def main():
    args = parse()
    # one hardware work queue per stream for up to 32 streams (the serving
    # engine runs each image size's shared launches, and any class outside
    # them, on a stream of its own); read when the CUDA context is created,
    # so set before the first CUDA call
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    if args.workload == "precision512":
        return run_precision(args)
    if args.workload == "precision512-rmse":
        return run_precision_rmse(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "chain512":
        return run_chain512(args)
    if args.workload == "bome":
        return run_bome(args)
    if args.workload == "drt":
        return run_drt(args)
    if args.workload == "fbp":
        return run_fbp(args)
    if args.workload == "rows":
        return run_rows(args)
    cfg = workload(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, cfg)
        return
    import torch

    from paper_1411_4622_gb300 import api
    from paper_1411_4622_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pk = measure_peaks(api)
    n, U, B, K, S = cfg["n"], cfg["n_angles"], cfg["n_bins"], cfg["bome_k"], cfg["n_sweeps"]
    first, slices = shard.slice_range(rank, cfg["slices"])
    phantoms, mask = make_slices(cfg, first, slices)
    P = n * n

    # Inputs: sinograms from the phantoms through an FP32 PILA (FP64-grade projection).
    pf = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    sino = api.pila_forward(pf, torch.tensor(phantoms, dtype=torch.float32, device="cuda")).float().contiguous()
    init = torch.tensor(np.stack([synth.initial_image(n, 0.5, mask)] * slices), dtype=torch.float32,
                        device="cuda")
    images = init.clone()
    seed0 = synth.slice_seeds(first)[2]  # chain c uses seed0 + c: global slice numbering
    run_kw = dict(bome_k=K, n_sweeps=S, t0=cfg["t0"], tn=cfg["tn"], beta=cfg["beta"], seed=seed0, resync_every=0,
                  residency=args.residency, group_warps=args.group_warps, flags=args.flags, plan=args.plan)
    stream = torch.cuda.current_stream()
    info = {}

    prec = {"f16": api.PILA_F16, "u8": api.PILA_U8, "f32": api.PILA_F32}[args.pila]

    def step():
        images.copy_(init)
        p = api.pila_build(n, U, B, prec, mask=mask)
        st = api.sat_run(p, sino, images, **run_kw)
        if not info:
            info.update(api.pila_info(p))
        api.pila_free(p)
        return st

    step_ms, stats, clk = timed_steps(args, step, stream, dist, local)
    st = stats[-1]
    sweep_ms = [x[0]["sweep_ms"] for x in stats]
    ms = shard.max_over_ranks(statistics.mean(step_ms), dist, device="cuda")
    M = int(mask.sum())
    moves_per_step = slices * S * M
    value = shard.weak_rate(world, moves_per_step, ms)
    acc = sum(s["accepted"] for s in st) / max(1, sum(s["proposed"] for s in st))
    final = images.cpu().numpy()
    rmse_batched = np.array([synth.rmse(final[i], phantoms[i], mask) for i in range(slices)])

    # Plain form: single chain at a time, FP32 PILA, on a sample of the same slices.
    plain_n = min(4, slices)
    plain_imgs, plain_ms = [], 0.0
    for i in range(plain_n):
        im = init[i:i + 1].clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kw = dict(run_kw)
        kw["seed"] = seed0 + i
        e0.record(stream)
        api.sat_run(pf, sino[i:i + 1], im, **kw)
        e1.record(stream)
        e1.synchronize()
        plain_ms += e0.elapsed_time(e1)
        plain_imgs.append(im.cpu().numpy()[0])
    rmse_plain = np.array([synth.rmse(plain_imgs[i], phantoms[i], mask) for i in range(plain_n)])
    plain = {"value": plain_n * S * M / (plain_ms / 1e3), "unit": UNIT, "slices": plain_n, "precision": "f32",
             "rmse_rel_diff_max": float(np.max(np.abs(rmse_batched[:plain_n] - rmse_plain) / rmse_plain))}

    # End to end through the C-ABI with host (pinned) buffers.
    sino_h = sino.cpu().pin_memory()
    img_h = init.cpu().pin_memory()
    e2e_ms = []
    for it in range(3):  # the first call is a warm-up
        work = img_h.clone().pin_memory()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        p = api.pila_build(n, U, B, prec, mask=mask)
        api.sat_run(p, sino_h, work, **run_kw)
        api.pila_free(p)
        if it > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t))
    e2e_t = shard.max_over_ranks(statistics.mean(e2e_ms), dist, device="cuda")
    e2e = {"value": shard.weak_rate(world, moves_per_step, e2e_t), "unit": UNIT,
           "h2d_bytes_per_step": int(sino_h.numel() * 4 + img_h.numel() * 4),
           "d2h_bytes_per_step": int(img_h.numel() * 4)}

    # Roofline of the sweep kernel: each class of its algorithmic bytes per
    # move against the measured rate of the level it is read from.  The PILA
    # row (consecutive 16-byte chunks) comes from L2 when the table fits there
    # (from HBM otherwise); the residual cells come from shared memory (the
    # windowed band) as scattered 4-byte words, or else as 32-byte sectors
    # from L2; the image words from L2.  The bound is the level with the
    # largest fraction; the issue rate is reported beside it (the move is a
    # sequential chain: one warp per scheduler).
    E = info["entries"] / P
    sweep_s = statistics.mean(sweep_ms) / 1e3
    rate = moves_per_step / sweep_s
    row_bytes = info["row_records"] * info["record_bytes"]
    resid_bytes = 4 * E * (1 + acc)
    img_bytes = 4 * (1 + acc)
    kernel = PLAN_KERNEL.get(st[0]["plan"], "sat_window_kernel")
    smem_resid = st[0]["plan"] in (1, 3, 9, 10)
    table_in_l2 = info["table_bytes"] < 64e6
    levels = {
        "table_rows": {"level": "l2" if table_in_l2 else "hbm", "bytes_per_move": row_bytes,
                       "achieved": row_bytes * rate / 1e9,
                       "peak": pk["l2_stream_gbs"] if table_in_l2 else pk["hbm_stream_gbs"], "pattern": "stream"},
        "residual": ({"level": "smem", "bytes_per_move": resid_bytes, "achieved": resid_bytes * rate / 1e9,
                      "peak": pk["smem_random_gbs"], "pattern": "scattered 4-byte words"} if smem_resid else
                     {"level": "l2", "bytes_per_move": 32 * E * (1 + acc),
                      "achieved": 32 * E * (1 + acc) * rate / 1e9, "peak": pk["l2_sector_gbs"],
                      "pattern": "32-byte sectors"}),
        "image": {"level": "l2", "bytes_per_move": 32 * (1 + acc), "achieved": 32 * (1 + acc) * rate / 1e9,
                  "peak": pk["l2_sector_gbs"], "pattern": "32-byte sectors"},
    }
    for v in levels.values():
        v["frac"] = v["achieved"] / v["peak"]
    top = max(levels, key=lambda k: levels[k]["frac"])
    tpm = stored_traffic(kernel)
    ipm = stored_profile(kernel, WORKLOAD, "inst_per_move")
    ipk, sms, mhz = issue_peak(clk)
    roof = {"bound": levels[top]["level"], "achieved": levels[top]["achieved"], "peak": levels[top]["peak"],
            "unit": "GB/s", "frac": levels[top]["frac"], "bytes": top,
            "traffic": (tpm * moves_per_step) if tpm is not None else None,
            "peak_kind": "measured (satpila_probe_*, this run)", "kernel": kernel,
            "bytes_per_move": row_bytes + resid_bytes + img_bytes, "sweep_ms": sweep_s * 1e3,
            "launches_per_step": 1, "levels": levels,
            "issue": {"inst_per_move": ipm, "achieved": ipm * rate if ipm else None, "peak": ipk,
                      "unit": "warp instructions/s", "frac": ipm * rate / ipk if ipm else None,
                      "peak_rule": f"{sms} SMs x 4 schedulers x {mhz:.0f} MHz, one instruction per cycle each",
                      "note": "one warp per chain and 3-4 chains per SM: at most one warp per scheduler, so "
                              "dependent instructions are not hidden (latency-bound)"}}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "slices_per_gpu": slices, "n": n, "angles": U, "bins": B,
                      "bome_k": K, "stages": S, "moves_per_stage": M, "pila": args.pila,
                      "l2": "flushed between timed steps (256 MB write)",
                      "launch": launch_name(st[0]["plan"], args.flags, args.plan), "graph": True},
           "evaluations_per_s": value * K, "acceptance": acc,
           "rmse": {"batched_mean": float(rmse_batched.mean())}, "plain": plain,
           "latency_ms": {"slice_p50": float(np.percentile(step_ms, 50)),
                          "slice_p99": float(np.percentile(step_ms, 99)),
                          "note": "every slice of a step completes with the step's one launch"},
           "e2e": e2e, "roofline": roof, "peaks": pk, "clocks": clk,
           "parity": {"per_move_dS": "within 1e-5 of the magnitude of its terms, 2|df| sum|r l| + df^2 sum l^2 "
                                     "(a difference of FP32 sums is bounded relative to its terms, not to itself)",
                      "decisions": "identical to the FP64 oracle's except recorded near-ties (margin below 2e-5 "
                                   "of the term scale)",
                      "full_size_test": "tests/test_gpu_parity.py::test_batched_workload_full_size_sampled_chains "
                                        "follows a sampled chain of this launch over all 644,600 moves",
                      "final_rmse_vs_plain_fp32": plain["rmse_rel_diff_max"]},
           # per step: PILA records, per-pixel sums, residual band, 2 resync
           # projections, 2 reductions, Eq. (8), the sweep between two timer
           # stamps, one copy (the sat_run part as one CUDA graph)
           "gpu_launches": args.steps * (1 + 1 + 1 + 2 + 2 + 1 + 3 + 1)}
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(cfg)
    # the other two configurations measured beside the headline (rank 0 only)
    if world == 1 and not args.no_c4:
        out["precision512"] = precision_sample(pk)
    if world == 1 and not args.no_serve:
        r = serve_stream(args.serve_requests, args.serve_rate)
        out["serve"] = dict(r, metric="SAT pixel-moves/s over a served request stream; request p50/p99 ms")
    api.pila_free(pf)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
