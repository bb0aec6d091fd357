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
    ap.add_argument("--flags", type=int, default=0, help="SAT_FLAG_* bits for the batched run")
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


def kernel_source_hash():
    """Hash of the CUDA sources; a stored DRAM-traffic figure only applies to them."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1411_4622_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(f.encode())
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def stored_traffic(kernel):
    """DRAM bytes per move of `kernel` from the committed ncu summary, or None
    when the summary is missing or was taken on different sources."""
    path = os.path.join(ROOT, "profiles", f"{kernel}__{WORKLOAD}.md")
    try:
        kv = {}
        for ln in open(path):
            if ":" in ln and ln.startswith("- "):
                k, v = ln[2:].split(":", 1)
                kv[k.strip()] = v.strip().strip("`")
        if kv.get("source_sha") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_move"])
    except (OSError, KeyError, ValueError):
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


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

    def run(self, stages):
        """All workers run their slice for `stages` stages; (moves, wall s)."""
        jobs = [(self.cfg, i, stages) for i in range(self.procs)]
        t = time.perf_counter()
        res = self.pool.map(_oracle_slice, jobs, chunksize=1)
        return sum(r[0] for r in res), time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_stages_for(cfg, budget_s):
    """Stages of one slice that take the oracle about budget_s on one core:
    per-stage time from a 1-stage and a 3-stage run (setup cancels)."""
    t1 = _oracle_slice((cfg, 0, 1))[1]
    t3 = _oracle_slice((cfg, 0, 3))[1]
    per = max((t3 - t1) / 2.0, 1e-4)
    return int(max(1, min(cfg["n_sweeps"] * 4, budget_s / per)))


def cpu_baseline(cfg, budget_s=12.0):
    """The FP64 oracle as it stands (single-threaded per process), one process
    per host core, each on its own slice of the workload for about budget_s."""
    stages = oracle_stages_for(cfg, budget_s)
    pool = OraclePool(cfg)
    try:
        moves, wall = pool.run(stages)
    finally:
        pool.close()
    return {"value": moves / wall, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
            "sample": f"{pool.procs} slices of {WORKLOAD} (one per process), {stages} stages x "
                      f"{moves // max(1, stages * pool.procs)} moves each, K={cfg['bome_k']}, FP64, "
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


def main():
    args = parse()
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
                  residency=args.residency, group_warps=args.group_warps, flags=args.flags)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    info = {}

    def step():
        images.copy_(init)
        p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
        st = api.sat_run(p, sino, images, **run_kw)
        if not info:
            info.update(api.pila_info(p))
        api.pila_free(p)
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, sweep_ms = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1.0)  # evict L2 between timed steps (outside the events)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        sweep_ms.append(st[0]["sweep_ms"])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
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
        p = api.pila_build(n, U, B, api.PILA_F16, mask=mask)
        api.sat_run(p, sino_h, work, **run_kw)
        api.pila_free(p)
        if it > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t))
    e2e_t = shard.max_over_ranks(statistics.mean(e2e_ms), dist, device="cuda")
    e2e = {"value": shard.weak_rate(world, moves_per_step, e2e_t), "unit": UNIT,
           "h2d_bytes_per_step": int(sino_h.numel() * 4 + img_h.numel() * 4),
           "d2h_bytes_per_step": int(img_h.numel() * 4)}

    # Roofline of the sweep kernel (algorithmic bytes per move).
    peak, peak_kind = peaks()
    E = info["entries"] / P
    bytes_per_move = info["row_records"] * info["record_bytes"] + 4 * E * (1 + acc) + 4 * (1 + acc)
    achieved = bytes_per_move * moves_per_step / (statistics.mean(sweep_ms) / 1e3) / 1e9
    kernel = "sat_window_kernel"
    tpm = stored_traffic(kernel)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": (tpm * moves_per_step) if tpm is not None else None, "peak_kind": peak_kind,
            "kernel": kernel, "bytes_per_move": bytes_per_move, "sweep_ms": statistics.mean(sweep_ms),
            "launches_per_step": 1}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "slices_per_gpu": slices, "n": n, "angles": U, "bins": B,
                      "bome_k": K, "stages": S, "moves_per_stage": M, "pila": "f16",
                      "l2": "flushed between timed steps (256 MB write)"},
           "evaluations_per_s": value * K, "acceptance": acc,
           "rmse": {"batched_mean": float(rmse_batched.mean())}, "plain": plain,
           "latency_ms": {"slice_p50": float(np.percentile(step_ms, 50)),
                          "slice_p99": float(np.percentile(step_ms, 99)),
                          "note": "every slice of a step completes with the step's one launch"},
           "e2e": e2e, "roofline": roof, "clocks": clk,
           # per step: PILA records, per-pixel sums, residual band, 2 resync
           # projections, 2 reductions, Eq. (8), the sweep between two timer
           # stamps, one copy (the sat_run part as one CUDA graph)
           "gpu_launches": args.steps * (1 + 1 + 1 + 2 + 2 + 1 + 3 + 1)}
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(cfg)
    api.pila_free(pf)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
