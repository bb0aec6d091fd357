"""The multi-GPU layout on CPU ranks (gloo, world size 2): each rank anneals
its own slices with the FP64 oracle, no data is exchanged, and the union of
the ranks' results equals one process running every slice; the step time
that is reported is the slowest rank's."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_1411_4622_gb300 import shard, synth  # noqa: E402

N, U, PER_RANK, STAGES, K = 16, 12, 3, 2, 4


def _slice(idx):
    B = synth.bins_for(N)
    mask = synth.disk_mask(N)
    ph = synth.phantom(N, 4, synth.slice_seeds(idx)[0]) * mask
    pm = oracle.drt(ph, U, B)
    img, st, _ = oracle.sat_run(pm, synth.initial_image(N, 0.5, mask), n_sweeps=STAGES, bome_k=K, mask=mask,
                                seed=synth.slice_seeds(idx)[2])
    return img, st["accepted"]


def _worker(rank, world, port, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = shard.slice_range(rank, PER_RANK)
    mine = [_slice(first + i) for i in range(count)]
    # the step time each rank reports; the job's is the maximum
    t = shard.max_over_ranks(10.0 + rank, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, (first, mine))
    if rank == 0:
        out_q.put((t, gathered))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_shard_slices_without_exchange():
    oracle.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    t, gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 11.0
    assert shard.weak_rate(world, 1000, 500.0) == 4000.0
    got = {}
    for first, res in gathered:
        for i, r in enumerate(res):
            got[first + i] = r
    assert sorted(got) == list(range(world * PER_RANK))
    for idx in range(world * PER_RANK):
        img, acc = _slice(idx)
        assert np.array_equal(got[idx][0], img) and got[idx][1] == acc
