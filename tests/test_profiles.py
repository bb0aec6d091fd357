"""The per-move figures bench.py reads from profiles/ (DRAM bytes and warp
instructions per move of the sweep kernels it reports) belong to the current
kernel sources: each summary's source hash equals the hash of those sources,
so the bench line carries the figures instead of nulls."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_profile_figures_match_current_sources():
    for kernel, workload, keys in (("sat_window_kernel", "batch128x512", ("dram_bytes_per_move", "inst_per_move")),
                                   ("sat_window_group_kernel", "precision512", ("dram_bytes_per_move",))):
        for key in keys:
            v = bench.stored_profile(kernel, workload, key)
            assert v is not None and v > 0, (kernel, key)
