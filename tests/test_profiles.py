"""The committed profiles stand for the current kernels: the counter files that
bench.py reads (DRAM bytes, warp instructions, FP64 flops) and every ncu summary
name the hash of the pass kernels' sources they were taken on, and that hash
must be the current one (bench.kernel_source_hash)."""
import glob
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_counter_files_match_the_kernel_sources():
    h = bench.kernel_source_hash()
    for name in ("pass_traffic_256cubed_fp32_16chains.json", "fp64_flops_256cubed_1chain.json"):
        with open(os.path.join(ROOT, "profiles", name)) as f:
            assert json.load(f)["source_hash"] == h, name


def test_summaries_name_the_current_hash():
    h = bench.kernel_source_hash()
    for fn in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(fn) as f:
            assert h in f.read(), os.path.basename(fn)
