"""The DRAM-traffic records the bench line cites (profiles/traffic.json): each is
keyed by kernel, grid and z-chunk, carries the grid of blocks ncu saw and the
hash of the kernel source it was captured from, and the bench uses it only for
the same source and the same launch shape (one block per 32 x 8 column tile and
z-chunk).  Checked on the CPU: no GPU, no capture."""
import json
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _records():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        return json.load(f)


def test_march_ctas():
    import bench
    assert bench.march_ctas((256, 96, 96), 32) == 8 * 12 * 3
    assert bench.march_ctas((256, 96, 96), 24) == 8 * 12 * 4
    assert bench.march_ctas((512, 512, 512), 96) == 16 * 64 * 6
    assert bench.march_ctas((70, 19, 13), 5) == 3 * 3 * 3          # ragged tiles and chunks
    assert bench.march_ctas((64, 16, 14), None) == 2 * 2 * 1       # no chunking: one per column


@pytest.mark.parametrize("key", sorted(_records()))
def test_record_matches_its_launch_shape(key):
    """Every committed record's grid is the grid the bench computes for its key."""
    import bench
    rec = _records()[key]
    m = re.fullmatch(r"(k_\w+_ws)_(\d+)x(\d+)x(\d+)_z(\d+)", key)
    assert m, key
    dims, zc = tuple(int(v) for v in m.group(2, 3, 4)), int(m.group(5))
    assert rec["grid_ctas"] == f"({bench.march_ctas(dims, zc)}, 1, 1)"
    assert rec["dram_bytes_per_launch"] > 0 and len(rec["launches"]) >= 2


def test_record_is_used_only_for_the_same_source_and_grid():
    import bench
    recs = _records()
    key = sorted(recs)[0]
    m = re.fullmatch(r"(k_\w+_ws)_(\d+)x(\d+)x(\d+)_z(\d+)", key)
    dims, zc = tuple(int(v) for v in m.group(2, 3, 4)), int(m.group(5))
    ctas = bench.march_ctas(dims, zc)
    got = bench.recorded_traffic(key, ctas)
    src = os.path.join(ROOT, "paper_2607_07687_gb300", "csrc", "gmg_kernels.cu")
    import hashlib
    current = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if recs[key]["source_sha256"] == current:
        assert got == recs[key]["dram_bytes_per_launch"]
    else:
        assert got is None                       # captured from other kernel source: not cited
    assert bench.recorded_traffic(key, ctas + 1) is None            # another launch shape
    assert bench.recorded_traffic("k_sweep_ws_1x1x1_z1", 1) is None  # no record
