"""Host-side helpers of bench.py (no GPU): the reading of the batched autotuner's tune cache
and the per-step work counts the rooflines divide by."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_read_tuning_decodes_family_and_grid(tmp_path):
    p = tmp_path / "tune.txt"
    p.write_text("f64:n16:g:m16 72\nf32:n32:g:m32 32\nf32:n4:s:m4 8\n")
    t = bench.read_tuning(str(p))
    assert t["f64:n16:g:m16"] == {"level_kernel_family": 1, "blocks_per_sm": 8}
    assert t["f32:n32:g:m32"] == {"level_kernel_family": 0, "blocks_per_sm": 32}
    assert t["f32:n4:s:m4"] == {"level_kernel_family": 0, "blocks_per_sm": 8}


def test_read_tuning_without_cache_is_empty(tmp_path):
    assert bench.read_tuning(str(tmp_path / "missing.txt")) == {}


def test_level_flops_lead_with_18_n_cubed():
    # the level phase is three n x n QRs of a triangle over a full block plus their companions
    # (n + 1, 2n + 1 and 1 columns): 18 n^3 flops per step to leading order, the lower-order
    # terms adding a share that shrinks with n
    ratios = [bench.flops_per_step(n, n, "fp64")["level"] / n ** 3 for n in (6, 48, 128, 512)]
    assert all(a > b for a, b in zip(ratios, ratios[1:])), ratios
    assert abs(ratios[-1] - 18.0) < 0.1, ratios
