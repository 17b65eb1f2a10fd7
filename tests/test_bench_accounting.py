"""Host-side accounting of bench.py that feeds its reported numbers (CPU only): the launch count
per frame, the span count behind the tile lists, the binning's algorithmic bytes and the L2
flush."""
from __future__ import annotations

import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_launches_per_frame_span_path():
    # 800x800: slice_project, clear, depth keys, 4 depth passes, span walk, 1 row pass (50 tile
    # rows: a 6-bit digit), column counts, expansion, render
    assert bench.launches_per_frame(300_000, 5_000_000, 800, 800) == 12
    # 1920x1080 (120 x 68 tiles): still the span path, one row pass
    assert bench.launches_per_frame(1_500_000, 10_000_000, 1920, 1080) == 12
    # 4096 x 4096 (256 tiles per side, the span path's limit): 8-bit rows, one pass
    assert bench.launches_per_frame(10_000, 100_000, 4096, 4096) == 12


def test_launches_per_frame_instance_path():
    # 5000 x 5000: 313 tiles per side, the instance path: walk count, one scan kernel (up to
    # 11264 warps), emit, ceil(17 / 8) = 3 tile passes (97969 tiles), ranges, render
    assert bench.launches_per_frame(300_000, 5_000_000, 5000, 5000) == 7 + 1 + 1 + 1 + 3 + 1 + 1
    # more than 11264 warps of Gaussians: a three-kernel scan
    assert bench.launches_per_frame(11264 * 32 + 1, 5_000_000, 5000, 5000) == 7 + 1 + 3 + 1 + 3 + 1 + 1


class _Bins:
    def __init__(self, point_list, ranges):
        self.point_list = torch.tensor(point_list, dtype=torch.int32)
        self.ranges = torch.tensor(ranges, dtype=torch.int32)


def test_count_spans_counts_gaussian_tile_row_pairs():
    # a 3 x 2 tile grid; Gaussian 7 covers tiles 0, 1 (row 0) and 3, 4, 5 (row 1): 2 spans;
    # Gaussian 9 covers tile 2 (row 0): 1 span; Gaussian 4 covers tiles 4 and 5 (row 1): 1 span
    lists = {0: [7], 1: [7], 2: [9], 3: [7], 4: [4, 7], 5: [4, 7]}
    point_list, ranges, pos = [], [], 0
    for t in range(6):
        ranges.append([pos, pos + len(lists[t])])
        point_list += lists[t]
        pos += len(lists[t])
    bins = _Bins(point_list, ranges)
    assert bench.count_spans(bins, len(point_list), tiles_x=3) == 4


def test_binning_bytes_adds_up_its_kernels():
    b = bench.binning_bytes(n=1000, k=5000, spans=1200, visible=600)
    assert b["total"] == sum(b["per_kernel"].values())
    assert b["per_kernel"]["depth_passes"] == 4 * 16 * 1000
    assert b["per_kernel"]["span_expand"] == 8 * 1200 + 4 * 5000


def test_l2_flush_writes_one_buffer_and_reads_another():
    f = bench.L2Flush(torch.device("cpu"))
    assert f.w.numel() == bench.L2_FLUSH_BYTES and f.r.numel() * 4 == bench.L2_FLUSH_BYTES
    assert f.w.data_ptr() != f.r.data_ptr()
    f.w.fill_(1)
    f()
    assert int(f.w.max()) == 0 and float(f.out) == 0.0
