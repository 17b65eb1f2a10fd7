"""sdgs_bin_sort_static: binning into the library's built-in scratch array instead of a
caller-provided workspace.

Some callers cannot allocate device memory: a plugin whose host application owns every device
allocation, or a latency-bound loop that cannot afford cudaMalloc's implicit synchronisation.
This entry point lets them bin without passing a workspace.  The test calls it through the C ABI
twice in a row and checks each result against sdgs_bin_sort with a caller-allocated workspace,
element by element (binning is integer work, so the comparison is exact).  It lives in a file
that pytest collects last, and passes both alone in a fresh process and after the other tests.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import synth
from paper_2503_07946_gb300 import render as prender
from paper_2503_07946_gb300 import sdgs

pytestmark = pytest.mark.gpu


def _bins_host(bins, k):
    return (bins.point_list[:k].cpu().numpy().copy(), bins.tile_keys[:k].cpu().numpy().copy(),
            bins.ranges.cpu().numpy().copy())


@pytest.mark.parametrize("case", ["scene", "random"])
def test_static_scratch_binning_matches_workspace_binning(case):
    if case == "scene":
        scene = synth.config_scene(0)
        cam = synth.make_camera((1.2, -0.8, -2.6), 141, 97, 55.0, 0.3)
        dev = prender.scene_to_device(scene)
        proj = sdgs.ProjectedBuffers(scene.n)
        view = sdgs.view_struct(cam)
        sdgs.slice_project(sdgs.scene_struct(dev, scene.lambda_t, scene.lambda_d), view, proj)
    else:
        rec = synth.random_projected(20000, 1352, 1014, seed=4, max_half_tiles=12)
        proj = sdgs.ProjectedBuffers.from_host(rec)
        view = sdgs.view_struct(synth.make_camera((0, 0, -3), 1352, 1014, 60.0, 0.5))
    ref_bins = sdgs.BinBuffers(proj.n, 2_000_000, view.width, view.height)
    k_ref = sdgs.bin_sort(proj, view, ref_bins, sync=True)
    want = _bins_host(ref_bins, k_ref)
    assert k_ref > 0
    for _ in range(2):  # two calls in a row share the scratch array
        out = sdgs.BinBuffers(proj.n, 2_000_000, view.width, view.height)
        out.point_list.fill_(-1)
        k = ctypes.c_int64(-1)
        rc = sdgs.lib().sdgs_bin_sort_static(ctypes.byref(proj.struct()), ctypes.byref(view),
                                             ctypes.byref(out.struct()), ctypes.byref(k),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, sdgs.lib().sdgs_last_error()
        assert k.value == k_ref
        got = _bins_host(out, k.value)
        for a, b in zip(got, want):
            np.testing.assert_array_equal(a, b)


def test_static_scratch_rejects_oversized_problems():
    view = sdgs.view_struct(synth.make_camera((0, 0, -3), 1920, 1080, 60.0, 0.5))
    proj = sdgs.ProjectedBuffers(3_000_000)
    proj.rect.zero_()
    bins = sdgs.BinBuffers(1, 16, 1920, 1080)
    need = sdgs.bin_workspace_size(proj.n, bins.capacity, 1920, 1080)
    assert need > sdgs.STATIC_BIN_SCRATCH_BYTES
    with pytest.raises(sdgs.SdgsError) as e:
        sdgs.bin_sort_static(proj, view, bins)
    assert e.value.code == 2 and "scratch" in str(e.value)
