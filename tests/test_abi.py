"""The C ABI on the CPU: the library builds, loads and exports every entry point of
include/sdgs.h; the ctypes structs match the C layout; argument errors are reported without
touching a GPU."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

from paper_2503_07946_gb300 import build as pbuild
from paper_2503_07946_gb300 import sdgs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sdgs.h")


@pytest.fixture(scope="module")
def lib():
    pbuild.build_library()
    return sdgs.lib()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sdgs_[a-z0-9_]+)\s*\(", src)))


def test_header_entry_points_are_exported(lib):
    names = _declared()
    assert "sdgs_slice_project" in names and "sdgs_render_bwd" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in sdgs.SIGNATURES, f"{name} missing from the binding"
    assert set(sdgs.SIGNATURES) <= set(names)


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sdgs.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu %zu\\n", sizeof(sdgs_scene), sizeof(sdgs_view), sizeof(sdgs_projected),'
        " sizeof(sdgs_bins), sizeof(sdgs_grads));\n"
        '  printf("%zu %zu %zu %zu\\n", offsetof(sdgs_view, width), offsetof(sdgs_view, d),'
        " offsetof(sdgs_scene, lambda_d), offsetof(sdgs_bins, capacity));\n"
        '  printf("%zu %zu\\n", offsetof(sdgs_scene, dir_mode), offsetof(sdgs_grads, dlambda));\n'
        "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    assert sizes[:5] == [ctypes.sizeof(sdgs.Scene), ctypes.sizeof(sdgs.View), ctypes.sizeof(sdgs.Projected),
                         ctypes.sizeof(sdgs.Bins), ctypes.sizeof(sdgs.Grads)]
    assert sizes[5:] == [sdgs.View.width.offset, sdgs.View.d.offset, sdgs.Scene.lambda_d.offset,
                         sdgs.Bins.capacity.offset, sdgs.Scene.dir_mode.offset, sdgs.Grads.dlambda.offset]


def test_version_and_workspace_size(lib):
    assert sdgs.version().startswith("sdgs ")
    small = sdgs.bin_workspace_size(100, 1000, 64, 64)
    big = sdgs.bin_workspace_size(100_000, 10_000_000, 800, 800)
    assert 0 < small < big
    with pytest.raises(sdgs.SdgsError) as e:
        sdgs.bin_workspace_size(-1, 10, 64, 64)
    assert e.value.code == 1
    assert sdgs.bwd_workspace_size(1000) >= 1000 * 4


def test_invalid_arguments_are_rejected_before_any_gpu_work(lib):
    v = sdgs.View()
    v.width, v.height, v.fx, v.fy = 64, 64, 50.0, 50.0
    rc = lib.sdgs_slice_project(None, ctypes.byref(v), None, None)
    assert rc == 1 and b"scene" in lib.sdgs_last_error()
    s = sdgs.Scene(None, None, None, None, 10, 2, 0.05, 0.05)
    rc = lib.sdgs_slice_project(ctypes.byref(s), ctypes.byref(v), None, None)
    assert rc == 1 and b"sh_degree" in lib.sdgs_last_error()
    s.sh_degree = 3
    rc = lib.sdgs_slice_project(ctypes.byref(s), ctypes.byref(v), None, None)
    assert rc == 1  # NULL arrays
    v.width = 0
    s.n = 0
    rc = lib.sdgs_slice_project(ctypes.byref(s), ctypes.byref(v), None, None)
    assert rc == 1 and b"image size" in lib.sdgs_last_error()


def test_new_entry_points_reject_invalid_arguments_before_any_gpu_work(lib):
    v = sdgs.View()
    v.width, v.height, v.fx, v.fy = 64, 64, 50.0, 50.0
    s = sdgs.Scene(None, None, None, None, 0, 3, 0.05, 0.05, 2)
    rc = lib.sdgs_slice_project(ctypes.byref(s), ctypes.byref(v), None, None)
    assert rc == 1 and b"dir_mode" in lib.sdgs_last_error()
    s.dir_mode = 0
    w = sdgs.Agr(None, None, None, None)
    rc = lib.sdgs_agr_refine(ctypes.byref(s), ctypes.byref(w), 0.5, None, None, None)
    assert rc == 1 and b"AGR" in lib.sdgs_last_error()
    rc = lib.sdgs_agr_refine(ctypes.byref(s), None, 0.5, None, None, None)
    assert rc == 1
    b = ctypes.c_size_t(0)
    assert lib.sdgs_agr_bwd_workspace_size(1000, ctypes.byref(b)) == 0 and b.value > 0
    assert lib.sdgs_agr_bwd_workspace_size(-1, ctypes.byref(b)) == 1
    rc = lib.sdgs_densify_stats(ctypes.byref(s), ctypes.byref(v), None, None, None)
    assert rc == 1 and b"densify" in lib.sdgs_last_error()
    cfg = sdgs.DensifyCfg(float("nan"), 0.05, 0.25, 0.01)
    out = sdgs.Densify(None, None, None, None, None, None)
    rc = lib.sdgs_densify_stats(ctypes.byref(s), ctypes.byref(v), ctypes.byref(cfg), ctypes.byref(out), None)
    assert rc == 1 and b"finite" in lib.sdgs_last_error()
    # an image whose tile count would not fit the binning's 32-bit prefix sums
    v.width = v.height = 65535 * 16
    rc = lib.sdgs_bin_workspace_size(10, 10, v.width, v.height, ctypes.byref(b))
    assert rc == 1


def test_failure_test_support_rejects_invalid_arguments_before_any_gpu_work(lib):
    b = ctypes.c_size_t(0)
    assert lib.sdgs_lookback_selftest_workspace_size(4096, ctypes.byref(b)) == 0 and b.value > 0
    assert lib.sdgs_lookback_selftest_workspace_size(-1, ctypes.byref(b)) == 1
    for n, ticket, spins in ((-1, 1, 100), (4096, (1 << 20) + 1, 100), (4096, 1, 0), (4096, 1, (1 << 20) + 1)):
        rc = lib.sdgs_lookback_selftest(None, None, None, None, n, ticket, spins, None, 0, None)
        assert rc == 1 and b"selftest" in lib.sdgs_last_error(), (n, ticket, spins)
    rc = lib.sdgs_lookback_selftest(None, None, None, None, 4096, 1, 100, None, 0, None)
    assert rc == 1 and b"NULL" in lib.sdgs_last_error()
    rc = lib.sdgs_bin_sort_failure_selftest(None, None, None, 0, None, None, None)
    assert rc == 1 and b"projected" in lib.sdgs_last_error()
    for ticket, spins in (((1 << 20) + 1, 100), (1, 0), (1, (1 << 20) + 1)):
        rc = lib.sdgs_span_walk_selftest(None, None, None, 0, None, None, ticket, spins, None)
        assert rc == 1 and b"self-test" in lib.sdgs_last_error(), (ticket, spins)
    rc = lib.sdgs_span_walk_selftest(None, None, None, 0, None, None, 1, 100, None)
    assert rc == 1 and b"projected" in lib.sdgs_last_error()


def test_deferred_renderer_raises_when_the_previous_frame_failed():
    """A negative instance count read back behind a frame means its binning gave up (its lists
    were left empty): the next forward reports it instead of rendering on."""
    import torch
    from paper_2503_07946_gb300 import render as prender

    class _Done:
        def synchronize(self):
            pass

    r = object.__new__(prender.Renderer)
    r._k_event, r._k_host, r._k_capacity, r.overflowed_frames = _Done(), torch.tensor([-1]), 1000, 0
    with pytest.raises(RuntimeError, match="failed"):
        r.check_deferred()
    r._k_event, r._k_host = _Done(), torch.tensor([500])
    assert r.check_deferred() is False and r.num_instances == 500
