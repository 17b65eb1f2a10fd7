"""ctypes binding of libsdgs (include/sdgs.h): the same entry points, with torch tensors as memory.

This module only marshals arguments: it fills the C structs with device pointers of torch
tensors and calls the library.  Every step of the render path runs in the CUDA kernels of
libsdgs; when the library is missing every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsdgs.so")

OK = 0
ERR_NAMES = {1: "INVALID_ARG", 2: "WORKSPACE", 3: "OVERFLOW", 4: "CUDA", 5: "TIMEOUT", 6: "BUSY",
             7: "OOM_BUDGET", 8: "NOT_FOUND"}
TILE = 16


class SdgsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sdgs error {ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Scene(ctypes.Structure):
    _fields_ = [("mean7", ctypes.c_void_p), ("L28", ctypes.c_void_p), ("opacity", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32),
                ("lambda_t", ctypes.c_float), ("lambda_d", ctypes.c_float), ("dir_mode", ctypes.c_int32)]


class View(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_float * 16), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("near_plane", ctypes.c_float), ("t", ctypes.c_float),
                ("d", ctypes.c_float * 3), ("bg", ctypes.c_float * 3)]


class Projected(ctypes.Structure):
    _fields_ = [("mean2d", ctypes.c_void_p), ("conic_opacity", ctypes.c_void_p), ("rgb", ctypes.c_void_p),
                ("depth", ctypes.c_void_p), ("rect", ctypes.c_void_p), ("radius", ctypes.c_void_p),
                ("n", ctypes.c_int64)]


class Bins(ctypes.Structure):
    _fields_ = [("tile_keys", ctypes.c_void_p), ("point_list", ctypes.c_void_p), ("ranges", ctypes.c_void_p),
                ("num_instances", ctypes.c_void_p), ("capacity", ctypes.c_int64)]


class Grads(ctypes.Structure):
    _fields_ = [("dmean7", ctypes.c_void_p), ("dL28", ctypes.c_void_p), ("dopacity", ctypes.c_void_p),
                ("dsh", ctypes.c_void_p), ("dlambda", ctypes.c_void_p), ("overwrite", ctypes.c_int32)]


class Agr(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p)]


class AgrGrads(ctypes.Structure):
    _fields_ = [("dw1", ctypes.c_void_p), ("db1", ctypes.c_void_p), ("dw2", ctypes.c_void_p), ("db2", ctypes.c_void_p)]


class DensifyCfg(ctypes.Structure):
    _fields_ = [("extent", ctypes.c_float), ("split_pt", ctypes.c_float), ("split_t", ctypes.c_float),
                ("prune_alpha", ctypes.c_float)]


class Densify(ctypes.Structure):
    _fields_ = [("scale", ctypes.c_void_p), ("rot", ctypes.c_void_p), ("pt_norm", ctypes.c_void_p),
                ("t_scale", ctypes.c_void_p), ("split", ctypes.c_void_p), ("prune", ctypes.c_void_p)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("device", ctypes.c_int32),
                ("batch_window_us", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("retried", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("max_batch", ctypes.c_uint64),
                ("max_inflight", ctypes.c_uint64), ("bytes_allocated", ctypes.c_size_t)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3

_lib = None

# Exported symbols and their argument types; the CPU tests check this list against include/sdgs.h.
SIGNATURES = {
    "sdgs_version": ([], ctypes.c_char_p),
    "sdgs_last_error": ([], ctypes.c_char_p),
    "sdgs_slice_project": ([ctypes.POINTER(Scene), ctypes.POINTER(View), ctypes.POINTER(Projected),
                            ctypes.c_void_p], ctypes.c_int),
    "sdgs_bin_workspace_size": ([ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                 ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "sdgs_bin_sort": ([ctypes.POINTER(Projected), ctypes.POINTER(View), ctypes.c_void_p, ctypes.c_size_t,
                       ctypes.POINTER(Bins), ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p], ctypes.c_int),
    "sdgs_bin_sort_batch": ([ctypes.POINTER(Projected), ctypes.POINTER(View), ctypes.POINTER(ctypes.c_void_p),
                             ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(Bins), ctypes.c_int32,
                             ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p], ctypes.c_int),
    "sdgs_bin_sort_failure_selftest": ([ctypes.POINTER(Projected), ctypes.POINTER(View), ctypes.c_void_p,
                                        ctypes.c_size_t, ctypes.POINTER(Bins), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.c_void_p], ctypes.c_int),
    "sdgs_span_walk_selftest": ([ctypes.POINTER(Projected), ctypes.POINTER(View), ctypes.c_void_p,
                                 ctypes.c_size_t, ctypes.POINTER(Bins), ctypes.POINTER(ctypes.c_int64),
                                 ctypes.c_uint32, ctypes.c_int32, ctypes.c_void_p], ctypes.c_int),
    "sdgs_bin_sort_static": ([ctypes.POINTER(Projected), ctypes.POINTER(View), ctypes.POINTER(Bins),
                              ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p], ctypes.c_int),
    "sdgs_alu_peak_probe": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.POINTER(ctypes.c_double), ctypes.c_void_p], ctypes.c_int),
    "sdgs_lookback_selftest_workspace_size": ([ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "sdgs_lookback_selftest": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_uint32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p],
                               ctypes.c_int),
    "sdgs_render_fwd": ([ctypes.POINTER(Projected), ctypes.POINTER(Bins), ctypes.POINTER(View),
                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                        ctypes.c_int),
    "sdgs_bwd_workspace_size": ([ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "sdgs_render_bwd": ([ctypes.POINTER(Scene), ctypes.POINTER(View), ctypes.POINTER(Projected),
                         ctypes.POINTER(Bins), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(Grads), ctypes.c_void_p],
                        ctypes.c_int),
    "sdgs_agr_refine": ([ctypes.POINTER(Scene), ctypes.POINTER(Agr), ctypes.c_float, ctypes.c_void_p,
                         ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "sdgs_agr_bwd_workspace_size": ([ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "sdgs_agr_refine_bwd": ([ctypes.POINTER(Scene), ctypes.POINTER(Agr), ctypes.c_float, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(AgrGrads),
                             ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int),
    "sdgs_densify_stats": ([ctypes.POINTER(Scene), ctypes.POINTER(View), ctypes.POINTER(DensifyCfg),
                            ctypes.POINTER(Densify), ctypes.c_void_p], ctypes.c_int),
    "sdgs_server_create": ([ctypes.POINTER(ServerCfg), ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "sdgs_server_add_scene": ([ctypes.c_void_p, ctypes.POINTER(Scene), ctypes.POINTER(ctypes.c_int32)],
                              ctypes.c_int),
    "sdgs_server_submit": ([ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(View), ctypes.c_void_p,
                            ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "sdgs_server_poll": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "sdgs_server_wait": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)],
                         ctypes.c_int),
    "sdgs_server_release": ([ctypes.c_void_p, ctypes.c_uint64], ctypes.c_int),
    "sdgs_server_get_stats": ([ctypes.c_void_p, ctypes.POINTER(ServerStats)], ctypes.c_int),
    "sdgs_server_destroy": ([ctypes.c_void_p], None),
}


def lib():
    """Load libsdgs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise SdgsError(rc, lib().sdgs_last_error().decode())


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libsdgs needs CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("libsdgs needs contiguous tensors")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# ------------------------------------------------------------------------------------------
# Struct builders
# ------------------------------------------------------------------------------------------

def scene_struct(t: dict, lambda_t: float, lambda_d: float, dir_mode: int = 0) -> Scene:
    """t: dict of CUDA float32 tensors mean7 [N,7], L28 [N,28], opacity [N], sh [N,16,3].
    dir_mode 0 conditions on the view's direction d, 1 on each Gaussian's direction from the
    camera centre."""
    n = t["mean7"].shape[0]
    for k, w in (("mean7", 7), ("L28", 28), ("opacity", 1), ("sh", 48)):
        if t[k].dtype != torch.float32 or t[k].numel() != n * w:
            raise ValueError(f"scene tensor {k} must be float32 with {w} values per Gaussian")
    return Scene(_ptr(t["mean7"]), _ptr(t["L28"]), _ptr(t["opacity"]), _ptr(t["sh"]), n, 3,
                 float(lambda_t), float(lambda_d), int(dir_mode))


def view_struct(cam) -> View:
    """From a synth.Camera (or anything with the same attributes)."""
    v = View()
    vm = np.asarray(cam.viewmat, dtype=np.float64).reshape(16)
    for i in range(16):
        v.viewmat[i] = float(vm[i])
    v.fx, v.fy, v.cx, v.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    v.width, v.height = int(cam.width), int(cam.height)
    v.near_plane = float(getattr(cam, "near", 0.2))
    v.t = float(cam.t)
    for i in range(3):
        v.d[i] = float(cam.d[i])
        v.bg[i] = float(cam.bg[i])
    return v


class ProjectedBuffers:
    """Device buffers of the per-Gaussian screen-space record."""

    def __init__(self, n: int, device="cuda"):
        self.n = n
        self.mean2d = torch.empty(n, 2, dtype=torch.float32, device=device)
        self.conic_opacity = torch.empty(n, 4, dtype=torch.float32, device=device)
        self.rgb = torch.empty(n, 3, dtype=torch.float32, device=device)
        self.depth = torch.empty(n, dtype=torch.float32, device=device)
        self.rect = torch.empty(n, 4, dtype=torch.int16, device=device)  # uint16 bit pattern
        self.radius = torch.empty(n, dtype=torch.int32, device=device)

    def struct(self) -> Projected:
        return Projected(_ptr(self.mean2d), _ptr(self.conic_opacity), _ptr(self.rgb), _ptr(self.depth),
                         _ptr(self.rect), _ptr(self.radius), self.n)

    @staticmethod
    def from_host(rec: dict, device="cuda") -> "ProjectedBuffers":
        """Upload screen-space records (e.g. synth.random_projected) for the binning / raster calls."""
        n = rec["mean2d"].shape[0]
        p = ProjectedBuffers(n, device)
        p.mean2d.copy_(torch.as_tensor(np.asarray(rec["mean2d"], np.float32)))
        co = np.concatenate([np.asarray(rec["conic"], np.float32),
                             np.asarray(rec["opacity"], np.float32)[:, None]], 1)
        p.conic_opacity.copy_(torch.as_tensor(co))
        p.rgb.copy_(torch.as_tensor(np.asarray(rec["rgb"], np.float32)))
        p.depth.copy_(torch.as_tensor(np.asarray(rec["depth"], np.float32)))
        p.rect.copy_(torch.as_tensor(np.asarray(rec["rect"]).astype(np.uint16).view(np.int16)))
        p.radius.zero_()
        return p

    def rect_host(self) -> np.ndarray:
        return self.rect.cpu().numpy().view(np.uint16).astype(np.int64)


class BinBuffers:
    """Sorted instance lists, tile ranges and the workspace of sdgs_bin_sort."""

    def __init__(self, n: int, capacity: int, width: int, height: int, device="cuda", tile_keys: bool = True):
        self.n, self.capacity, self.width, self.height = n, int(capacity), width, height
        self.num_tiles = ((width + TILE - 1) // TILE) * ((height + TILE - 1) // TILE)
        self.tile_keys = (torch.empty(max(self.capacity, 1), dtype=torch.int32, device=device)
                          if tile_keys else None)
        self.point_list = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=device)
        self.ranges = torch.empty(self.num_tiles, 2, dtype=torch.int32, device=device)
        self.num_instances = torch.zeros(1, dtype=torch.int64, device=device)
        self.ws_bytes = bin_workspace_size(n, self.capacity, width, height)
        self.workspace = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=device)

    def struct(self) -> Bins:
        return Bins(_ptr(self.tile_keys), _ptr(self.point_list), _ptr(self.ranges), _ptr(self.num_instances),
                    self.capacity)


# ------------------------------------------------------------------------------------------
# Entry points (same names as the C ABI, minus the prefix)
# ------------------------------------------------------------------------------------------

def version() -> str:
    return lib().sdgs_version().decode()


def slice_project(scene: Scene, view: View, out: ProjectedBuffers, stream=None):
    _check(lib().sdgs_slice_project(ctypes.byref(scene), ctypes.byref(view), ctypes.byref(out.struct()),
                                    _stream(stream)))


def bin_workspace_size(n: int, capacity: int, width: int, height: int) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().sdgs_bin_workspace_size(n, capacity, width, height, ctypes.byref(b)))
    return int(b.value)


def bin_sort(proj: ProjectedBuffers, view: View, bins: BinBuffers, sync: bool = True, stream=None):
    """Returns the instance count K when sync=True (raises SdgsError(OVERFLOW) when K > capacity)."""
    k = ctypes.c_int64(0)
    _check(lib().sdgs_bin_sort(ctypes.byref(proj.struct()), ctypes.byref(view), _ptr(bins.workspace),
                               bins.ws_bytes, ctypes.byref(bins.struct()),
                               ctypes.byref(k) if sync else None, _stream(stream)))
    return int(k.value) if sync else None


def bin_sort_batch(projs: list, views: list, bins: list, sync: bool = True, stream=None):
    """sdgs_bin_sort_batch: bins several problems with one launch per step; returns the list of
    instance counts when sync=True."""
    n = len(projs)
    P = (Projected * n)(*[p.struct() for p in projs])
    V = (View * n)(*views)
    B = (Bins * n)(*[b.struct() for b in bins])
    W = (ctypes.c_void_p * n)(*[_ptr(b.workspace) for b in bins])
    S = (ctypes.c_size_t * n)(*[b.ws_bytes for b in bins])
    K = (ctypes.c_int64 * n)()
    _check(lib().sdgs_bin_sort_batch(P, V, W, S, B, n, K if sync else None, _stream(stream)))
    return [int(k) for k in K] if sync else None


def bin_sort_failure_selftest(proj: ProjectedBuffers, view: View, bins: BinBuffers, sync: bool = True,
                              stream=None):
    """sdgs_bin_sort_failure_selftest: bin_sort with its sort's first pass marked as having given up
    (test support for the failure path)."""
    k = ctypes.c_int64(0)
    _check(lib().sdgs_bin_sort_failure_selftest(ctypes.byref(proj.struct()), ctypes.byref(view), _ptr(bins.workspace),
                                                bins.ws_bytes, ctypes.byref(bins.struct()),
                                                ctypes.byref(k) if sync else None, _stream(stream)))
    return int(k.value) if sync else None


def span_walk_selftest(proj: ProjectedBuffers, view: View, bins: BinBuffers, first_ticket: int, spin_limit: int,
                       sync: bool = True, stream=None):
    """sdgs_span_walk_selftest: bin_sort with the span walk's block tickets starting at first_ticket
    and its waits giving up after spin_limit rounds (test support for its bounded wait)."""
    k = ctypes.c_int64(0)
    _check(lib().sdgs_span_walk_selftest(ctypes.byref(proj.struct()), ctypes.byref(view), _ptr(bins.workspace),
                                         bins.ws_bytes, ctypes.byref(bins.struct()), ctypes.byref(k) if sync else None,
                                         int(first_ticket), int(spin_limit), _stream(stream)))
    return int(k.value) if sync else None


STATIC_BIN_SCRATCH_BYTES = 64 << 20


def bin_sort_static(proj: ProjectedBuffers, view: View, bins: BinBuffers, sync: bool = True, stream=None):
    """sdgs_bin_sort_static: binning into the library's built-in scratch array (no workspace).

    For callers that cannot allocate device memory.  Same results as bin_sort; problems whose
    workspace would exceed the 64 MiB built-in scratch raise SdgsError(WORKSPACE).  Calls that
    overlap on the GPU share that scratch and race.
    """
    k = ctypes.c_int64(0)
    _check(lib().sdgs_bin_sort_static(ctypes.byref(proj.struct()), ctypes.byref(view), ctypes.byref(bins.struct()),
                                      ctypes.byref(k) if sync else None, _stream(stream)))
    return int(k.value) if sync else None


def alu_peak_probe(kind: int, iters: int, sink: torch.Tensor, stream=None) -> float:
    """sdgs_alu_peak_probe: enqueue one probe launch (0 FFMA, 1 paired FFMA, 2 MUFU ex2); returns
    the operations it performs (FLOP or ex2 evaluations)."""
    ops = ctypes.c_double(0.0)
    _check(lib().sdgs_alu_peak_probe(kind, iters, _ptr(sink), sink.numel(), ctypes.byref(ops), _stream(stream)))
    return float(ops.value)


def lookback_selftest(keys: torch.Tensor, vals: torch.Tensor, keys_out: torch.Tensor, vals_out: torch.Tensor,
                      n: int, first_ticket: int, spin_limit: int, stream=None):
    """sdgs_lookback_selftest: one 8-bit radix pass of the binning sort with its block tickets
    starting at first_ticket (test support for the sort's bounded waits).  Raises
    SdgsError(TIMEOUT) when a wait gave up."""
    b = ctypes.c_size_t(0)
    _check(lib().sdgs_lookback_selftest_workspace_size(n, ctypes.byref(b)))
    ws = torch.empty(max(int(b.value), 256), dtype=torch.uint8, device=keys.device)
    _check(lib().sdgs_lookback_selftest(_ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), n, first_ticket,
                                        spin_limit, _ptr(ws), int(b.value), _stream(stream)))


def render_fwd(proj: ProjectedBuffers, bins: BinBuffers, view: View, image: torch.Tensor,
               final_T: torch.Tensor, n_contrib: torch.Tensor, n_evaluated: torch.Tensor | None = None,
               stream=None):
    """n_evaluated: optional device int64 [2]; (evaluated, blended) (pixel, Gaussian) pairs are added."""
    if n_evaluated is not None and n_evaluated.numel() < 2:
        raise ValueError("n_evaluated needs 2 int64 elements (evaluations, contributions)")
    _check(lib().sdgs_render_fwd(ctypes.byref(proj.struct()), ctypes.byref(bins.struct()), ctypes.byref(view),
                                 _ptr(image), _ptr(final_T), _ptr(n_contrib), _ptr(n_evaluated),
                                 _stream(stream)))


def bwd_workspace_size(n: int) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().sdgs_bwd_workspace_size(n, ctypes.byref(b)))
    return int(b.value)


def render_bwd(scene: Scene, view: View, proj: ProjectedBuffers, bins: BinBuffers, final_T: torch.Tensor,
               n_contrib: torch.Tensor, dL_dimage: torch.Tensor, workspace: torch.Tensor, grads: dict,
               stream=None, overwrite: bool = False):
    """grads: mean7, L28, opacity, sh (and optionally lam) tensors; the call adds to them, or with
    overwrite=True writes them (they need no zeroing)."""
    g = Grads(_ptr(grads["mean7"]), _ptr(grads["L28"]), _ptr(grads["opacity"]), _ptr(grads["sh"]),
              _ptr(grads.get("lam")), 1 if overwrite else 0)
    _check(lib().sdgs_render_bwd(ctypes.byref(scene), ctypes.byref(view), ctypes.byref(proj.struct()),
                                 ctypes.byref(bins.struct()), _ptr(final_T), _ptr(n_contrib), _ptr(dL_dimage),
                                 _ptr(workspace), workspace.numel(), ctypes.byref(g), _stream(stream)))


AGR_SHAPES = dict(w1=(4, 64, 27), b1=(4, 64), w2=(35, 64), b2=(35,))


def agr_struct(w: dict) -> Agr:
    """w: dict of CUDA float32 tensors w1 [4,64,27], b1 [4,64], w2 [35,64], b2 [35] (contiguous)."""
    for k, shape in AGR_SHAPES.items():
        if w[k].dtype != torch.float32 or tuple(w[k].shape) != shape or not w[k].is_contiguous():
            raise ValueError(f"AGR weight {k} must be contiguous float32 of shape {shape}")
    return Agr(_ptr(w["w1"]), _ptr(w["b1"]), _ptr(w["w2"]), _ptr(w["b2"]))


def agr_refine(scene: Scene, w: dict, t: float, mean7_out: torch.Tensor, L28_out: torch.Tensor, stream=None):
    a = agr_struct(w)
    _check(lib().sdgs_agr_refine(ctypes.byref(scene), ctypes.byref(a), float(t), _ptr(mean7_out), _ptr(L28_out),
                                 _stream(stream)))


def agr_bwd_workspace_size(n: int) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().sdgs_agr_bwd_workspace_size(n, ctypes.byref(b)))
    return int(b.value)


def agr_refine_bwd(scene: Scene, w: dict, t: float, dmean7_hat, dL28_hat, dmean7, dL28, dw: dict,
                   workspace: torch.Tensor, stream=None):
    a = agr_struct(w)
    g = AgrGrads(_ptr(dw["w1"]), _ptr(dw["b1"]), _ptr(dw["w2"]), _ptr(dw["b2"]))
    _check(lib().sdgs_agr_refine_bwd(ctypes.byref(scene), ctypes.byref(a), float(t), _ptr(dmean7_hat),
                                     _ptr(dL28_hat), _ptr(dmean7), _ptr(dL28), ctypes.byref(g), _ptr(workspace),
                                     workspace.numel(), _stream(stream)))


def densify_stats(scene: Scene, view: View, n: int, extent: float, split_pt: float = 0.05, split_t: float = 0.25,
                  prune_alpha: float = 0.01, stream=None) -> dict:
    """sdgs_densify_stats into fresh device tensors: scale [n,3], rot [n,3,3], pt_norm, t_scale [n],
    split, prune [n] (bool)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    out = dict(scale=torch.empty(n, 3, device=dev), rot=torch.empty(n, 3, 3, device=dev),
               pt_norm=torch.empty(n, device=dev), t_scale=torch.empty(n, device=dev),
               split=torch.empty(n, dtype=torch.uint8, device=dev), prune=torch.empty(n, dtype=torch.uint8, device=dev))
    o = Densify(*(_ptr(out[k]) for k in ("scale", "rot", "pt_norm", "t_scale", "split", "prune")))
    cfg = DensifyCfg(float(extent), float(split_pt), float(split_t), float(prune_alpha))
    _check(lib().sdgs_densify_stats(ctypes.byref(scene), ctypes.byref(view), ctypes.byref(cfg), ctypes.byref(o),
                                    _stream(stream)))
    out["split"] = out["split"].bool()
    out["prune"] = out["prune"].bool()
    return out


class Server:
    """The sdgs_server_* entry points: resident scenes, continuous batching of render requests.

    Scene tensors (and output images) must stay alive while the server uses them; this wrapper
    keeps references to the scenes it registered.
    """

    def __init__(self, budget_bytes: int = 8 << 30, slots: int = 4, queue_capacity: int = 4096, device: int = 0,
                 batch_window_us: int = 0):
        cfg = ServerCfg(budget_bytes, slots, queue_capacity, device, batch_window_us)
        h = ctypes.c_void_p()
        _check(lib().sdgs_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._scenes = []

    def add_scene(self, tensors: dict, lambda_t: float, lambda_d: float) -> int:
        sid = ctypes.c_int32(-1)
        st = scene_struct(tensors, lambda_t, lambda_d)
        _check(lib().sdgs_server_add_scene(self.handle, ctypes.byref(st), ctypes.byref(sid)))
        self._scenes.append(tensors)
        return int(sid.value)

    def submit(self, scene_id: int, view: View, out_image: torch.Tensor) -> int:
        """out_image: [H, W, 3] float32, on the device or in page-locked host memory."""
        if out_image.dtype != torch.float32 or not out_image.is_contiguous():
            raise ValueError("out_image must be contiguous float32")
        rid = ctypes.c_uint64(0)
        _check(lib().sdgs_server_submit(self.handle, scene_id, ctypes.byref(view), out_image.data_ptr(),
                                        ctypes.byref(rid)))
        return int(rid.value)

    def poll(self, rid: int):
        st, lat = ctypes.c_int32(-1), ctypes.c_float(0)
        _check(lib().sdgs_server_poll(self.handle, rid, ctypes.byref(st), ctypes.byref(lat)))
        return int(st.value), float(lat.value)

    def wait(self, rid: int, timeout_ms: int = 10_000) -> float:
        lat = ctypes.c_float(0)
        _check(lib().sdgs_server_wait(self.handle, rid, timeout_ms, ctypes.byref(lat)))
        return float(lat.value)

    def release(self, rid: int = 0) -> int:
        return int(lib().sdgs_server_release(self.handle, rid))

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().sdgs_server_get_stats(self.handle, ctypes.byref(st)))
        return {k: int(getattr(st, k)) for k, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            lib().sdgs_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
