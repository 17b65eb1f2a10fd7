"""Pipeline wrappers over the C ABI: a reusable renderer and the autograd Function.

These only sequence the library calls (slice_project -> bin_sort -> render_fwd, and
render_bwd) and own the device buffers; all arithmetic is in the CUDA kernels.
"""
from __future__ import annotations

import warnings

import numpy as np
import torch

from . import sdgs


def scene_to_device(scene, device="cuda") -> dict:
    """Upload a synth.Scene (host float32 arrays) to contiguous CUDA tensors."""
    return dict(mean7=torch.as_tensor(np.ascontiguousarray(scene.mean7), device=device),
                L28=torch.as_tensor(np.ascontiguousarray(scene.L28), device=device),
                opacity=torch.as_tensor(np.ascontiguousarray(scene.opacity), device=device),
                sh=torch.as_tensor(np.ascontiguousarray(scene.sh), device=device).reshape(-1, 16, 3))


class Renderer:
    """Owns the projected record, bins and image buffers for one (n, width, height).

    `capacity` bounds the (tile, Gaussian) instances; when a frame needs more, the bins are
    reallocated at 1.25x the count and binning runs again.

    deferred_check=True removes the host synchronisation after binning: the frame's instance
    count is copied to pinned host memory behind the binning and read at the next forward (by
    then the GPU is normally past it, so the host never waits for an idle GPU).  A frame that
    needed more than the capacity is then rendered with the nearest `capacity` instances (the
    overflow contract of sdgs_bin_sort); the next forward warns, counts it in
    `overflowed_frames` and grows the bins.  Meant for training loops, where the capacity is
    sized by the first frames.
    """

    def __init__(self, n: int, width: int, height: int, capacity: int | None = None, device="cuda",
                 tile_keys: bool = False, deferred_check: bool = False):
        self.n, self.width, self.height, self.device = n, width, height, device
        self.tile_keys = tile_keys
        self.deferred_check = deferred_check
        self.overflowed_frames = 0
        self._k_host = torch.zeros(1, dtype=torch.int64, pin_memory=True) if deferred_check else None
        self._k_event = None
        self._k_capacity = 0
        self.proj = sdgs.ProjectedBuffers(n, device)
        self.bins = sdgs.BinBuffers(n, capacity if capacity is not None else max(4096, 16 * n), width,
                                    height, device, tile_keys=tile_keys)
        self.image = torch.empty(height, width, 3, dtype=torch.float32, device=device)
        self.final_T = torch.empty(height, width, dtype=torch.float32, device=device)
        self.n_contrib = torch.empty(height, width, dtype=torch.int32, device=device)
        self.num_instances = 0
        self.frames = 0  # forwards so far: a backward needs the lists of its own frame

    def grow(self, k: int):
        self.bins = sdgs.BinBuffers(self.n, int(k * 1.25) + 1024, self.width, self.height, self.device,
                                    tile_keys=self.tile_keys)

    def bin(self, view: sdgs.View, stream=None) -> int:
        try:
            k = sdgs.bin_sort(self.proj, view, self.bins, sync=True, stream=stream)
        except sdgs.SdgsError as e:
            if e.code != 3:
                raise
            self.grow(int(self.bins.num_instances.item()))
            k = sdgs.bin_sort(self.proj, view, self.bins, sync=True, stream=stream)
        self.num_instances = k
        return k

    def check_deferred(self) -> bool:
        """Reads the instance count of the last deferred frame (waiting only for that point of its
        stream); grows the bins and returns True when that frame exceeded the capacity."""
        if self._k_event is None:
            return False
        self._k_event.synchronize()
        self._k_event = None
        k = int(self._k_host[0])
        self.num_instances = k
        if k < 0:  # a bounded wait inside the binning sort gave up: that frame's lists were empty
            raise RuntimeError("binning of the previous frame failed (a sort wait gave up); "
                               "its image holds only the background")
        if k <= self._k_capacity:
            return False
        self.overflowed_frames += 1
        if k > self.bins.capacity:
            self.grow(k)
        return True

    def _bin_deferred(self, view: sdgs.View, stream=None):
        if self.check_deferred():
            warnings.warn("the previous frame had more (tile, Gaussian) instances than the bins' capacity and "
                          "was rendered with the nearest ones; the bins have grown", RuntimeWarning, stacklevel=3)
        sdgs.bin_sort(self.proj, view, self.bins, sync=False, stream=stream)
        st = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(st):
            self._k_host.copy_(self.bins.num_instances, non_blocking=True)
            self._k_event = torch.cuda.Event()
            self._k_event.record(st)
        self._k_capacity = self.bins.capacity

    def forward(self, scene: sdgs.Scene, view: sdgs.View, stream=None, image: torch.Tensor | None = None
                ) -> torch.Tensor:
        """Renders into `image` ([height, width, 3] float32 CUDA) when given, else into the
        renderer's own image buffer; returns the image."""
        self.frames += 1
        sdgs.slice_project(scene, view, self.proj, stream)
        if self.deferred_check:
            self._bin_deferred(view, stream)
        else:
            self.bin(view, stream)
        out = self.image if image is None else image
        sdgs.render_fwd(self.proj, self.bins, view, out, self.final_T, self.n_contrib, stream=stream)
        return out

    def forward_async(self, scene: sdgs.Scene, view: sdgs.View, stream=None) -> torch.Tensor:
        """Same three calls without the host read of the instance count (capacity must suffice)."""
        self.frames += 1
        sdgs.slice_project(scene, view, self.proj, stream)
        sdgs.bin_sort(self.proj, view, self.bins, sync=False, stream=stream)
        sdgs.render_fwd(self.proj, self.bins, view, self.image, self.final_T, self.n_contrib, stream=stream)
        return self.image


class Render7DGS(torch.autograd.Function):
    """image = render(mean7, L28, opacity, sh, lam) for one view, with the CUDA adjoint as backward.

    Gradients flow to all four parameter tensors and to lam = (lambda_t, lambda_d); opacity is
    the activated alpha and L28 the packed Cholesky factor as given (activations live in torch).
    """

    @staticmethod
    def forward(ctx, mean7, L28, opacity, sh, lam, view: sdgs.View, renderer: Renderer, dir_mode: int):
        t = dict(mean7=mean7.contiguous(), L28=L28.contiguous(), opacity=opacity.contiguous(),
                 sh=sh.contiguous())
        lam_t, lam_d = (float(x) for x in lam.detach().cpu().tolist())  # no device round trip for a host lam
        scene = sdgs.scene_struct(t, lam_t, lam_d, dir_mode)
        image = renderer.forward(scene, view, image=torch.empty_like(renderer.image))  # (the caller keeps it)
        ctx.renderer, ctx.view, ctx.lam, ctx.dir_mode = renderer, view, (lam_t, lam_d), dir_mode
        ctx.frame = renderer.frames
        ctx.lam_device = lam.device
        # the backward reads the renderer's final_T and n_contrib of this frame; it refuses to run
        # once the renderer has rendered another frame, so they need no copy
        ctx.save_for_backward(t["mean7"], t["L28"], t["opacity"], t["sh"])
        return image

    @staticmethod
    def backward(ctx, grad_image):
        mean7, L28, opacity, sh = ctx.saved_tensors
        t = dict(mean7=mean7, L28=L28, opacity=opacity, sh=sh)
        scene = sdgs.scene_struct(t, *ctx.lam, ctx.dir_mode)
        grads = {k: torch.empty_like(v) for k, v in t.items()}  # (written whole by the call)
        want_lam = ctx.needs_input_grad[4]
        if want_lam:  # otherwise no dlambda: the kernel skips that reduction
            grads["lam"] = torch.empty(2, dtype=torch.float32, device=mean7.device)
        r = ctx.renderer
        if r.frames != ctx.frame:  # its projected records and tile lists now belong to a later frame
            raise RuntimeError("Render7DGS.backward: the Renderer has rendered %d more frame(s) since this image; "
                               "take the gradient before rendering again with it, or render each image whose "
                               "gradient is needed with its own Renderer" % (r.frames - ctx.frame))
        ws = torch.empty(max(sdgs.bwd_workspace_size(r.n), 256), dtype=torch.uint8, device=mean7.device)
        sdgs.render_bwd(scene, ctx.view, r.proj, r.bins, r.final_T, r.n_contrib, grad_image.contiguous(), ws, grads,
                        overwrite=True)
        dlam = grads["lam"].to(ctx.lam_device) if want_lam else None
        return grads["mean7"], grads["L28"], grads["opacity"], grads["sh"], dlam, None, None, None


def render_image(mean7, L28, opacity, sh, view: sdgs.View, lambda_t, lambda_d, renderer: Renderer,
                 dir_mode: int = 0) -> torch.Tensor:
    """lambda_t, lambda_d: floats or 0-d tensors (gradients reach tensors that require them).

    The kernels take lambda by value, so a device tensor is read back to the host (one
    synchronisation); plain floats stay on the host."""
    if torch.is_tensor(lambda_t) or torch.is_tensor(lambda_d):
        dev = mean7.device
        lam = torch.stack([torch.as_tensor(lambda_t, dtype=torch.float32, device=dev).reshape(()),
                           torch.as_tensor(lambda_d, dtype=torch.float32, device=dev).reshape(())])
    else:
        lam = torch.tensor([float(lambda_t), float(lambda_d)], dtype=torch.float32)
    return Render7DGS.apply(mean7, L28, opacity, sh, lam, view, renderer, dir_mode)


_AGR_UNUSED: dict = {}


def _agr_unused_arrays(n: int, device) -> tuple[torch.Tensor, torch.Tensor]:
    """Opacity and SH arrays for the scene struct of the refinement calls, which read neither
    (the ABI still wants valid arrays of the scene's size); allocated once per (n, device)."""
    key = (n, str(device))
    if key not in _AGR_UNUSED:
        _AGR_UNUSED.clear()
        _AGR_UNUSED[key] = (torch.zeros(n, device=device), torch.zeros(n, 16, 3, device=device))
    return _AGR_UNUSED[key]


class AGRRefine(torch.autograd.Function):
    """(mean7^, L28^) = adaptive refinement of (mean7, L28) at time t by the four MLPs (w1, b1, w2,
    b2); backward is the CUDA adjoint (input and weight gradients)."""

    @staticmethod
    def forward(ctx, mean7, L28, w1, b1, w2, b2, t: float):
        w = dict(w1=w1.contiguous(), b1=b1.contiguous(), w2=w2.contiguous(), b2=b2.contiguous())
        m7, l28 = mean7.contiguous(), L28.contiguous()
        n = m7.shape[0]
        opacity, sh = _agr_unused_arrays(n, m7.device)
        scene = sdgs.scene_struct(dict(mean7=m7, L28=l28, opacity=opacity, sh=sh), 0.0, 0.0)
        m_out, l_out = torch.empty_like(m7), torch.empty_like(l28)
        sdgs.agr_refine(scene, w, t, m_out, l_out)
        ctx.t = float(t)
        ctx.save_for_backward(m7, l28, w["w1"], w["b1"], w["w2"], w["b2"])
        return m_out, l_out

    @staticmethod
    def backward(ctx, d_m, d_l):
        m7, l28, w1, b1, w2, b2 = ctx.saved_tensors
        n = m7.shape[0]
        w = dict(w1=w1, b1=b1, w2=w2, b2=b2)
        opacity, sh = _agr_unused_arrays(n, m7.device)
        scene = sdgs.scene_struct(dict(mean7=m7, L28=l28, opacity=opacity, sh=sh), 0.0, 0.0)
        d_m = torch.zeros_like(m7) if d_m is None else d_m.contiguous()
        d_l = torch.zeros_like(l28) if d_l is None else d_l.contiguous()
        gm = torch.zeros_like(m7)
        dw = {k: torch.zeros_like(v) for k, v in w.items()}
        ws = torch.empty(max(sdgs.agr_bwd_workspace_size(n), 256), dtype=torch.uint8, device=m7.device)
        # the residual of L does not depend on L: its gradient passes through unchanged (dL28 = NULL)
        sdgs.agr_refine_bwd(scene, w, ctx.t, d_m, d_l, gm, None, dw, ws)
        return gm, d_l, dw["w1"], dw["b1"], dw["w2"], dw["b2"], None


def agr_refine(mean7, L28, weights: dict, t: float):
    """Differentiable adaptive refinement: returns (mean7^, L28^)."""
    return AGRRefine.apply(mean7, L28, weights["w1"], weights["b1"], weights["w2"], weights["b2"], float(t))
