"""Gradients of the CUDA adjoint (through the C ABI and the autograd Function) against the
FP64 oracle's autograd gradients."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from oracle import render as orender
from paper_2503_07946_gb300 import render as prender
from paper_2503_07946_gb300 import sdgs

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3  # per tensor: max|g - g_ref| <= 1e-3 max|g_ref|


def _gpu_grads(scene, cam, dL):
    dev = prender.scene_to_device(scene)
    params = {k: v.clone().requires_grad_(True) for k, v in dev.items()}
    lam = torch.tensor([scene.lambda_t, scene.lambda_d], dtype=torch.float32, device="cuda", requires_grad=True)
    r = prender.Renderer(scene.n, cam.width, cam.height)
    img = prender.render_image(params["mean7"], params["L28"], params["opacity"], params["sh"],
                               sdgs.view_struct(cam), lam[0], lam[1], r, scene.dir_mode)
    (img * torch.as_tensor(dL, dtype=torch.float32, device="cuda")).sum().backward()
    out = {k: v.grad.cpu().numpy() for k, v in params.items()}
    out["lam"] = lam.grad.cpu().numpy()
    return out, img.detach().cpu().numpy()


def _check(scene, cam, seed):
    rng = np.random.default_rng(seed)
    dL = rng.normal(size=(cam.height, cam.width, 3))
    got, img = _gpu_grads(scene, cam, dL)
    ref = orender.vjp(scene, cam, dL)
    report = {}
    for k in ("mean7", "L28", "opacity", "sh", "lam"):
        g, r = got[k].reshape(-1), ref[k].reshape(-1)
        scale = np.abs(r).max()
        report[k] = float(np.abs(g - r).max() / scale)
    return report


def _case(case):
    if case == "config0":
        return synth.config_scene(0), synth.config_cameras(0)[0]
    if case == "rotated":
        scene = synth.config_scene(0, n=2048)
        return scene, synth.make_camera((1.2, -0.8, -2.6), 141, 97, 55.0, 0.3, bg=(0.2, 0.4, 0.6))
    if case == "small":
        scene = synth.make_scene(64, seed=16, box=0.6)
        return scene, synth.make_camera((0.0, 0.0, -3.0), 32, 32, 60.0, 0.5, bg=(0.3, 0.3, 0.3))
    # per-Gaussian conditioning direction, broad direction blocks so most Gaussians stay visible
    scene = synth.make_scene(2048, seed=31, box=1.0, diag=(0.05, 0.4), lambda_t=0.1, lambda_d=0.2)
    scene.dir_mode = 1
    return scene, synth.make_camera((0.9, -0.4, -2.8), 120, 90, 55.0, 0.6, bg=(0.1, 0.2, 0.3))


@pytest.mark.parametrize("case", ["config0", "rotated", "small", "gaussian_dir"])
def test_gradients_match_oracle(case):
    """Gradients of all parameter tensors and of (lambda_t, lambda_d)."""
    scene, cam = _case(case)
    rep = _check(scene, cam, seed=3)
    for k, v in rep.items():
        assert v <= GRAD_TOL, (k, rep)


@pytest.mark.parametrize("lam_kind", ["host_float", "host_tensor"])
def test_host_lambda_matches_device_lambda(lam_kind):
    """Lambdas given on the host (no device round trip; a plain float also skips the lambda
    reduction) give the image and parameter gradients of device lambdas; a host tensor that
    requires grad gets its gradient on the host."""
    scene, cam = _case("rotated")
    rng = np.random.default_rng(4)
    dL = torch.as_tensor(rng.normal(size=(cam.height, cam.width, 3)), dtype=torch.float32, device="cuda")
    dev = prender.scene_to_device(scene)
    view = sdgs.view_struct(cam)
    runs = []
    for kind in ("device", lam_kind):
        params = {k: v.clone().requires_grad_(True) for k, v in dev.items()}
        r = prender.Renderer(scene.n, cam.width, cam.height)
        lam = None
        if kind == "host_float":
            lt, ld = scene.lambda_t, scene.lambda_d
        else:
            lam = torch.tensor([scene.lambda_t, scene.lambda_d], dtype=torch.float32,
                               device="cuda" if kind == "device" else "cpu", requires_grad=True)
            lt, ld = lam[0], lam[1]
        img = prender.render_image(params["mean7"], params["L28"], params["opacity"], params["sh"], view,
                                   lt, ld, r)
        (img * dL).sum().backward()
        grads = {k: v.grad.cpu() for k, v in params.items()}
        if lam is not None:
            assert lam.grad.device == lam.device
            grads["lam"] = lam.grad.cpu()
        runs.append((img.detach().cpu(), grads))
    assert torch.equal(runs[0][0], runs[1][0])
    for k, g in runs[1][1].items():
        ref = runs[0][1][k]
        # the same sums, added by atomics in another order
        assert float((g - ref).abs().max()) <= 1e-4 * float(ref.abs().max()), k


def test_backward_after_another_forward_on_the_same_renderer_raises():
    """The backward replays the renderer's lists of its own frame: after a second forward on the
    same Renderer (another view, a target image) those lists are gone, so it must refuse."""
    scene, cam = _case("small")
    dev = prender.scene_to_device(scene)
    params = {k: v.clone().requires_grad_(True) for k, v in dev.items()}
    r = prender.Renderer(scene.n, cam.width, cam.height)
    view = sdgs.view_struct(cam)
    img = prender.render_image(params["mean7"], params["L28"], params["opacity"], params["sh"], view,
                               scene.lambda_t, scene.lambda_d, r)
    with torch.no_grad():
        r.forward(sdgs.scene_struct(dev, scene.lambda_t, scene.lambda_d), view)  # e.g. a target render
    with pytest.raises(RuntimeError, match="rendered 1 more frame"):
        img.sum().backward()
    img2 = prender.render_image(params["mean7"], params["L28"], params["opacity"], params["sh"], view,
                                scene.lambda_t, scene.lambda_d, r)
    img2.sum().backward()  # its own frame: fine
    assert float(params["opacity"].grad.abs().sum()) > 0


def test_fp32_adjoint_matches_central_differences_of_the_fp32_render():
    """The CUDA adjoint against central differences of the CUDA forward itself (both FP32), on the
    N = 64, 32 x 32 differentiation case: no oracle in the loop.  A parameter whose step flips a
    discrete decision (visibility, a rectangle, the 1/255 skip, the 0.99 clamp, the stop rule)
    shows up as a jump: its two one-sided differences disagree, and it is set aside (counted)."""
    scene, cam = _case("small")
    rng = np.random.default_rng(23)
    dL = rng.normal(size=(cam.height, cam.width, 3))
    got, _ = _gpu_grads(scene, cam, dL)
    dev = prender.scene_to_device(scene)
    view = sdgs.view_struct(cam)
    r = prender.Renderer(scene.n, cam.width, cam.height)
    dLt = torch.as_tensor(dL, dtype=torch.float64)

    def loss(t):
        st = sdgs.scene_struct(t, scene.lambda_t, scene.lambda_d)
        img = r.forward(st, view).double().cpu()
        return float((img * dLt).sum())

    base = loss(dev)
    vis = (r.proj.rect[:, 2] > r.proj.rect[:, 0]).cpu().numpy()
    checked = jumps = 0
    worst = 0.0
    for name in ("mean7", "L28", "opacity", "sh"):
        flat = dev[name].reshape(-1)
        per = flat.numel() // scene.n
        g = got[name].reshape(-1)
        scale = float(np.abs(g).max())
        cand = [i for i in rng.permutation(flat.numel()) if vis[i // per]][:30]
        for i in cand:
            x0 = float(flat[i])
            h = 2e-3 * max(1.0, abs(x0)) if name != "opacity" else 2e-3
            vals = []
            for s in (1, -1):
                t = {k: v.clone() for k, v in dev.items()}
                t[name].reshape(-1)[i] = x0 + s * h
                vals.append(loss(t))
            fwd, bwd = (vals[0] - base) / h, (base - vals[1]) / h
            if abs(fwd - bwd) > 0.05 * max(abs(fwd), abs(bwd), 1e-3 * scale):
                jumps += 1
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            err = abs(fd - float(g[i])) / max(abs(fd), abs(float(g[i])), 1e-2 * scale)
            worst = max(worst, err)
            checked += 1
    assert checked >= 80, (checked, jumps)
    assert worst < 0.05, worst


def test_written_gradients_equal_added_gradients():
    """render_bwd writing the gradients (into arrays full of NaN) gives what adding them into zeroed
    arrays gives (the autograd Function uses the written form), and adding twice gives twice.  (The
    per-Gaussian screen-space sums are added up by atomics across tiles, so two calls agree to
    rounding, not bit for bit.)"""
    scene, cam = _case("rotated")
    dev = prender.scene_to_device(scene)
    st = sdgs.scene_struct(dev, scene.lambda_t, scene.lambda_d, scene.dir_mode)
    view = sdgs.view_struct(cam)
    r = prender.Renderer(scene.n, cam.width, cam.height)
    r.forward(st, view)
    dL = torch.as_tensor(np.random.default_rng(5).normal(size=(cam.height, cam.width, 3)), dtype=torch.float32,
                         device="cuda")
    ws = torch.empty(max(sdgs.bwd_workspace_size(scene.n), 256), dtype=torch.uint8, device="cuda")
    added = {k: torch.zeros_like(v) for k, v in dev.items()}
    added["lam"] = torch.zeros(2, dtype=torch.float32, device="cuda")
    written = {k: torch.full_like(v, float("nan")) for k, v in dev.items()}
    written["lam"] = torch.full((2,), float("nan"), dtype=torch.float32, device="cuda")
    sdgs.render_bwd(st, view, r.proj, r.bins, r.final_T, r.n_contrib, dL, ws, added)
    sdgs.render_bwd(st, view, r.proj, r.bins, r.final_T, r.n_contrib, dL, ws, written, overwrite=True)
    torch.cuda.synchronize()
    culled = (r.proj.rect[:, 2] <= r.proj.rect[:, 0]) | (r.proj.rect[:, 3] <= r.proj.rect[:, 1])
    assert 0 < int(culled.sum()) < scene.n
    for k in ("mean7", "L28", "opacity", "sh", "lam"):
        w, a = written[k], added[k]
        assert not torch.isnan(w).any(), k  # every entry written
        tol = 1e-5 * float(a.abs().max())
        torch.testing.assert_close(w, a, rtol=1e-4, atol=tol)
        if k != "lam":
            assert (w.reshape(scene.n, -1)[culled] == 0).all(), k  # culled Gaussians: zero
    sdgs.render_bwd(st, view, r.proj, r.bins, r.final_T, r.n_contrib, dL, ws, added)
    torch.cuda.synchronize()
    for k in ("mean7", "L28", "opacity", "sh"):
        torch.testing.assert_close(added[k], 2 * written[k], rtol=1e-4, atol=2e-5 * float(written[k].abs().max()))
