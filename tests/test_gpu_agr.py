"""Adaptive Gaussian Refinement (Sec. 4.3) of the CUDA path against the FP64 oracle: refined
parameters, the adjoint (input and weight gradients), and a refined render with its gradients."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from oracle import agr as oagr
from oracle import render as orender
from paper_2503_07946_gb300 import render as prender
from paper_2503_07946_gb300 import sdgs

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
COLOUR_TOL = 2e-4


def _weights_dev(w):
    return {k: torch.as_tensor(v, device="cuda").contiguous() for k, v in w.items()}


def _gpu_refine(scene, w, t):
    dev = prender.scene_to_device(scene)
    st = sdgs.scene_struct(dev, scene.lambda_t, scene.lambda_d)
    m, l = torch.empty_like(dev["mean7"]), torch.empty_like(dev["L28"])
    sdgs.agr_refine(st, _weights_dev(w), t, m, l)
    torch.cuda.synchronize()
    return m.cpu().numpy(), l.cpu().numpy()


@pytest.mark.parametrize("t,scale", [(0.375, 1.0), (0.8125, 0.1), (0.37, 1.0)])
def test_refined_parameters_match_oracle(t, scale):
    scene = synth.make_scene(5000, seed=61, box=1.0)
    w = synth.make_agr_weights(seed=62, scale=scale)
    m, l = _gpu_refine(scene, w, t)
    wt = oagr.weights_to_torch(w)
    mr, lr = oagr.refine(torch.tensor(scene.mean7, dtype=torch.float64), torch.tensor(scene.L28, dtype=torch.float64),
                         float(np.float32(t)), wt)
    # FP32 residuals of a 27 -> 64 -> 35 network: within 2e-6 of the residual scale
    res_scale = max(np.abs(mr.numpy() - scene.mean7).max(), np.abs(lr.numpy() - scene.L28).max())
    np.testing.assert_allclose(m, mr.numpy(), rtol=0, atol=2e-6 * max(1.0, res_scale) + 1e-6)
    np.testing.assert_allclose(l, lr.numpy(), rtol=0, atol=2e-6 * max(1.0, res_scale) + 1e-6)
    assert res_scale > 1e-3  # the refinement moved the parameters


def test_refinement_adjoint_matches_oracle_and_is_deterministic():
    n, t = 20000, 0.4375
    scene = synth.make_scene(n, seed=63, box=1.0)
    w = synth.make_agr_weights(seed=64, scale=1.0)
    rng = np.random.default_rng(65)
    dm_hat = rng.normal(size=(n, 7)).astype(np.float32)
    dl_hat = rng.normal(size=(n, 28)).astype(np.float32)
    dev = prender.scene_to_device(scene)
    st = sdgs.scene_struct(dev, scene.lambda_t, scene.lambda_d)
    wd = _weights_dev(w)
    ws = torch.empty(sdgs.agr_bwd_workspace_size(n), dtype=torch.uint8, device="cuda")
    runs = []
    for with_dl28 in (True, True, False):
        gm, gl = torch.zeros(n, 7, device="cuda"), torch.zeros(n, 28, device="cuda")
        dw = {k: torch.zeros_like(v) for k, v in wd.items()}
        sdgs.agr_refine_bwd(st, wd, t, torch.tensor(dm_hat, device="cuda"), torch.tensor(dl_hat, device="cuda"),
                            gm, gl if with_dl28 else None, dw, ws)
        torch.cuda.synchronize()
        runs.append(dict(mean7=gm.cpu().numpy(), L28=gl.cpu().numpy(), **{k: v.cpu().numpy() for k, v in dw.items()}))
    for k in runs[0]:
        np.testing.assert_array_equal(runs[0][k], runs[1][k])  # fixed reduction order
    # dL28 = NULL: the same mean and weight gradients, and dL28 left alone (the caller's to take)
    for k in runs[0]:
        if k != "L28":
            np.testing.assert_array_equal(runs[2][k], runs[0][k])
    np.testing.assert_array_equal(runs[2]["L28"], 0.0)
    np.testing.assert_array_equal(runs[0]["L28"], dl_hat)
    got = runs[0]
    m7 = torch.tensor(scene.mean7, dtype=torch.float64, requires_grad=True)
    l28 = torch.tensor(scene.L28, dtype=torch.float64, requires_grad=True)
    wt = oagr.weights_to_torch(w, requires_grad=True)
    mh, lh = oagr.refine(m7, l28, t, wt)
    ((mh * torch.tensor(dm_hat, dtype=torch.float64)).sum() + (lh * torch.tensor(dl_hat, dtype=torch.float64)).sum()).backward()
    ref = dict(mean7=m7.grad.numpy(), L28=l28.grad.numpy(), **{k: v.grad.numpy() for k, v in wt.items()})
    # a hidden unit whose pre-activation is within FP32 error of 0 may take the other ReLU branch;
    # the per-Gaussian input gradients of those Gaussians are compared separately, loosely
    f = oagr.features(torch.tensor(scene.mean7, dtype=torch.float64), t)
    z = torch.stack([f @ wt["w1"][m].detach().T + wt["b1"][m].detach() for m in range(4)], 1).reshape(n, -1)
    kink = (z.abs() < 1e-5).any(1).numpy()
    assert kink.sum() < n // 100
    for k in ref:
        g, r = got[k], ref[k]
        if k == "mean7":
            g, r = g[~kink], r[~kink]
        err = np.abs(g - r).max() / np.abs(r).max()
        assert err <= GRAD_TOL, (k, err)


def test_refined_render_and_gradients_match_oracle():
    """Refine (CUDA) -> render (CUDA) vs the oracle's refine -> render; gradients of the weights
    and of the raw parameters through both."""
    scene = synth.config_scene(0, n=2048)
    cam = synth.make_camera((0.6, -0.4, -2.8), 96, 72, 55.0, 0.375, bg=(0.2, 0.3, 0.4))
    w = synth.make_agr_weights(seed=66, scale=0.1)
    dev = prender.scene_to_device(scene)
    params = {k: v.clone().requires_grad_(True) for k, v in dev.items()}
    wd = {k: v.clone().requires_grad_(True) for k, v in _weights_dev(w).items()}
    r = prender.Renderer(scene.n, cam.width, cam.height)
    m_hat, l_hat = prender.agr_refine(params["mean7"], params["L28"], wd, cam.t)
    img = prender.render_image(m_hat, l_hat, params["opacity"], params["sh"], sdgs.view_struct(cam),
                               scene.lambda_t, scene.lambda_d, r)
    rng = np.random.default_rng(67)
    dL = rng.normal(size=(cam.height, cam.width, 3))
    (img * torch.as_tensor(dL, dtype=torch.float32, device="cuda")).sum().backward()
    ref = orender.vjp(scene, cam, dL, agr_weights=w)
    np.testing.assert_allclose(img.detach().cpu().numpy(), ref["image"], rtol=0, atol=COLOUR_TOL)
    got = {k: v.grad.cpu().numpy() for k, v in params.items()}
    got.update({k: v.grad.cpu().numpy() for k, v in wd.items()})
    for k in ("mean7", "L28", "opacity", "sh", "w1", "b1", "w2", "b2"):
        err = np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max()
        assert err <= GRAD_TOL, (k, err)
