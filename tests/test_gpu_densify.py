"""Densification statistics (Algorithm 1 step 7, Sec. 4.4) of the CUDA path against the FP64
oracle, through the C ABI."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from oracle import densify
from paper_2503_07946_gb300 import render as prender
from paper_2503_07946_gb300 import sdgs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dir_mode", [0, 1])
def test_densify_stats_match_oracle(dir_mode):
    scene = synth.make_scene(20000, seed=43, box=1.0, diag=(0.02, 0.4), off_sigma=0.08)
    scene.opacity[::50] *= 0.01  # some below the pruning threshold
    cam = synth.make_camera((1.0, -0.5, -2.8), 320, 240, 55.0, 0.4)
    extent = 1.7
    dev = prender.scene_to_device(scene)
    st = sdgs.scene_struct(dev, scene.lambda_t, scene.lambda_d, dir_mode)
    got = {k: v.cpu().numpy() for k, v in sdgs.densify_stats(st, sdgs.view_struct(cam), scene.n, extent).items()}
    torch.cuda.synchronize()
    ref = densify.densify_stats(scene.mean7, scene.L28, scene.opacity, cam.t, cam.d, scene.lambda_t,
                                scene.lambda_d, extent, dir_mode=dir_mode, center=np.asarray(cam.center))
    S, Sr = got["scale"], ref["scale"]
    # scales: relative to the largest scale of each Gaussian (FP32 slicing of Sigma_cond)
    np.testing.assert_allclose(S / Sr[:, :1], Sr / Sr[:, :1], rtol=0, atol=2e-4)
    R = got["rot"]
    np.testing.assert_allclose(np.einsum("nij,nik->njk", R, R), np.broadcast_to(np.eye(3), R.shape), atol=2e-5)
    np.testing.assert_allclose(np.linalg.det(R.astype(np.float64)), 1.0, atol=5e-5)
    # the axes are unique up to sign where the scales are well separated
    gap = np.minimum(Sr[:, 0] - Sr[:, 1], Sr[:, 1] - Sr[:, 2]) / Sr[:, 0]
    sep = gap > 0.05
    assert sep.sum() > scene.n // 2
    for j in range(3):
        c = np.abs(np.einsum("ni,ni->n", R[sep, :, j], ref["rot"][sep, :, j]))
        assert np.all(c > 1 - 1e-4), (j, c.min())
    # R diag(S)^2 R^T reproduces Sigma_cond
    rec = np.einsum("nij,nj,nkj->nik", R.astype(np.float64), S.astype(np.float64) ** 2, R.astype(np.float64))
    scale = Sr[:, 0] ** 2
    assert np.max(np.abs(rec - ref["Sigma_cond"]) / scale[:, None, None]) < 5e-4
    np.testing.assert_allclose(got["pt_norm"], ref["pt_norm"], rtol=2e-5, atol=1e-7)
    np.testing.assert_allclose(got["t_scale"], ref["t_scale"], rtol=2e-6)
    # the decisions agree away from their thresholds
    near = (np.abs(ref["pt_norm"] - 0.05 * extent) < 1e-5) | (np.abs(ref["t_scale"] - 0.25) < 1e-5)
    np.testing.assert_array_equal(got["split"][~near], ref["split"][~near])
    assert ref["split"].any() and not ref["split"].all()
    np.testing.assert_array_equal(got["prune"], ref["prune"])
    assert ref["prune"].sum() >= 100
