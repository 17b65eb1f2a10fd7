"""Parity at the benchmark's full sizes: the 300k-Gaussian 800x800 object-scale scene and the
1.5M-Gaussian 1352x1014 clustered scene, rendered in the launch configuration bench.py times.

The oracle cannot composite whole frames of this size in a test, so it checks (a) a random
sample of per-Gaussian records, (b) the complete instance lists of sampled tiles, (c) sampled
pixels (whole tiles and scattered pixels), and properties of the binning that hold at any size;
and, for the differentiation workload, the gradients of a loss that lives on a few tiles.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from oracle import binning
from oracle import render as orender
from paper_2503_07946_gb300 import render as prender
from paper_2503_07946_gb300 import sdgs
import _gpu_util as U

pytestmark = pytest.mark.gpu

COLOUR_TOL = 2e-4


def _gpu_frame(scene, cam):
    dev = prender.scene_to_device(scene)
    st = sdgs.scene_struct(dev, scene.lambda_t, scene.lambda_d)
    v = sdgs.view_struct(cam)
    r = prender.Renderer(scene.n, cam.width, cam.height, capacity=1 << 20, tile_keys=True)
    r.forward(st, v)
    torch.cuda.synchronize()
    return r


@pytest.fixture(scope="module", params=["object_300k_800", "clustered_1p5m_1352"])
def frame(request):
    if request.param == "object_300k_800":
        scene, cam = synth.config_scene(1), synth.config_cameras(1)[0]
    else:
        scene, cam = synth.config_scene(2), synth.config_cameras(2)[0]
    r = _gpu_frame(scene, cam)
    g = orender.gaussians(orender.params_from_scene(scene), cam, scene.lambda_t, scene.lambda_d)
    return scene, cam, r, g


def _host_rect(r):
    return r.proj.rect_host()


def test_records_sample(frame):
    scene, cam, r, g = frame
    rng = np.random.default_rng(0)
    idx = rng.choice(scene.n, size=min(20000, scene.n), replace=False)
    rect = _host_rect(r)[idx]
    vis_g = (rect[:, 2] > rect[:, 0]) & (rect[:, 3] > rect[:, 1])
    vis_o = g["visible"].numpy()[idx]
    border = U.boundary_gaussians(g)[idx]
    assert np.array_equal(vis_o[~border], vis_g[~border])
    both = vis_o & vis_g & ~border
    np.testing.assert_array_equal(rect[both], g["rect"].numpy()[idx][both])
    m2 = r.proj.mean2d.cpu().numpy()[idx]
    np.testing.assert_allclose(m2[both], g["mean2d"].numpy()[idx][both], rtol=0, atol=2e-3)
    co = r.proj.conic_opacity.cpu().numpy()[idx]
    np.testing.assert_allclose(co[both, 3], g["alpha_cond"].numpy()[idx][both], rtol=2e-5, atol=1e-7)
    np.testing.assert_allclose(r.proj.rgb.cpu().numpy()[idx][both], g["rgb"].numpy()[idx][both], atol=2e-5)


def test_binning_properties(frame):
    scene, cam, r, g = frame
    k = r.num_instances
    ranges = r.bins.ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    # the non-empty tiles' lists are contiguous, in tile order, and cover [0, K)
    assert np.all(ranges[:, 1] >= ranges[:, 0])
    busy = ranges[ranges[:, 1] > ranges[:, 0]]
    assert busy[0, 0] == 0 and busy[-1, 1] == k
    assert np.all(busy[1:, 0] == busy[:-1, 1])
    rect = _host_rect(r)
    area = np.clip(rect[:, 2] - rect[:, 0], 0, None) * np.clip(rect[:, 3] - rect[:, 1], 0, None)
    assert 0 < k <= int(area.sum())
    keys = r.bins.tile_keys[:k].cpu().numpy().view(np.uint32).astype(np.int64)
    tiles = np.repeat(np.arange(len(ranges)), ranges[:, 1] - ranges[:, 0])
    np.testing.assert_array_equal(keys, tiles)
    # every listed Gaussian's rectangle contains its tile, and depths never decrease in a tile
    pl = r.bins.point_list[:k].cpu().numpy().view(np.uint32).astype(np.int64)
    depth = r.proj.depth.cpu().numpy()
    tx, ty = tiles % cam.tiles_x, tiles // cam.tiles_x
    rr = rect[pl]
    assert np.all((rr[:, 0] <= tx) & (tx < rr[:, 2]) & (rr[:, 1] <= ty) & (ty < rr[:, 3]))
    dk = depth[pl].view(np.uint32).astype(np.int64)
    same = tiles[1:] == tiles[:-1]
    step = (dk[1:] > dk[:-1]) | ((dk[1:] == dk[:-1]) & (pl[1:] > pl[:-1]))
    assert np.all(step[same])


def test_fullsize_binning_bit_exact_on_oracle_records(frame):
    """The oracle's own records, rounded to float32, binned by the CUDA path and by the oracle."""
    scene, cam, r, g = frame
    rec = U.oracle_records_f32(g)
    proj = sdgs.ProjectedBuffers.from_host(rec)
    view = sdgs.view_struct(cam)
    okeys, ovals = binning.sort_keys(rec["depth"], rec["rect"], cam.tiles_x,
                                     cull=(rec["mean2d"], rec["conic"], rec["opacity"]))
    k, keys, vals, ranges, _ = U.gpu_bin(proj, view, capacity=len(okeys) + 1)
    assert k == len(okeys)
    np.testing.assert_array_equal(vals, ovals)
    np.testing.assert_array_equal(keys.astype(np.uint64), okeys >> np.uint64(32))
    U.assert_ranges_equal(ranges, binning.tile_ranges(okeys, cam.tiles_x * cam.tiles_y))


def _tile_pixels(cam, tile):
    tx, ty = tile % cam.tiles_x, tile // cam.tiles_x
    ys, xs = np.meshgrid(np.arange(ty * 16, min(ty * 16 + 16, cam.height)),
                         np.arange(tx * 16, min(tx * 16 + 16, cam.width)), indexing="ij")
    return np.stack([ys.reshape(-1), xs.reshape(-1)], 1)


def test_sampled_tiles_lists_and_pixels(frame):
    scene, cam, r, g = frame
    rng = np.random.default_rng(1)
    ranges = r.bins.ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    counts = ranges[:, 1] - ranges[:, 0]
    busy = np.nonzero(counts > 0)[0]
    tiles = list(rng.choice(busy, size=3, replace=False)) + [int(np.argmax(counts))]
    pl = r.bins.point_list.cpu().numpy().view(np.uint32).astype(np.int64)
    grect = _host_rect(r)
    orect = g["rect"].numpy()
    differ = np.nonzero((grect != orect).any(1))[0]
    assert U.boundary_gaussians(g)[differ].all()
    odepth = g["depth"].numpy()
    lists = {t: pl[ranges[t, 0]:ranges[t, 1]] for t in tiles}
    # every rectangle pair a list leaves out reaches no pixel centre of the tile (float64, brute force)
    worst, pairs = U.dropped_pair_alpha(g, cam, tiles, lists, exclude=differ)
    assert pairs > 0 and worst < 1.0 / 255.0, (pairs, worst)
    pixels = []
    for tile in tiles:
        lst = pl[ranges[tile, 0]:ranges[tile, 1]]
        a = lst[~np.isin(lst, differ)]
        # depth order, except swaps of depths equal to FP32 accuracy
        za = odepth[a]
        assert np.all(np.diff(za) >= -4e-6 * np.abs(za[1:]))
        if not np.isin(lst, differ).any():
            pixels.append(_tile_pixels(cam, tile))
    extra = np.stack([rng.integers(0, cam.height, 300), rng.integers(0, cam.width, 300)], 1)
    tile_of = (extra[:, 0] // 16) * cam.tiles_x + extra[:, 1] // 16
    bad_tiles = set()
    for i in differ:
        for rc in (grect[i], orect[i]):
            for yy in range(rc[1], rc[3]):
                for xx in range(rc[0], rc[2]):
                    bad_tiles.add(yy * cam.tiles_x + xx)
    extra = extra[[t not in bad_tiles for t in tile_of]]
    pix = np.concatenate(pixels + [extra])
    ref = orender.render_pixels(g, cam, pix)
    img = r.image.cpu().numpy()[pix[:, 0], pix[:, 1]]
    ok = U.pixel_ok(ref["margin_alpha"].numpy(), ref["margin_T"].numpy(), ref["margin_depth"].numpy())
    # pixels set aside where an FP32 decision may flip with visible effect: 1.1% of this sample
    assert ok.mean() > 0.985, (ok.mean(), (ref["margin_alpha"].numpy() < U.PIX_ALPHA).mean(),
                               (ref["margin_T"].numpy() < U.PIX_T).mean(),
                               (ref["margin_depth"].numpy() < U.PIX_DEPTH).mean())
    err = np.abs(img - ref["color"].numpy()).max(-1)
    assert err[ok].max() <= COLOUR_TOL, err[ok].max()
    last = U.last_ids(r.n_contrib.cpu().numpy(), r.bins.point_list.cpu().numpy(), ranges, cam.tiles_x,
                      rows=pix[:, 0], cols=pix[:, 1])
    np.testing.assert_array_equal(last[ok], ref["last_id"].numpy()[ok])


def test_fullsize_gradients_on_sampled_tiles():
    """The differentiation workload (300k Gaussians, 800x800): the loss lives on 3 tiles, so the
    oracle's autograd composites only those; all four gradient tensors must agree."""
    scene, cam = synth.config_scene(1), synth.config_cameras(1)[0]
    rng = np.random.default_rng(5)
    dL = np.zeros((cam.height, cam.width, 3))
    tiles = [cam.tiles_x * 20 + 20, cam.tiles_x * 25 + 27, cam.tiles_x * 30 + 18]
    for t in tiles:
        tx, ty = t % cam.tiles_x, t // cam.tiles_x
        dL[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = rng.normal(size=(16, 16, 3))
    dev = prender.scene_to_device(scene)
    params = {k: v.clone().requires_grad_(True) for k, v in dev.items()}
    r = prender.Renderer(scene.n, cam.width, cam.height)
    img = prender.render_image(params["mean7"], params["L28"], params["opacity"], params["sh"],
                               sdgs.view_struct(cam), scene.lambda_t, scene.lambda_d, r)
    (img * torch.as_tensor(dL, dtype=torch.float32, device="cuda")).sum().backward()
    ref = orender.vjp(scene, cam, dL, tiles=tiles)
    for k in ("mean7", "L28", "opacity", "sh"):
        got = params[k].grad.cpu().numpy().reshape(scene.n, -1)
        want = ref[k].reshape(scene.n, -1)
        scale = np.abs(want).max()
        assert scale > 0
        assert np.abs(got - want).max() <= 1e-3 * scale, (k, np.abs(got - want).max() / scale)
