"""Parity of the CUDA forward path (through the C ABI) with the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from oracle import binning, render
import _gpu_util as U

pytestmark = pytest.mark.gpu

COLOUR_TOL = 2e-4  # max-abs per channel, FP32 CUDA vs FP64 oracle


def _cams():
    """Config 0's camera, a rotated ragged-size camera, and a config-1-like camera."""
    c0 = synth.config_cameras(0)[0]
    c1 = synth.make_camera((1.2, -0.8, -2.6), 141, 97, 55.0, 0.3, bg=(0.2, 0.4, 0.6))
    c2 = synth.config_cameras(1, count=1, width=160, height=120)[0]
    return [c0, c1, c2]


@pytest.fixture(scope="module")
def scene0():
    return synth.config_scene(0)


@pytest.mark.parametrize("ci,dir_mode", [(0, 0), (1, 0), (2, 0), (1, 1)])
def test_slice_project_records(scene0, ci, dir_mode):
    cam = _cams()[ci]
    scene0 = scene0.subset(np.arange(scene0.n))
    scene0.dir_mode = dir_mode
    got, _ = U.gpu_project(scene0, cam)
    g = render.gaussians(render.params_from_scene(scene0), cam, scene0.lambda_t, scene0.lambda_d, dir_mode)
    vis_o = g["visible"].numpy()
    vis_g = (got["rect"][:, 2] > got["rect"][:, 0]) & (got["rect"][:, 3] > got["rect"][:, 1])
    border = U.boundary_gaussians(g)
    assert np.array_equal(vis_o[~border], vis_g[~border])
    both = vis_o & vis_g & ~border
    assert both.sum() > 100
    np.testing.assert_array_equal(got["rect"][both], g["rect"].numpy()[both])
    np.testing.assert_array_equal(got["radius"][both], g["radius"].numpy()[both].astype(np.int32))
    np.testing.assert_allclose(got["mean2d"][both], g["mean2d"].numpy()[both], rtol=0, atol=1e-3)
    np.testing.assert_allclose(got["depth"][both], g["depth"].numpy()[both], rtol=4e-6)
    co = got["conic_opacity"][both]
    cref = g["conic"].numpy()[both]
    scale = np.abs(cref).max(1, keepdims=True)
    np.testing.assert_allclose(co[:, :3] / scale, cref / scale, rtol=0, atol=1e-4)
    np.testing.assert_allclose(co[:, 3], g["alpha_cond"].numpy()[both], rtol=2e-5, atol=1e-7)
    np.testing.assert_allclose(got["rgb"][both], g["rgb"].numpy()[both], rtol=0, atol=2e-5)


def _random_bin_cases():
    return [
        (0, 64, 64, 0),          # no Gaussians
        (1, 16, 16, 1),          # one tile: one row, no row pass
        (300, 100, 70, 2),       # ragged image, 7 x 5 tiles
        (5000, 256, 256, 3),     # several radix blocks of Gaussians
        (20000, 1352, 1014, 4),  # 85 x 64 tiles, the row spans of many sort blocks
        (3000, 1920, 1080, 5),   # 8160 tiles
        (600_000, 800, 800, 6),  # hundreds of sort tiles in both sorts
        (16000, 48, 32, 9),      # tile lists of 8.8k-10k instances
        (20000, 2048, 2048, 8),  # 128 x 128 tiles
        (2000, 16, 600, 12),     # one tile column
        (3000, 4096, 48, 13),    # 256 tiles per row: the widest rows of span binning
        (4000, 4224, 64, 10),    # 264 tiles per row: instance records and the tile radix sort
        (4000, 64, 4224, 11),    # 264 tile rows: instance records and the tile radix sort
    ]


@pytest.mark.parametrize("n,W,H,seed", _random_bin_cases())
def test_bin_sort_bit_exact_on_random_records(n, W, H, seed):
    rec = synth.random_projected(n, W, H, seed=seed, max_half_tiles=3 if W < 100 else (12 if n < 100_000 else 2))
    proj = U.sdgs.ProjectedBuffers.from_host(rec)
    view = U.sdgs.view_struct(synth.make_camera((0, 0, -3), W, H, 60.0, 0.5))
    okeys, ovals = binning.sort_keys(rec["depth"], rec["rect"], (W + 15) // 16,
                                     cull=(rec["mean2d"], rec["conic"], rec["opacity"]))
    k, keys, vals, ranges, _ = U.gpu_bin(proj, view, capacity=len(okeys) + 7)
    assert k == len(okeys)
    np.testing.assert_array_equal(keys.astype(np.uint64), okeys >> np.uint64(32))
    np.testing.assert_array_equal(vals, ovals)
    tiles = ((W + 15) // 16) * ((H + 15) // 16)
    U.assert_ranges_equal(ranges, binning.tile_ranges(okeys, tiles))


def test_bin_sort_bit_exact_with_long_spans():
    """Gaussians up to 81 tiles wide: chunks of the span expansion with more instances than its
    shared-memory stage, which write their lists in place."""
    W, H = 1024, 256
    rec = synth.random_projected(6000, W, H, seed=15, max_half_tiles=40, empty_frac=0.0)
    rec["conic"][:] = np.array([1e-4, 0.0, 1e-4], np.float32)  # wide, reaching every tile of the rectangle
    proj = U.sdgs.ProjectedBuffers.from_host(rec)
    view = U.sdgs.view_struct(synth.make_camera((0, 0, -3), W, H, 60.0, 0.5))
    okeys, ovals = binning.sort_keys(rec["depth"], rec["rect"], W // 16,
                                     cull=(rec["mean2d"], rec["conic"], rec["opacity"]))
    k, keys, vals, ranges, _ = U.gpu_bin(proj, view, capacity=len(okeys) + 7)
    assert k == len(okeys)
    np.testing.assert_array_equal(keys.astype(np.uint64), okeys >> np.uint64(32))
    np.testing.assert_array_equal(vals, ovals)
    U.assert_ranges_equal(ranges, binning.tile_ranges(okeys, (W // 16) * (H // 16)))


def test_bin_sort_overflow_is_reported_and_safe():
    rec = synth.random_projected(2000, 256, 256, seed=7)
    proj = U.sdgs.ProjectedBuffers.from_host(rec)
    view = U.sdgs.view_struct(synth.make_camera((0, 0, -3), 256, 256, 60.0, 0.5))
    okeys, _ = binning.sort_keys(rec["depth"], rec["rect"], 16,
                                 cull=(rec["mean2d"], rec["conic"], rec["opacity"]))
    with pytest.raises(U.sdgs.SdgsError) as e:
        U.gpu_bin(proj, view, capacity=len(okeys) // 3)
    assert e.value.code == 3
    # the truncated lists still render without faulting
    bins = U.sdgs.BinBuffers(2000, len(okeys) // 3, 256, 256)
    U.sdgs.bin_sort(proj, view, bins, sync=False)
    U.gpu_render(proj, bins, view)
    k, _, _, _, _ = U.gpu_bin(proj, view, capacity=len(okeys))
    assert k == len(okeys)


@pytest.mark.parametrize("frac", [5, 40])
def test_bin_sort_overflow_keeps_the_nearest_instances(frac):
    """With K > capacity the lists hold the first `capacity` instances in emission order (Gaussians
    by (float32 depth, id), each rectangle's kept tiles row-major), sorted by tile.  A small
    capacity also leaves the kept-tile bitmask too small for the later Gaussians, whose tiles are
    then tested a second time while writing: both ways must give the same lists."""
    W, H = 1352, 1014
    rec = synth.random_projected(20000, W, H, seed=4, max_half_tiles=12)
    proj = U.sdgs.ProjectedBuffers.from_host(rec)
    view = U.sdgs.view_struct(synth.make_camera((0, 0, -3), W, H, 60.0, 0.5))
    tile, gid = binning.instances(rec["rect"], (W + 15) // 16, cull=(rec["mean2d"], rec["conic"], rec["opacity"]))
    dbits = np.asarray(rec["depth"], np.float32).view(np.uint32)
    emitted = np.argsort(dbits[gid], kind="stable")  # Gaussian-id order, then rows, kept among ties
    cap = len(tile) // frac
    first = emitted[:cap]
    by_tile = first[np.argsort(tile[first], kind="stable")]
    bins = U.sdgs.BinBuffers(proj.n, cap, W, H)
    with pytest.raises(U.sdgs.SdgsError) as e:
        U.sdgs.bin_sort(proj, view, bins, sync=True)
    assert e.value.code == 3
    np.testing.assert_array_equal(bins.point_list.cpu().numpy().view(np.uint32), gid[by_tile])
    np.testing.assert_array_equal(bins.tile_keys.cpu().numpy().view(np.uint32), tile[by_tile])
    tiles = ((W + 15) // 16) * ((H + 15) // 16)
    keys = tile[by_tile].astype(np.uint64) << np.uint64(32)
    U.assert_ranges_equal(bins.ranges.cpu().numpy().view(np.uint32).astype(np.int64),
                          binning.tile_ranges(keys, tiles))


@pytest.mark.parametrize("ci", [0, 1, 2])
def test_bin_and_render_on_oracle_records(scene0, ci):
    """Binning + compositing given the oracle's float32-rounded screen-space records."""
    cam = _cams()[ci]
    g = render.gaussians(render.params_from_scene(scene0), cam, scene0.lambda_t, scene0.lambda_d)
    rec = U.oracle_records_f32(g)
    proj = U.sdgs.ProjectedBuffers.from_host(rec)
    view = U.sdgs.view_struct(cam)
    k, keys, vals, ranges, bins = U.gpu_bin(proj, view)
    okeys, ovals = binning.sort_keys(rec["depth"], rec["rect"], cam.tiles_x,
                                     cull=(rec["mean2d"], rec["conic"], rec["opacity"]))
    assert k == len(okeys) and k > 0
    np.testing.assert_array_equal(vals, ovals)
    np.testing.assert_array_equal(keys.astype(np.uint64), okeys >> np.uint64(32))
    img, T, nc = U.gpu_render(proj, bins, view)
    # the oracle composites over the rectangle lists (no reachability filter)
    ref = render.render_projected(rec, cam.width, cam.height, cam.bg)
    ok = U.pixel_ok(ref["margin_alpha"].numpy(), ref["margin_T"].numpy())
    assert ok.mean() > 0.99
    err = np.abs(img - ref["image"].numpy()).max(-1)
    assert err[ok].max() <= COLOUR_TOL, err[ok].max()
    np.testing.assert_allclose(T[ok], ref["final_T"].numpy()[ok], atol=COLOUR_TOL)
    last = U.last_ids(nc, bins.point_list.cpu().numpy(), ranges, cam.tiles_x)
    np.testing.assert_array_equal(last[ok], ref["last_id"].numpy()[ok])
    # n_contrib is a position in the binned list: equal to the oracle's over the filtered lists
    kept = render.render_projected(rec, cam.width, cam.height, cam.bg, reach=True)
    np.testing.assert_array_equal(nc[ok], kept["n_contrib"].numpy()[ok])


@pytest.mark.parametrize("ci", [0, 1, 2])
def test_render_end_to_end_against_fp64_oracle(scene0, ci):
    cam = _cams()[ci]
    got, (dev, st, view, proj) = U.gpu_project(scene0, cam)
    k, _, _, _, bins = U.gpu_bin(proj, view)
    img, T, nc = U.gpu_render(proj, bins, view)
    ref = render.render(scene0, cam)
    g = ref["g"]
    # A Gaussian whose tile rectangle FP32 decides differently must lie within the FP32 margin of
    # a decision boundary; the tiles where the two rectangles differ are set aside.
    orect = g["rect"].numpy()
    differ = np.nonzero((got["rect"] != orect).any(1))[0]
    assert U.boundary_gaussians(g)[differ].all(), differ
    excl = np.zeros((cam.tiles_y, cam.tiles_x), bool)
    for i in differ:
        a = np.zeros_like(excl)
        b = np.zeros_like(excl)
        a[got["rect"][i, 1]:got["rect"][i, 3], got["rect"][i, 0]:got["rect"][i, 2]] = True
        b[orect[i, 1]:orect[i, 3], orect[i, 0]:orect[i, 2]] = True
        excl |= a ^ b
    excl_pix = np.kron(excl, np.ones((16, 16), bool))[:cam.height, :cam.width]
    ok = U.pixel_ok(ref["margin_alpha"].numpy(), ref["margin_T"].numpy(), ref["margin_depth"].numpy())
    ok &= ~excl_pix
    assert ok.mean() > 0.99, ok.mean()
    err = np.abs(img - ref["image"].numpy()).max(-1)
    assert err[ok].max() <= COLOUR_TOL, err[ok].max()
    # the oracle's lists are the rectangle lists, so compare who contributed last, not where
    last = U.last_ids(nc, bins.point_list.cpu().numpy(), bins.ranges.cpu().numpy().view(np.uint32), cam.tiles_x)
    np.testing.assert_array_equal(last[ok], ref["last_id"].numpy()[ok])


@pytest.mark.parametrize("ci", [0, 1, 2])
def test_dropped_pairs_reach_no_pixel(scene0, ci):
    """Every (tile, Gaussian) pair of the oracle's rectangles that the CUDA binning leaves out of a
    tile list is one that no pixel centre of the tile takes: float64 alpha < 1/255 at all 256
    centres, by brute force, on every tile of the image."""
    cam = _cams()[ci]
    got, (dev, st, view, proj) = U.gpu_project(scene0, cam)
    k, _, vals, ranges, bins = U.gpu_bin(proj, view)
    g = render.gaussians(render.params_from_scene(scene0), cam, scene0.lambda_t, scene0.lambda_d)
    differ = np.nonzero((got["rect"] != g["rect"].numpy()).any(1))[0]
    assert U.boundary_gaussians(g)[differ].all(), differ
    vals = vals.astype(np.int64)
    tiles = range(cam.tiles_x * cam.tiles_y)
    lists = {t: vals[ranges[t, 0]:ranges[t, 1]] for t in tiles}
    worst, pairs = U.dropped_pair_alpha(g, cam, tiles, lists, exclude=differ)
    assert pairs > k // 2, (pairs, k)  # the rule drops a large share of the rectangle pairs
    assert worst < 1.0 / 255.0, worst


def test_renderer_deferred_check_matches_and_grows(scene0):
    """Renderer(deferred_check=True) renders the frames of the synchronising renderer; a frame
    that exceeded the capacity is reported at the next forward, which grows the bins first."""
    import warnings as _w
    from paper_2503_07946_gb300 import render as prender
    cam = _cams()[1]
    dev = prender.scene_to_device(scene0)
    st = U.sdgs.scene_struct(dev, scene0.lambda_t, scene0.lambda_d)
    view = U.sdgs.view_struct(cam)
    ref_r = prender.Renderer(scene0.n, cam.width, cam.height)
    ref = ref_r.forward(st, view).clone()
    k = ref_r.num_instances
    r = prender.Renderer(scene0.n, cam.width, cam.height, deferred_check=True)
    with _w.catch_warnings():
        _w.simplefilter("error")
        for _ in range(2):
            img = r.forward(st, view).clone()
            assert torch.equal(img, ref)
    assert not r.check_deferred() and r.num_instances == k and r.overflowed_frames == 0
    small = prender.Renderer(scene0.n, cam.width, cam.height, capacity=k // 4, deferred_check=True)
    small.forward(st, view)  # truncated to the nearest k // 4 instances
    with pytest.warns(RuntimeWarning):
        img = small.forward(st, view).clone()
    assert small.overflowed_frames == 1 and small.bins.capacity >= k
    assert torch.equal(img, ref)
    assert not small.check_deferred() and small.num_instances == k


def test_bin_sort_batch_equals_binning_each_problem_alone():
    """sdgs_bin_sort_batch (one launch per step for several problems, as the render server bins
    the requests it admits together) gives every problem exactly the lists, ranges and count of
    sdgs_bin_sort on its own: mixed sizes and tile grids (span binning and, for an image 264 tiles
    wide, instance records), an empty problem, a single-tile image, and an overflowing capacity."""
    cases = [(4000, 4224, 64, 10), (20000, 1352, 1014, 4), (0, 64, 64, 0), (1, 16, 16, 1),
             (3000, 1920, 1080, 5), (16000, 48, 32, 9), (300, 100, 70, 2), (20000, 1352, 1014, 11)]
    projs, views, alone, batch = [], [], [], []
    for n, W, H, seed in cases:
        rec = synth.random_projected(n, W, H, seed=seed, max_half_tiles=3 if W < 100 else 12)
        projs.append(U.sdgs.ProjectedBuffers.from_host(rec))
        views.append(U.sdgs.view_struct(synth.make_camera((0, 0, -3), W, H, 60.0, 0.5)))
    for j, (p, v) in enumerate(zip(projs, views)):
        cap = max(1024, 64 * max(p.n, 1))
        if j == len(cases) - 1:
            cap = 20000  # far below K: the lists keep the nearest `cap` instances
        for dst in (alone, batch):
            dst.append(U.sdgs.BinBuffers(p.n, cap, v.width, v.height))
    ks = []
    for p, v, b in zip(projs, views, alone):
        try:
            ks.append(U.sdgs.bin_sort(p, v, b, sync=True))
        except U.sdgs.SdgsError as e:
            assert e.code == 3
            ks.append(int(b.num_instances.item()))
    with pytest.raises(U.sdgs.SdgsError) as e:  # the last problem overflows
        U.sdgs.bin_sort_batch(projs, views, batch, sync=True)
    assert e.value.code == 3
    torch.cuda.synchronize()
    for j, (a, b) in enumerate(zip(alone, batch)):
        k = int(b.num_instances.item())
        assert k == ks[j], j
        m = min(k, a.capacity)
        assert torch.equal(a.ranges, b.ranges), j
        assert torch.equal(a.point_list[:m], b.point_list[:m]), j
        assert torch.equal(a.tile_keys[:m], b.tile_keys[:m]), j
    # and without the overflow the batch call returns every K
    ks2 = U.sdgs.bin_sort_batch(projs[:-1], views[:-1], batch[:-1], sync=True)
    assert ks2 == ks[:-1]


def test_renderer_on_a_side_stream_matches_the_default_stream(scene0):
    """Renderer.forward(..., stream) runs every call on that stream and gives the same image."""
    from paper_2503_07946_gb300 import render as prender
    cam = _cams()[1]
    dev = prender.scene_to_device(scene0)
    st = U.sdgs.scene_struct(dev, scene0.lambda_t, scene0.lambda_d)
    view = U.sdgs.view_struct(cam)
    ref = prender.Renderer(scene0.n, cam.width, cam.height).forward(st, view).clone()
    side = torch.cuda.Stream()
    r = prender.Renderer(scene0.n, cam.width, cam.height, deferred_check=True)
    with torch.cuda.stream(side):
        for _ in range(2):
            img = r.forward(st, view, side)
    side.synchronize()
    assert torch.equal(img, ref)


def test_clamped_opacities_and_non_positive_definite_records(scene0):
    """Caller-made records.  (1) A tenth of the Gaussians at opacity 0.999, so that the 0.99 clamp
    of alpha acts near their centres and their tiles' batches take the clamped blend: the image
    matches the oracle's.  (2) Records whose conic is not positive definite, in front of
    everything and listed on every tile of the image: every pixel skips them (their exponent could
    otherwise overflow), so the image and transmittance equal those without them, bit for bit."""
    cam = _cams()[0]
    g = render.gaussians(render.params_from_scene(scene0), cam, scene0.lambda_t, scene0.lambda_d)
    rec = U.oracle_records_f32(g)
    rng = np.random.default_rng(7)
    hi = rng.random(len(rec["opacity"])) < 0.1
    rec["opacity"] = np.where(hi, np.float32(0.999), rec["opacity"]).astype(np.float32)
    view = U.sdgs.view_struct(cam)
    proj = U.sdgs.ProjectedBuffers.from_host(rec)
    k, keys, vals, ranges, bins = U.gpu_bin(proj, view)
    img, T, nc = U.gpu_render(proj, bins, view)
    ref = render.render_projected(rec, cam.width, cam.height, cam.bg)
    ok = U.pixel_ok(ref["margin_alpha"].numpy(), ref["margin_T"].numpy())
    assert ok.mean() > 0.99
    assert np.abs(img - ref["image"].numpy()).max(-1)[ok].max() <= COLOUR_TOL
    clamped = (hi[:, None] & (rec["rect"][:, 2] > rec["rect"][:, 0])[:, None]).any()
    assert clamped

    m = 16
    extra = dict(
        mean2d=rng.uniform(0, [cam.width, cam.height], size=(m, 2)).astype(np.float32),
        conic=np.tile(np.array([[-0.01, 0.0, 0.02], [0.01, 0.05, 0.01], [0.0, 0.0, 0.0], [0.3, 0.0, -0.2]],
                               np.float32), (m // 4, 1)),
        opacity=np.full(m, 0.5, np.float32),
        rgb=np.full((m, 3), 0.3, np.float32),
        depth=np.full(m, 0.5 * float(rec["depth"].min()), np.float32),
        rect=np.tile(np.array([[0, 0, cam.tiles_x, cam.tiles_y]], np.int64), (m, 1)))
    rec2 = {key: np.concatenate([rec[key], extra[key]], 0) for key in extra}
    proj2 = U.sdgs.ProjectedBuffers.from_host(rec2)
    k2, _, _, _, bins2 = U.gpu_bin(proj2, view)
    assert k2 >= k + m * cam.tiles_x * cam.tiles_y  # listed on every tile
    img2, T2, _ = U.gpu_render(proj2, bins2, view)
    np.testing.assert_array_equal(img2, img)
    np.testing.assert_array_equal(T2, T)
