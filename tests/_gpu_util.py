"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and fetch results."""
from __future__ import annotations

import numpy as np
import torch

from paper_2503_07946_gb300 import render as prender
from paper_2503_07946_gb300 import sdgs


def gpu_project(scene, cam):
    """sdgs_slice_project on a synth.Scene; returns host copies of the projected record."""
    dev = prender.scene_to_device(scene)
    st = sdgs.scene_struct(dev, scene.lambda_t, scene.lambda_d, scene.dir_mode)
    view = sdgs.view_struct(cam)
    proj = sdgs.ProjectedBuffers(scene.n)
    sdgs.slice_project(st, view, proj)
    torch.cuda.synchronize()
    return dict(mean2d=proj.mean2d.cpu().numpy(), conic_opacity=proj.conic_opacity.cpu().numpy(),
                rgb=proj.rgb.cpu().numpy(), depth=proj.depth.cpu().numpy(), rect=proj.rect_host(),
                radius=proj.radius.cpu().numpy()), (dev, st, view, proj)


def gpu_bin(proj: sdgs.ProjectedBuffers, view, capacity=None):
    n = proj.n
    bins = sdgs.BinBuffers(n, capacity if capacity is not None else max(1024, 64 * max(n, 1)),
                           view.width, view.height)
    k = sdgs.bin_sort(proj, view, bins, sync=True)
    keys = bins.tile_keys[:k].cpu().numpy().view(np.uint32) if k else np.zeros(0, np.uint32)
    vals = bins.point_list[:k].cpu().numpy().view(np.uint32) if k else np.zeros(0, np.uint32)
    ranges = bins.ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    return k, keys, vals, ranges, bins


def gpu_render(proj, bins, view):
    H, W = view.height, view.width
    image = torch.empty(H, W, 3, dtype=torch.float32, device="cuda")
    final_T = torch.empty(H, W, dtype=torch.float32, device="cuda")
    n_contrib = torch.empty(H, W, dtype=torch.int32, device="cuda")
    sdgs.render_fwd(proj, bins, view, image, final_T, n_contrib)
    torch.cuda.synchronize()
    return image.cpu().numpy(), final_T.cpu().numpy(), n_contrib.cpu().numpy()


def oracle_records_f32(g: dict) -> dict:
    """The oracle's own per-Gaussian screen-space record rounded to float32 (culled -> empty rect)."""
    vis = g["visible"].numpy()
    rect = g["rect"].numpy().copy()
    rect[~vis] = 0
    return dict(mean2d=g["mean2d"].detach().numpy().astype(np.float32),
                conic=g["conic"].detach().numpy().astype(np.float32),
                opacity=g["alpha_cond"].detach().numpy().astype(np.float32),
                rgb=g["rgb"].detach().numpy().astype(np.float32),
                depth=np.where(vis, g["depth"].detach().numpy(), 1.0).astype(np.float32),
                rect=rect)


# Decision margins (relative or in pixels) below which an FP32 evaluation may legitimately decide
# the other way from the FP64 oracle.
Z_REL = 1e-5
RADIUS_REL = 2e-6
EDGE_PX = 5e-3
PIX_ALPHA = 1e-4
PIX_T = 1e-4
PIX_DEPTH = 2e-6


def boundary_gaussians(g: dict) -> np.ndarray:
    m = g["margins"]
    vis_any = np.ones(g["visible"].shape[0], bool)
    return vis_any & ((m["z_rel"].numpy() < Z_REL) | (m["radius_rel"].numpy() < RADIUS_REL)
                      | (m["edge_px"].numpy() < EDGE_PX))


def pixel_ok(margin_alpha, margin_T, margin_depth=None, depth_rel=PIX_DEPTH):
    ok = (np.asarray(margin_alpha) >= PIX_ALPHA) & (np.asarray(margin_T) >= PIX_T)
    if margin_depth is not None:
        ok &= np.asarray(margin_depth) >= depth_rel
    return ok


def last_ids(n_contrib: np.ndarray, point_list: np.ndarray, ranges: np.ndarray, tiles_x: int,
             rows=None, cols=None) -> np.ndarray:
    """Id of the last Gaussian each pixel took (-1 if none), from n_contrib and its tile's list.

    Unlike n_contrib (a list position) this does not depend on which skipped candidates a tile
    list holds, so it compares with the oracle's rectangle lists.  rows / cols select pixels of a
    full image; by default n_contrib is the whole image [H, W].
    """
    nc = np.asarray(n_contrib, np.int64)
    if rows is None:
        rows, cols = np.meshgrid(np.arange(nc.shape[0]), np.arange(nc.shape[1]), indexing="ij")
    else:
        nc = nc[rows, cols]
    tile = (np.asarray(rows) // 16) * tiles_x + np.asarray(cols) // 16
    pl = np.asarray(point_list).view(np.uint32).astype(np.int64)
    pos = np.asarray(ranges, np.int64)[tile, 0] + nc - 1
    return np.where(nc > 0, pl[np.clip(pos, 0, max(len(pl) - 1, 0))], -1)


def dropped_pair_alpha(g: dict, cam, tiles, lists: dict, exclude=()) -> tuple[float, int]:
    """Brute force over the (tile, Gaussian) pairs that the rectangle rule gives but a GPU tile
    list leaves out: the largest alpha_cond exp(power) over the 16 x 16 pixel centres of the tile,
    in float64 from the oracle's record.  Below 1/255 means every pixel would skip the Gaussian.

    lists: tile -> GPU Gaussian ids; Gaussians in `exclude` (their rectangles differ between the
    two sides) are left out.  Also asserts every listed Gaussian's oracle rectangle holds the tile.
    Returns (largest alpha, number of pairs checked)."""
    rect = g["rect"].numpy()
    vis = g["visible"].numpy()
    m2 = g["mean2d"].detach().numpy()
    co = g["conic"].detach().numpy()
    al = g["alpha_cond"].detach().numpy()
    excl = np.zeros(len(rect), bool)
    excl[np.asarray(list(exclude), np.int64)] = True
    worst, pairs = 0.0, 0
    for tile in tiles:
        tx, ty = tile % cam.tiles_x, tile // cam.tiles_x
        inside = vis & (rect[:, 0] <= tx) & (tx < rect[:, 2]) & (rect[:, 1] <= ty) & (ty < rect[:, 3])
        got = np.asarray(lists[tile], np.int64)
        got = got[~excl[got]]
        assert inside[got].all(), (tile, got[~inside[got]])
        miss = np.setdiff1d(np.nonzero(inside & ~excl)[0], got)
        if len(miss) == 0:
            continue
        px, py = np.meshgrid(np.arange(16) + 0.5 + 16 * tx, np.arange(16) + 0.5 + 16 * ty)
        px, py = px.reshape(1, -1), py.reshape(1, -1)
        for c0 in range(0, len(miss), 4096):
            m = miss[c0:c0 + 4096]
            dx, dy = px - m2[m, 0:1], py - m2[m, 1:2]
            power = -0.5 * (co[m, 0:1] * dx * dx + co[m, 2:3] * dy * dy) - co[m, 1:2] * dx * dy
            a = al[m, None] * np.exp(np.minimum(power, 0.0))
            worst = max(worst, float(a.max()))
        pairs += len(miss)
    return worst, pairs


def assert_ranges_equal(got: np.ndarray, want: np.ndarray):
    """Tile ranges: counts everywhere, starts of non-empty tiles (an empty range may sit anywhere)."""
    got, want = np.asarray(got, np.int64), np.asarray(want, np.int64)
    np.testing.assert_array_equal(got[:, 1] - got[:, 0], want[:, 1] - want[:, 0])
    busy = want[:, 1] > want[:, 0]
    np.testing.assert_array_equal(got[busy], want[busy])
