"""Tile binning by a stable sort on (tile, depth) keys (oracle, NumPy).

A visible Gaussian emits one instance per tile of its rectangle, in Gaussian-id order; the
instance list is sorted by the 64-bit key tile_id << 32 | bits(float32 depth), stable, so equal
keys keep ascending Gaussian id (the 3DGS tile sort the paper's rasteriser relies on, Sec. 4.4).
tile_id = ty * Tx + tx.  Tile ranges are the [start, end) spans of each tile in the sorted list.

Tiles of the rectangle where the Gaussian cannot reach alpha >= 1/255 at any pixel are dropped
(`tile_reachable`, a span of tiles per row).  The rule is conservative: a dropped tile's pixels
would all skip the Gaussian, so the image is the same with or without it.  It decides which
(tile, Gaussian) instances exist, an integer outcome, so it is evaluated in float32 with
correctly rounded operations only (+ - * / sqrt, no fused multiply-add), in the order written
below, exactly as the CUDA binning evaluates it.
"""
from __future__ import annotations

import numpy as np


F32 = np.float32


def alpha_exponent_bound(alpha: np.ndarray) -> np.ndarray:
    """Upper bound of 2 ln(255 alpha): ln y <= k (y^(1/k) - 1) for k > 0; k = 256, y^(1/256) by eight
    square roots.  Exceeds 2 ln(255 alpha) by at most 1.1% for alpha <= 1.  (fmin / fmax below
    ignore NaN operands, as the C functions do.)"""
    y = F32(255.0) * np.asarray(alpha, F32)
    for _ in range(8):
        y = np.sqrt(y)
    return F32(512.0) * (y - F32(1.0))


def tile_reachable(mean2d, conic, alpha, tx, ty) -> np.ndarray:
    """Whether tile (tx, ty) of a Gaussian's rectangle is kept (vectorised over any shape).

    The row span rule.  With ac - b^2 = det, m = 1e-4 + 2^-18 (ac + b^2) / det (a bound on the
    relative float32 error of the conic's quadratic form) and lim = 2 ln(255 alpha)_bound + 1e-3,
    the ellipse {a dx^2 + 2b dx dy + c dy^2 <= Q}, Q = lim (1 + 8m) / (1 - m), contains every
    pixel centre where alpha_cond exp(-q/2) >= 1/255.  For the tile row ty, whose pixel centres
    span dy in [ey0, ey1] (relative to the mean), the ellipse's x-extent over that band is
    attained at the clamped dy of its rightmost and leftmost points (the extent is concave in dy):
        hx = sqrt(Q c / det), hy = sqrt(Q a / det), dy_r = (-b / c) hx
        d1 = clamp(dy_r, ey0, ey1),  x_max = (-b d1 + sqrt(max(aQ - det d1^2, 0))) / a + pad_x
        d2 = clamp(-dy_r, ey0, ey1), x_min = (-b d2 - sqrt(max(aQ - det d2^2, 0))) / a - pad_x
    with pad_x = 0.05 + 2e-3 hx covering the float32 error of the square roots near the
    ellipse's top and bottom.  The row is empty when the band misses [-hy - pad_y, hy + pad_y]
    (pad_y = 0.05 + 2e-3 hy) and everything is dropped when lim < 0 (alpha < 1/255); otherwise
    the kept tiles are those whose pixel-centre x-range [16 tx + 0.5, 16 tx + 15.5] meets
    [u + x_min, u + x_max]:  ceil((u + x_min - 15.5) / 16) <= tx <= floor((u + x_max - 0.5) / 16).
    Nothing is dropped when det <= 0, m >= 1/2, a <= 0 or lim is NaN.  A NaN bound keeps the row.
    """
    u = np.asarray(mean2d[..., 0], F32)
    v = np.asarray(mean2d[..., 1], F32)
    a = np.asarray(conic[..., 0], F32)
    b = np.asarray(conic[..., 1], F32)
    c = np.asarray(conic[..., 2], F32)
    with np.errstate(all="ignore"):
        ac = a * c
        bb = b * b
        det = ac - bb
        m = F32(1e-4) + F32(2.0 ** -18) * ((ac + bb) / det)
        lim = alpha_exponent_bound(alpha) + F32(1e-3)
        never = ~(det > F32(0.0)) | ~(m < F32(0.5)) | ~(a > F32(0.0)) | (lim != lim)
        Q = (lim * (F32(1.0) + F32(8.0) * m)) / (F32(1.0) - m)
        hx = np.sqrt((Q * c) / det)
        hy = np.sqrt((Q * a) / det)
        dyr = ((-b) / c) * hx
        padx = F32(0.05) + F32(2e-3) * hx
        pady = F32(0.05) + F32(2e-3) * hy
        aQ = a * Q
        y0 = (np.asarray(ty, np.int64) * 16).astype(F32) + F32(0.5)
        ey0 = y0 - v
        ey1 = (y0 + F32(15.0)) - v
        reach_y = hy + pady
        row_hit = ~(ey0 > reach_y) & ~(ey1 < -reach_y)
        d1 = np.fmin(ey1, np.fmax(ey0, dyr))
        x_max = ((-(b * d1)) + np.sqrt(np.fmax(aQ - (det * d1) * d1, F32(0.0)))) / a + padx
        d2 = np.fmin(ey1, np.fmax(ey0, -dyr))
        x_min = ((-(b * d2)) - np.sqrt(np.fmax(aQ - (det * d2) * d2, F32(0.0)))) / a - padx
        lo = np.ceil(((u + x_min) - F32(15.5)) / F32(16.0))
        hi = np.floor(((u + x_max) - F32(0.5)) / F32(16.0))
        txf = np.asarray(tx, np.int64).astype(F32)
        in_span = ~(txf < lo) & ~(txf > hi)
        keep = never | (~(lim < F32(0.0)) & row_hit & in_span)
    return keep


def instances(rect: np.ndarray, tiles_x: int, cull=None, block: int = 65536) -> tuple[np.ndarray, np.ndarray]:
    """(tile_id, gaussian_id) for every instance, emitted in Gaussian-id order, tiles row-major.

    With `cull` = (mean2d, conic, alpha), only reachable tiles are kept; Gaussians are then
    processed `block` at a time to bound memory.
    """
    rect = np.asarray(rect, dtype=np.int64).reshape(-1, 4)
    if cull is not None and rect.shape[0] > block:
        parts = [instances(rect[i:i + block], tiles_x, tuple(np.asarray(x)[i:i + block] for x in cull), block)
                 for i in range(0, rect.shape[0], block)]
        return (np.concatenate([p[0] for p in parts]),
                np.concatenate([p[1] + i for p, i in zip(parts, range(0, rect.shape[0], block))]))
    w = np.clip(rect[:, 2] - rect[:, 0], 0, None)
    h = np.clip(rect[:, 3] - rect[:, 1], 0, None)
    count = w * h
    gid = np.repeat(np.arange(rect.shape[0], dtype=np.int64), count)
    first = np.cumsum(count) - count  # index of each Gaussian's first instance
    k = np.arange(gid.shape[0], dtype=np.int64) - first[gid]  # position inside the rectangle
    tx = rect[gid, 0] + k % w[gid]
    ty = rect[gid, 1] + k // w[gid]
    if cull is not None:  # (mean2d, conic, alpha) as float32: keep only reachable tiles
        mean2d, conic, alpha = (np.asarray(x, F32) for x in cull)
        keep = tile_reachable(mean2d[gid], conic[gid], alpha[gid], tx, ty)
        tx, ty, gid = tx[keep], ty[keep], gid[keep]
    return ty * tiles_x + tx, gid


def sort_keys(depth32: np.ndarray, rect: np.ndarray, tiles_x: int, cull=None):
    """Stable sort of the 64-bit (tile, float32 depth bits) keys; returns keys, values."""
    tile, gid = instances(rect, tiles_x, cull)
    dbits = np.asarray(depth32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    keys = (tile.astype(np.uint64) << np.uint64(32)) | dbits[gid]
    order = np.argsort(keys, kind="stable")
    return keys[order], gid[order].astype(np.uint32)


def tile_ranges(sorted_keys: np.ndarray, num_tiles: int) -> np.ndarray:
    """[num_tiles, 2] int64 (start, end); empty tiles are (0, 0)."""
    ranges = np.zeros((num_tiles, 2), dtype=np.int64)
    tile = (sorted_keys >> np.uint64(32)).astype(np.int64)
    for i in range(tile.shape[0]):
        if i == 0 or tile[i] != tile[i - 1]:
            ranges[tile[i], 0] = i
        if i == tile.shape[0] - 1 or tile[i] != tile[i + 1]:
            ranges[tile[i], 1] = i + 1
    return ranges


def tile_lists(depth: np.ndarray, rect: np.ndarray, tiles_x: int, num_tiles: int, cull=None) -> list:
    """Per tile, the Gaussians whose rectangle contains it (and that may reach it), ordered by
    (depth, id).

    Works for float64 depths as well: this is the same ordering as the key sort but without
    rounding the depth to float32.
    """
    tile, gid = instances(rect, tiles_x, cull)
    order = np.lexsort((gid, np.asarray(depth)[gid], tile))
    tile, gid = tile[order], gid[order]
    bounds = np.searchsorted(tile, np.arange(num_tiles + 1))
    return [gid[bounds[i]:bounds[i + 1]] for i in range(num_tiles)]
