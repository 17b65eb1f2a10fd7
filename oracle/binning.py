"""Tile binning by a stable sort on (tile, depth) keys (oracle, NumPy).

A visible Gaussian emits one instance per tile of its rectangle, in Gaussian-id order; the
instance list is sorted by the 64-bit key tile_id << 32 | bits(float32 depth), stable, so equal
keys keep ascending Gaussian id (the 3DGS tile sort the paper's rasteriser relies on, Sec. 4.4).
tile_id = ty * Tx + tx.  Tile ranges are the [start, end) spans of each tile in the sorted list.

Tiles of the rectangle where the Gaussian cannot reach alpha >= 1/255 at any pixel are dropped
(`tile_reachable`).  The rule is a conservative bound: a dropped tile's pixels would all skip the
Gaussian, so the image is the same with or without it.  It decides which (tile, Gaussian)
instances exist, an integer outcome, so it is evaluated in float32 with correctly rounded
operations only (+ - * / sqrt, no fused multiply-add), in the order written below, exactly as the
CUDA binning evaluates it.
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


def _q(a, b, c, dx, dy):
    """a dx^2 + 2 b dx dy + c dy^2, float32, in this rounding order."""
    return ((a * dx) * dx + ((F32(2.0) * b) * dx) * dy) + (c * dy) * dy


def tile_reachable(mean2d, conic, alpha, tx, ty) -> np.ndarray:
    """Whether a pixel of tile (tx, ty) may see alpha >= 1/255 from each Gaussian (vectorised).

    q_min = min over the box of pixel centres [16 tx + 0.5, 16 tx + 15.5] x [...] of
    a dx^2 + 2b dx dy + c dy^2.  It is 0 when the mean is inside the box.  Otherwise the minimum of
    this convex form lies on an edge that faces the mean (the segment from the mean to any point
    of the box first crosses such an edge, and the form grows along it), so only the facing x edge
    (left if u < x0, right if u > x1) and the facing y edge are evaluated, each at its clamped
    stationary point dy = clamp((-b / c) dx) or dx = clamp((-b / a) dy).  The tile is dropped when
    q_min (1 - m) > 2 ln(255 alpha)_bound + 1e-3, m = 1e-4 + 64 * 2^-24 (ac + b^2) / (ac - b^2)
    (the relative FP32 error of the quadratic form grows with that ratio), unless ac - b^2 <= 0 or
    m >= 1/2 (never dropped).
    """
    u = np.asarray(mean2d[..., 0], F32)
    v = np.asarray(mean2d[..., 1], F32)
    a = np.asarray(conic[..., 0], F32)
    b = np.asarray(conic[..., 1], F32)
    c = np.asarray(conic[..., 2], F32)
    x0 = (np.asarray(tx, np.int64) * 16).astype(F32) + F32(0.5)
    x1 = x0 + F32(15.0)
    y0 = (np.asarray(ty, np.int64) * 16).astype(F32) + F32(0.5)
    y1 = y0 + F32(15.0)
    with np.errstate(all="ignore"):
        lo_x, hi_x, lo_y, hi_y = u < x0, u > x1, v < y0, v > y1
        facing_x, facing_y = lo_x | hi_x, lo_y | hi_y
        ex0, ex1, ey0, ey1 = x0 - u, x1 - u, y0 - v, y1 - v
        sx, sy = (-b) / c, (-b) / a  # slopes of the stationary points: dy* = sx dx, dx* = sy dy
        dx = np.where(lo_x, ex0, ex1)
        qx = _q(a, b, c, dx, np.fmin(ey1, np.fmax(ey0, sx * dx)))
        dy = np.where(lo_y, ey0, ey1)
        qy = _q(a, b, c, np.fmin(ex1, np.fmax(ex0, sy * dy)), dy)
        best = np.fmin(np.where(facing_x, qx, F32(np.inf)), np.where(facing_y, qy, F32(np.inf)))
        qmin = np.where(facing_x | facing_y, np.fmax(best, F32(0.0)), F32(0.0))
        ac = a * c
        bb = b * b
        det = ac - bb
        m = F32(1e-4) + F32(64.0 * 2.0 ** -24) * ((ac + bb) / det)
        thr = alpha_exponent_bound(alpha)
        drop = (det > F32(0.0)) & (m < F32(0.5)) & (qmin * (F32(1.0) - m) > thr + F32(1e-3))
    return ~drop


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
