"""Tile binning by a stable sort on (tile, depth) keys (oracle, NumPy).

A visible Gaussian emits one instance per tile of its rectangle, in Gaussian-id order; the
instance list is sorted by the 64-bit key tile_id << 32 | bits(float32 depth), stable, so equal
keys keep ascending Gaussian id (the 3DGS tile sort the paper's rasteriser relies on, Sec. 4.3).
tile_id = ty * Tx + tx.  Tile ranges are the [start, end) spans of each tile in the sorted list.
"""
from __future__ import annotations

import numpy as np


def instances(rect: np.ndarray, tiles_x: int) -> tuple[np.ndarray, np.ndarray]:
    """(tile_id, gaussian_id) for every instance, emitted in Gaussian-id order, tiles row-major."""
    rect = np.asarray(rect, dtype=np.int64).reshape(-1, 4)
    w = np.clip(rect[:, 2] - rect[:, 0], 0, None)
    h = np.clip(rect[:, 3] - rect[:, 1], 0, None)
    count = w * h
    gid = np.repeat(np.arange(rect.shape[0], dtype=np.int64), count)
    first = np.cumsum(count) - count  # index of each Gaussian's first instance
    k = np.arange(gid.shape[0], dtype=np.int64) - first[gid]  # position inside the rectangle
    tx = rect[gid, 0] + k % w[gid]
    ty = rect[gid, 1] + k // w[gid]
    return ty * tiles_x + tx, gid


def sort_keys(depth32: np.ndarray, rect: np.ndarray, tiles_x: int):
    """Stable sort of the 64-bit (tile, float32 depth bits) keys; returns keys, values."""
    tile, gid = instances(rect, tiles_x)
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


def tile_lists(depth: np.ndarray, rect: np.ndarray, tiles_x: int, num_tiles: int) -> list:
    """Per tile, the Gaussians whose rectangle contains it, ordered by (depth, id).

    Works for float64 depths as well: this is the same ordering as the key sort but without
    rounding the depth to float32.
    """
    tile, gid = instances(rect, tiles_x)
    order = np.lexsort((gid, np.asarray(depth)[gid], tile))
    tile, gid = tile[order], gid[order]
    bounds = np.searchsorted(tile, np.arange(num_tiles + 1))
    return [gid[bounds[i]:bounds[i + 1]] for i in range(num_tiles)]
