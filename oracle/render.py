"""The whole 7DGS render path in float64, plus sampled pixels and autograd gradients (oracle).

Pipeline (Sec. 4.4: after slicing, rendering is the unchanged 3DGS pipeline):
  slicing (Algorithm 1 steps 3-6) -> projection + SH colour -> tile binning by (tile, depth) ->
  front-to-back compositing.  SH colour is evaluated at the unit direction from the camera
  centre to mu_cond.  Gradients of any scalar of the image are PyTorch autograd through this
  forward, with the discrete decisions (culling, radius, rectangles, order, stop) held fixed.
"""
from __future__ import annotations

import numpy as np
import torch

from . import agr, binning, composite, projection, sh, slicing

F64 = torch.float64
TILE = 16


def params_from_scene(scene, requires_grad: bool = False) -> dict:
    p = dict(mean7=torch.tensor(np.asarray(scene.mean7), dtype=F64),
             L28=torch.tensor(np.asarray(scene.L28), dtype=F64),
             opacity=torch.tensor(np.asarray(scene.opacity), dtype=F64),
             sh=torch.tensor(np.asarray(scene.sh), dtype=F64).reshape(-1, 16, 3))
    if requires_grad:
        for v in p.values():
            v.requires_grad_(True)
    return p


def gaussians(params: dict, cam, lambda_t, lambda_d, dir_mode: int = 0) -> dict:
    """Per-Gaussian slicing, modulation, projection, radius, tile rectangle, colour, visibility."""
    sl = slicing.slice_gaussians(params["mean7"], params["L28"], params["opacity"], cam.t, cam.d,
                                 lambda_t, lambda_d, dir_mode, np.asarray(cam.center))
    pr = projection.project(sl["mu_cond"], sl["Sigma_cond"], cam)
    centre = torch.as_tensor(np.asarray(cam.center), dtype=F64)
    diff = sl["mu_cond"] - centre
    dirs = diff / torch.linalg.norm(diff, dim=1, keepdim=True)
    rgb = sh.colour(params["sh"], dirs)
    with torch.no_grad():
        radius = torch.ceil(pr["extent"])
        u, v = pr["mean2d"][:, 0], pr["mean2d"][:, 1]
        rect = projection.tile_rect(u, v, radius, cam.tiles_x, cam.tiles_y)
        nonempty = (rect[:, 2] > rect[:, 0]) & (rect[:, 3] > rect[:, 1])
        visible = ((pr["depth"] >= projection.NEAR) & (pr["det"] > 0)
                   & (sl["alpha_cond"] >= projection.ALPHA_MIN) & nonempty)
        visible &= torch.isfinite(pr["extent"])
        rect[~visible] = 0
        margins = projection.decision_margins(pr, sl["alpha_cond"], radius, cam)
    out = dict(sl)
    out.update(pr)
    out.update(rgb=rgb, dirs=dirs, radius=radius, rect=rect, visible=visible, margins=margins)
    return out


def pixel_centres(cam, tile: int) -> tuple[torch.Tensor, torch.Tensor]:
    """Pixel centres of one tile that lie inside the image, and their (row, col) indices."""
    tx, ty = tile % cam.tiles_x, tile // cam.tiles_x
    xs = torch.arange(tx * TILE, min((tx + 1) * TILE, cam.width))
    ys = torch.arange(ty * TILE, min((ty + 1) * TILE, cam.height))
    yy, xx = torch.meshgrid(ys, xs, indexing="ij")
    rc = torch.stack([yy.reshape(-1), xx.reshape(-1)], 1)
    pix = torch.stack([xx.reshape(-1).to(F64) + 0.5, yy.reshape(-1).to(F64) + 0.5], 1)
    return pix, rc


def cull_inputs(mean2d, conic, alpha):
    """The float32 screen-space values the tile-reachability rule of binning reads."""
    f = lambda x: x.detach().numpy().astype(np.float32)
    return (f(mean2d), f(conic), f(alpha))


def composite_all(mean2d, conic, alpha, rgb, depth, rect, cam, bg, tiles=None, reach: bool = False) -> dict:
    """Composite every tile (or the listed ones) of the image.

    Each tile's candidates are the Gaussians whose tile rectangle contains it (Sec. 4.4, the 3DGS
    blending rule).  With reach=True they are further restricted to the tiles the binning's
    reachability rule keeps, which can only drop candidates that no pixel of the tile takes
    (alpha < 1/255 everywhere): the image is the same, but list positions (n_contrib) then match
    the binned lists.
    """
    num_tiles = cam.tiles_x * cam.tiles_y
    lists = binning.tile_lists(depth.detach().numpy(), rect.numpy(), cam.tiles_x, num_tiles,
                               cull=cull_inputs(mean2d, conic, alpha) if reach else None)
    H, W = cam.height, cam.width
    colors, Ts, ncs, lasts, margins, rcs = [], [], [], [], [], []
    for tile in (range(num_tiles) if tiles is None else tiles):
        pix, rc = pixel_centres(cam, tile)
        g = torch.as_tensor(lists[tile], dtype=torch.int64)
        r = composite.composite_tile(pix, g, mean2d, conic, alpha, rgb, bg, depth=depth.detach())
        colors.append(r["color"]); Ts.append(r["final_T"]); ncs.append(r["n_contrib"])
        lasts.append(r["last_id"]); margins.append(r["margin"]); rcs.append(rc)
    rc = torch.cat(rcs)
    flat = rc[:, 0] * W + rc[:, 1]
    color = torch.cat(colors)
    image = torch.zeros(H * W, 3, dtype=color.dtype).index_add(0, flat, color).reshape(H, W, 3)
    out = dict(image=image)
    with torch.no_grad():
        for name, vals, fill in (("final_T", Ts, 1.0), ("n_contrib", ncs, 0), ("last_id", lasts, -1),
                                 ("margin_alpha", [m["alpha"] for m in margins], float("inf")),
                                 ("margin_T", [m["T"] for m in margins], float("inf")),
                                 ("margin_depth", [m["depth"] for m in margins], float("inf"))):
            v = torch.cat(vals)
            buf = torch.full((H * W,), fill, dtype=v.dtype)
            buf[flat] = v
            out[name] = buf.reshape(H, W)
        covered = torch.zeros(H * W, dtype=torch.bool)
        covered[flat] = True
        out["covered"] = covered.reshape(H, W)
    return out


def render(scene, cam, tiles=None, params: dict | None = None, reach: bool = False) -> dict:
    """Full-image (or listed-tile) render of a scene; returns image [H, W, 3] and per-Gaussian data."""
    p = params if params is not None else params_from_scene(scene)
    g = gaussians(p, cam, scene.lambda_t, scene.lambda_d, scene.dir_mode)
    bg = torch.as_tensor(cam.bg, dtype=F64)
    out = composite_all(g["mean2d"], g["conic"], g["alpha_cond"], g["rgb"], g["depth"], g["rect"],
                        cam, bg, tiles, reach)
    out["g"] = g
    return out


def render_pixels(g: dict, cam, pixels: np.ndarray, reach: bool = False) -> dict:
    """Colour, final_T, n_contrib, last contributor id and margins of listed pixels [P, 2] (row,
    col) from per-Gaussian data.

    Candidate lists are built per tile from rectangle containment over all Gaussians, so this
    scales to full-size scenes for a sample of pixels; reach=True restricts them as in
    composite_all.
    """
    bg = torch.as_tensor(cam.bg, dtype=F64)
    pixels = np.asarray(pixels, dtype=np.int64)
    tiles = (pixels[:, 0] // TILE) * cam.tiles_x + pixels[:, 1] // TILE
    rect = g["rect"]
    depth = g["depth"].detach()
    keys = ("color", "final_T", "n_contrib", "last_id", "margin_alpha", "margin_T", "margin_depth")
    res = {k: [None] * len(pixels) for k in keys}
    for tile in np.unique(tiles):
        sel = np.nonzero(tiles == tile)[0]
        tx, ty = int(tile % cam.tiles_x), int(tile // cam.tiles_x)
        inside = (rect[:, 0] <= tx) & (tx < rect[:, 2]) & (rect[:, 1] <= ty) & (ty < rect[:, 3])
        ids = torch.nonzero(inside).reshape(-1)
        if reach:
            m2, co, al = cull_inputs(g["mean2d"][ids], g["conic"][ids], g["alpha_cond"][ids])
            ids = ids[torch.as_tensor(binning.tile_reachable(m2, co, al, tx, ty))]
        order = np.lexsort((ids.numpy(), depth[ids].numpy()))
        cand = ids[torch.as_tensor(order, dtype=torch.int64)]
        pix = torch.as_tensor(pixels[sel][:, ::-1].copy(), dtype=F64) + 0.5
        r = composite.composite_tile(pix, cand, g["mean2d"].detach(), g["conic"].detach(),
                                     g["alpha_cond"].detach(), g["rgb"].detach(), bg, depth=depth)
        for k in ("alpha", "T", "depth"):
            r["margin_" + k] = r["margin"][k]
        for j, i in enumerate(sel):
            for k in res:
                res[k][i] = r[k][j]
    return {k: torch.stack(v) for k, v in res.items()}


def render_projected(rec: dict, width: int, height: int, bg, tiles=None, reach: bool = False) -> dict:
    """Composite given screen-space records (float32 inputs evaluated in float64).

    rec: mean2d [N, 2], conic [N, 3], opacity [N], rgb [N, 3], depth [N] (float32), rect [N, 4].
    Binning uses the float32 depth bits exactly as stored.
    """
    class _Cam:
        pass
    cam = _Cam()
    cam.width, cam.height = width, height
    cam.tiles_x, cam.tiles_y = (width + TILE - 1) // TILE, (height + TILE - 1) // TILE
    t = lambda k: torch.as_tensor(np.asarray(rec[k], dtype=np.float32).astype(np.float64))
    rect = torch.as_tensor(np.asarray(rec["rect"], dtype=np.int64))
    return composite_all(t("mean2d"), t("conic"), t("opacity"), t("rgb"), t("depth"), rect, cam,
                         torch.as_tensor(bg, dtype=F64), tiles, reach)


def refined_params(scene, agr_weights: dict | None, t, requires_grad: bool = False):
    """Scene parameters as float64 tensors, refined by the adaptive refinement MLPs (Sec. 4.3)
    at time t when agr_weights (float32 arrays) are given.  Returns (leaves, params, weights)."""
    leaf = params_from_scene(scene, requires_grad=requires_grad)
    if agr_weights is None:
        return leaf, leaf, None
    w = agr.weights_to_torch(agr_weights, requires_grad=requires_grad)
    m, l = agr.refine(leaf["mean7"], leaf["L28"], t, w)
    return leaf, dict(leaf, mean7=m, L28=l), w


def render_agr(scene, cam, agr_weights: dict, tiles=None) -> dict:
    """render() of the scene refined at the camera's time t."""
    _, p, _ = refined_params(scene, agr_weights, cam.t)
    return render(scene, cam, tiles, params={k: v.detach() for k, v in p.items()})


def vjp(scene, cam, dL_dimage: np.ndarray, tiles=None, agr_weights: dict | None = None) -> dict:
    """Gradients of sum(dL_dimage * image) w.r.t. mean7, L28, opacity, sh and (lambda_t,
    lambda_d) -- and, with agr_weights, w.r.t. the refinement weights -- in float64.

    The visible set is found first without gradients; the forward is then re-run on the
    visible Gaussians only, so culled Gaussians receive exactly zero gradient.  With `tiles`,
    only those tiles are composited: exact when dL_dimage is zero outside them.
    """
    with torch.no_grad():
        _, p0, _ = refined_params(scene, agr_weights, cam.t)
        vis = gaussians(p0, cam, scene.lambda_t, scene.lambda_d, scene.dir_mode)["visible"]
    idx = torch.nonzero(vis).reshape(-1)
    leaf, p, w = refined_params(scene, agr_weights, cam.t, requires_grad=True)
    lam = torch.tensor([scene.lambda_t, scene.lambda_d], dtype=F64, requires_grad=True)
    sub = {k: v[idx] for k, v in p.items()}
    g = gaussians(sub, cam, lam[0], lam[1], scene.dir_mode)
    bg = torch.as_tensor(cam.bg, dtype=F64)
    out = composite_all(g["mean2d"], g["conic"], g["alpha_cond"], g["rgb"], g["depth"], g["rect"],
                        cam, bg, tiles)
    loss = (out["image"] * torch.as_tensor(dL_dimage, dtype=F64)).sum()
    loss.backward()
    res = dict(mean7=leaf["mean7"].grad.numpy(), L28=leaf["L28"].grad.numpy(),
               opacity=leaf["opacity"].grad.numpy(), sh=leaf["sh"].grad.numpy(),
               lam=lam.grad.numpy(), image=out["image"].detach().numpy(), loss=float(loss.detach()))
    if w is not None:
        res.update({k: v.grad.numpy() for k, v in w.items()})
    return res
