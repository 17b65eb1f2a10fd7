"""Perspective (EWA) projection of conditional 3D Gaussians (oracle, float64).

The paper converts each sliced Gaussian to the 3DGS format and projects it with the
standard 3DGS perspective projection (Sec. 4.4, rendering pipeline).  The paper does
not restate those rules, so this module fixes them as the following readings:
  * OpenCV pinhole: p_cam = R mu + t with the world->camera matrix [R | t]; depth z = p_cam.z;
    image position u = fx x/z + cx, v = fy y/z + cy, pixel (i, j) centred at (i + 1/2, j + 1/2).
  * Cull if z < near (0.2).
  * Local affine (EWA) Jacobian at p_cam, with x/z and y/z clamped to +-1.3 tan(fov/2) for J
    only: J = [[fx/z, 0, -fx x'/z^2], [0, fy/z, -fy y'/z^2]], x' = z clamp(x/z), y' likewise.
  * Sigma_2D = J R Sigma_cond R^T J^T + 0.3 I; cull if det(Sigma_2D) <= 0; conic = Sigma_2D^{-1}.
  * lambda_max = m + sqrt(max(0, m^2 - det)), m = trace/2; radius r = ceil(3 sqrt(lambda_max)).
  * Tile rectangle (16x16 tiles): rx0 = clamp(floor((u - r)/16), 0, Tx),
    rx1 = clamp(floor((u + r)/16) + 1, 0, Tx), likewise in y; cull if the rectangle is empty.
  * Cull if alpha_cond < 1/255 (no pixel could pass the compositing threshold).
"""
from __future__ import annotations

import torch

NEAR = 0.2
JAC_CLAMP = 1.3
DILATION = 0.3
EXTENT = 3.0
TILE = 16
ALPHA_MIN = 1.0 / 255.0


def camera_tensors(cam):
    V = torch.as_tensor(cam.viewmat, dtype=torch.float64)
    return V[:3, :3], V[:3, 3]


def project(mu_cond: torch.Tensor, Sigma_cond: torch.Tensor, cam) -> dict:
    R, tvec = camera_tensors(cam)
    p = mu_cond @ R.T + tvec
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    fx, fy = cam.fx, cam.fy
    lim_x = JAC_CLAMP * (0.5 * cam.width / fx)
    lim_y = JAC_CLAMP * (0.5 * cam.height / fy)
    xc = z * torch.clamp(x / z, -lim_x, lim_x)
    yc = z * torch.clamp(y / z, -lim_y, lim_y)
    zero = torch.zeros_like(z)
    J = torch.stack([torch.stack([fx / z, zero, -fx * xc / (z * z)], dim=1),
                     torch.stack([zero, fy / z, -fy * yc / (z * z)], dim=1)], dim=1)  # [N, 2, 3]
    S_cam = R @ Sigma_cond @ R.T
    S2 = J @ S_cam @ J.transpose(-1, -2)
    a = S2[:, 0, 0] + DILATION
    b = S2[:, 0, 1]
    c = S2[:, 1, 1] + DILATION
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], dim=1)
    u = fx * x / z + cam.cx
    v = fy * y / z + cam.cy
    mid = 0.5 * (a + c)
    lam_max = mid + torch.sqrt(torch.clamp_min(mid * mid - det, 0.0))
    extent = EXTENT * torch.sqrt(lam_max)
    return dict(p_cam=p, depth=z, mean2d=torch.stack([u, v], dim=1), cov2d=torch.stack([a, b, c], 1),
                det=det, conic=conic, extent=extent)


def tile_rect(u: torch.Tensor, v: torch.Tensor, radius: torch.Tensor, tiles_x: int, tiles_y: int):
    """Tiles whose pixel boxes meet the square [u - r, u + r] x [v - r, v + r]."""
    rx0 = torch.clamp(torch.floor((u - radius) / TILE), 0, tiles_x)
    rx1 = torch.clamp(torch.floor((u + radius) / TILE) + 1, 0, tiles_x)
    ry0 = torch.clamp(torch.floor((v - radius) / TILE), 0, tiles_y)
    ry1 = torch.clamp(torch.floor((v + radius) / TILE) + 1, 0, tiles_y)
    return torch.stack([rx0, ry0, rx1, ry1], dim=1).to(torch.int64)


def _dist_to_int(x: torch.Tensor) -> torch.Tensor:
    return torch.abs(x - torch.round(x))


def decision_margins(proj: dict, alpha_cond: torch.Tensor, radius: torch.Tensor, cam) -> dict:
    """Distances of every discrete decision in projection to its threshold.

    Used by the parity tests to set aside Gaussians whose culling, radius or tile rectangle an
    FP32 evaluation could legitimately decide the other way.
    """
    z = proj["depth"]
    u, v = proj["mean2d"][:, 0], proj["mean2d"][:, 1]
    ext = proj["extent"]
    return dict(
        z_rel=torch.abs(z - NEAR) / NEAR,
        alpha_rel=torch.abs(alpha_cond - ALPHA_MIN) / ALPHA_MIN,
        radius_rel=_dist_to_int(ext) / torch.clamp_min(ext, 1.0),
        edge_px=torch.min(torch.stack([
            _dist_to_int((u - radius) / TILE), _dist_to_int((u + radius) / TILE),
            _dist_to_int((v - radius) / TILE), _dist_to_int((v + radius) / TILE)], 1), 1).values * TILE,
    )

