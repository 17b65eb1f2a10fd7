"""Seeded synthetic 7D Gaussian scenes and pinhole cameras.

Every array is drawn with NumPy's PCG64 generator from an explicit seed, so the
CUDA path and the oracle see bit-identical inputs.  Scene parameters follow the
7D Gaussian record of Sec. 4.1 (mean mu = (mu_p, mu_t, mu_d) in R^7, covariance
Sigma = L L^T with L lower-triangular, a base opacity alpha and degree-3
spherical-harmonic colour coefficients).  Nothing here evaluates the method.

Layouts (all float32, C-contiguous):
    mean7    [N, 7]      (mu_p.xyz, mu_t, mu_d.xyz)
    L28      [N, 28]     lower-triangular L packed row-major: L[i][j] at i*(i+1)/2 + j, j <= i
    opacity  [N]         base opacity alpha in (0, 1)
    sh       [N, 16, 3]  real SH coefficients, index l*l + l + m, RGB innermost
Camera: world->camera 4x4 row-major `viewmat` (OpenCV axes: +x right, +y down,
+z forward), pinhole intrinsics fx, fy, cx, cy in pixels, image W x H.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SH_COEFFS = 16
TILE = 16


@dataclasses.dataclass
class Scene:
    mean7: np.ndarray
    L28: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray
    lambda_t: float
    lambda_d: float
    bg: tuple = (0.0, 0.0, 0.0)
    dir_mode: int = 0  # conditioning direction: 0 the request's, 1 camera centre -> mu_p per Gaussian

    @property
    def n(self) -> int:
        return int(self.mean7.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.mean7[idx].copy(), self.L28[idx].copy(), self.opacity[idx].copy(),
                     self.sh[idx].copy(), self.lambda_t, self.lambda_d, self.bg, self.dir_mode)


@dataclasses.dataclass
class Camera:
    viewmat: np.ndarray  # float64 [4, 4], world -> camera
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    t: float
    d: np.ndarray  # float64 [3], unit conditioning view direction (camera forward axis in world)
    bg: tuple = (0.0, 0.0, 0.0)
    near: float = 0.2

    @property
    def tiles_x(self) -> int:
        return (self.width + TILE - 1) // TILE

    @property
    def tiles_y(self) -> int:
        return (self.height + TILE - 1) // TILE

    @property
    def center(self) -> np.ndarray:
        R = self.viewmat[:3, :3]
        return -R.T @ self.viewmat[:3, 3]


def _packed_index(i: int, j: int) -> int:
    return i * (i + 1) // 2 + j


def _draw_L(rng: np.random.Generator, n: int, diag_lo: float, diag_hi: float,
            off_sigma: float) -> np.ndarray:
    """Packed lower-triangular factors: log-uniform diagonal, N(0, off_sigma^2) below it."""
    L = np.zeros((n, 28), dtype=np.float64)
    diag = np.exp(rng.uniform(math.log(diag_lo), math.log(diag_hi), size=(n, 7)))
    off = rng.normal(0.0, off_sigma, size=(n, 21))
    k = 0
    for i in range(7):
        for j in range(i):
            L[:, _packed_index(i, j)] = off[:, k]
            k += 1
        L[:, _packed_index(i, i)] = diag[:, i]
    return L.astype(np.float32)


def _unit(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def make_scene(n: int, seed: int, *, box: float = 1.0, diag=(0.02, 0.3), off_sigma: float = 0.05,
               clusters: int = 0, cluster_sigma: float = 0.3, cluster_box: float = 5.0,
               lambda_t: float = 0.05, lambda_d: float = 0.05, bg=(0.0, 0.0, 0.0)) -> Scene:
    """Draw N 7D Gaussians.

    Spatial means are uniform in [-box, box]^3, or (clusters > 0) a clustered
    mixture: `clusters` centres uniform in [-cluster_box, cluster_box]^3 plus
    N(0, cluster_sigma^2) per point.  mu_t ~ U[0, 1]; mu_d is a random unit
    vector.  Opacity is sigmoid(N(0, 1)); SH DC ~ N(0.5, 0.2^2), the other 15
    bands ~ N(0, 0.1^2) per channel.
    """
    rng = np.random.default_rng(seed)
    if clusters > 0:
        centres = rng.uniform(-cluster_box, cluster_box, size=(clusters, 3))
        which = rng.integers(0, clusters, size=n)
        mu_p = centres[which] + rng.normal(0.0, cluster_sigma, size=(n, 3))
    else:
        mu_p = rng.uniform(-box, box, size=(n, 3))
    mu_t = rng.uniform(0.0, 1.0, size=(n, 1))
    mu_d = _unit(rng, n)
    mean7 = np.concatenate([mu_p, mu_t, mu_d], axis=1).astype(np.float32)
    L28 = _draw_L(rng, n, diag[0], diag[1], off_sigma)
    opacity = (1.0 / (1.0 + np.exp(-rng.normal(size=n)))).astype(np.float32)
    sh = rng.normal(0.0, 0.1, size=(n, SH_COEFFS, 3))
    sh[:, 0, :] = rng.normal(0.5, 0.2, size=(n, 3))
    return Scene(np.ascontiguousarray(mean7), np.ascontiguousarray(L28),
                 np.ascontiguousarray(opacity), np.ascontiguousarray(sh.astype(np.float32)),
                 float(lambda_t), float(lambda_d), tuple(float(b) for b in bg))


def look_at(eye, target=(0.0, 0.0, 0.0), down=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World->camera matrix for an OpenCV camera at `eye` looking at `target`.

    Camera +z is the forward axis, +x = normalize(down x z), +y = z x x.  When
    the forward axis is nearly parallel to `down`, the reference vector is
    swapped to +z.
    """
    eye = np.asarray(eye, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - eye
    z /= np.linalg.norm(z)
    ref = np.asarray(down, dtype=np.float64)
    if abs(float(np.dot(ref, z))) > 0.999:
        ref = np.array([0.0, 0.0, 1.0])
    x = np.cross(ref, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    V = np.eye(4)
    V[:3, :3] = R
    V[:3, 3] = -R @ eye
    return V


def make_camera(eye, width: int, height: int, fov_x_deg: float, t: float,
                target=(0.0, 0.0, 0.0), bg=(0.0, 0.0, 0.0)) -> Camera:
    V = look_at(eye, target)
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(viewmat=V, fx=fx, fy=fx, cx=width / 2.0, cy=height / 2.0, width=int(width),
                  height=int(height), t=float(t), d=V[2, :3].copy(), bg=tuple(float(b) for b in bg))


# ---------------------------------------------------------------------------------------------
# The five workloads.  Config 0 is the small case the oracle renders completely; configs 1-2 are
# the object-scale and large-scene forward renders; config 3 is the differentiation workload;
# config 4 the serving scenes.  lambda_t = lambda_d is 0.05 for the object-scale scenes and 0.1
# for the large clustered scenes.
# ---------------------------------------------------------------------------------------------

WHITE = (1.0, 1.0, 1.0)
BLACK = (0.0, 0.0, 0.0)


def config_scene(cfg: int, n: int | None = None, lam: float | None = None) -> Scene:
    if cfg == 0:
        return make_scene(n or 4096, seed=0, box=1.0, lambda_t=lam or 0.05, lambda_d=lam or 0.05,
                          bg=BLACK)
    if cfg in (1, 3):
        return make_scene(n or 300_000, seed=1, box=1.5, lambda_t=lam or 0.05,
                          lambda_d=lam or 0.05, bg=WHITE)
    if cfg == 2:
        return make_scene(n or 1_500_000, seed=2, diag=(0.005, 0.2), clusters=64,
                          cluster_sigma=0.3, cluster_box=5.0, lambda_t=lam or 0.1,
                          lambda_d=lam or 0.1, bg=BLACK)
    raise ValueError(f"unknown config {cfg}")


def config_cameras(cfg: int, count: int | None = None, width: int | None = None,
                   height: int | None = None) -> list[Camera]:
    if cfg == 0:
        return [make_camera((0.0, 0.0, -3.0), width or 128, height or 128, 60.0, 0.5, bg=BLACK)]
    if cfg in (1, 3):
        rng = np.random.default_rng(1001)  # config 3 renders config 1's cameras
        m = count or 100
        dirs = _unit(rng, m)
        frames = rng.integers(0, 300, size=m)
        return [make_camera(4.0 * dirs[i], width or 800, height or 800, 60.0,
                            float(frames[i]) / 299.0, bg=WHITE) for i in range(m)]
    if cfg == 2:
        rng = np.random.default_rng(1002)
        m = count or 50
        yaws = np.linspace(-30.0, 30.0, m)
        ts = rng.uniform(0.0, 1.0, size=m)
        cams = []
        for i in range(m):
            a = math.radians(yaws[i])
            eye = (8.0 * math.sin(a), 0.0, -8.0 * math.cos(a))
            cams.append(make_camera(eye, width or 1352, height or 1014, 60.0, float(ts[i]),
                                    bg=BLACK))
        return cams
    raise ValueError(f"unknown config {cfg}")


def perturb_scene(scene: Scene, seed: int = 2000, mean_sigma: float = 0.01,
                  L_sigma: float = 0.005, diag_floor: float = 1e-3) -> Scene:
    """Differentiation target: means + N(0, 0.01^2), L + N(0, 0.005^2), diagonal kept >= 1e-3."""
    rng = np.random.default_rng(seed)
    mean7 = scene.mean7 + rng.normal(0.0, mean_sigma, size=scene.mean7.shape)
    L28 = scene.L28 + rng.normal(0.0, L_sigma, size=scene.L28.shape)
    for i in range(7):
        k = _packed_index(i, i)
        L28[:, k] = np.maximum(L28[:, k], diag_floor)
    return Scene(mean7.astype(np.float32), L28.astype(np.float32), scene.opacity.copy(),
                 scene.sh.copy(), scene.lambda_t, scene.lambda_d, scene.bg, scene.dir_mode)


def serving_scenes() -> list[Scene]:
    """Four resident scenes of 100k, 300k (object scale) and 800k, 1.5M (clustered)."""
    return [make_scene(100_000, seed=41, box=1.5, bg=WHITE),
            make_scene(300_000, seed=42, box=1.5, bg=WHITE),
            make_scene(800_000, seed=43, diag=(0.005, 0.2), clusters=64, lambda_t=0.1,
                       lambda_d=0.1, bg=BLACK),
            make_scene(1_500_000, seed=44, diag=(0.005, 0.2), clusters=64, lambda_t=0.1,
                       lambda_d=0.1, bg=BLACK)]


def random_projected(n: int, width: int, height: int, seed: int, *, empty_frac: float = 0.1,
                     max_half_tiles: int = 6, tie_frac: float = 0.2) -> dict:
    """Arbitrary screen-space records for exercising binning and compositing on their own.

    Rectangles are random tile ranges [rx0, rx1) x [ry0, ry1) inside the tile grid (a fraction
    empty, some covering the full grid); depths are positive float32 values, a fraction of them
    drawn from a handful of repeated values so that equal keys occur.  Conics are random SPD
    2x2 inverses, opacities in (0, 0.99], colours in [0, 1].
    """
    rng = np.random.default_rng(seed)
    tx, ty = (width + TILE - 1) // TILE, (height + TILE - 1) // TILE
    cx = rng.integers(0, tx, size=n)
    cy = rng.integers(0, ty, size=n)
    hx = rng.integers(0, max_half_tiles + 1, size=n)
    hy = rng.integers(0, max_half_tiles + 1, size=n)
    rx0 = np.clip(cx - hx, 0, tx)
    rx1 = np.clip(cx + hx + 1, 0, tx)
    ry0 = np.clip(cy - hy, 0, ty)
    ry1 = np.clip(cy + hy + 1, 0, ty)
    full = rng.random(n) < 0.01
    rx0[full], ry0[full], rx1[full], ry1[full] = 0, 0, tx, ty
    empty = rng.random(n) < empty_frac
    rx0[empty], rx1[empty], ry0[empty], ry1[empty] = 0, 0, 0, 0
    rect = np.stack([rx0, ry0, rx1, ry1], axis=1).astype(np.int32)
    depth = rng.uniform(0.5, 10.0, size=n).astype(np.float32)
    ties = rng.random(n) < tie_frac
    depth[ties] = rng.choice(np.array([1.0, 2.5, 3.25], dtype=np.float32), size=int(ties.sum()))
    mean2d = np.stack([(cx + 0.5) * TILE + rng.uniform(-8, 8, size=n),
                       (cy + 0.5) * TILE + rng.uniform(-8, 8, size=n)], axis=1).astype(np.float32)
    qa = 1.0 / rng.uniform(2.0, 40.0, size=n) ** 2
    qc = 1.0 / rng.uniform(2.0, 40.0, size=n) ** 2
    qb = rng.uniform(-0.8, 0.8, size=n) * np.sqrt(qa * qc)
    conic = np.stack([qa, qb, qc], axis=1).astype(np.float32)
    opacity = rng.uniform(0.0, 0.99, size=n).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)
    return dict(mean2d=mean2d, conic=conic, opacity=opacity, rgb=rgb, depth=depth, rect=rect,
                width=width, height=height)


def make_agr_weights(seed: int = 3000, scale: float = 0.1) -> dict:
    """Random weights of the four refinement MLPs (27 -> 64 -> 3, 1, 3, 28): uniform
    +-1/sqrt(fan_in) as a freshly initialised linear layer, times `scale` so that the residuals
    stay small next to the parameters.  float32 arrays w1 [4, 64, 27], b1 [4, 64], w2 [35, 64],
    b2 [35]."""
    rng = np.random.default_rng(seed)
    a1, a2 = 1.0 / np.sqrt(27.0), 1.0 / np.sqrt(64.0)
    return dict(w1=(rng.uniform(-a1, a1, size=(4, 64, 27)) * scale).astype(np.float32),
                b1=(rng.uniform(-a1, a1, size=(4, 64)) * scale).astype(np.float32),
                w2=(rng.uniform(-a2, a2, size=(35, 64)) * scale).astype(np.float32),
                b2=(rng.uniform(-a2, a2, size=(35,)) * scale).astype(np.float32))
