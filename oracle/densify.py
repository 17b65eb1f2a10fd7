"""Densification statistics of the conditional 3D Gaussians (oracle, float64; test
infrastructure only -- the CUDA path never imports it).

Algorithm 1 step 7 and Sec. 4.4:
  * Sigma_cond = U D U^T (eigendecomposition of the symmetric positive semi-definite Sigma_cond,
    which is its SVD), R = U, S = sqrt(diag(D)); the last column of R is multiplied by
    sign(det R) so that R is a proper rotation.  Order (a reading: the paper fixes none): the
    scales in descending order, R's columns in the same order.
  * Split statistics: |Sigma_pt| (Euclidean norm of the 3-vector coupling space and time) and
    the temporal scale sqrt(Sigma_t) (time is normalised to [0, 1], so this is already the
    "normalised" scale -- a reading).  Split when |Sigma_pt| > split_pt * extent and
    sqrt(Sigma_t) > split_t (0.05 relative to the scene extent and 0.25 in the paper).
  * Prune when the base opacity alpha < prune_alpha (tau_min = 0.01 in the paper).
"""
from __future__ import annotations

import numpy as np
import torch

from . import slicing


def scale_rotation(Sigma_cond: torch.Tensor) -> tuple[np.ndarray, np.ndarray]:
    """[N, 3, 3] -> S [N, 3] (descending), R [N, 3, 3] with det R = +1 (columns = axes)."""
    evals, evecs = torch.linalg.eigh(Sigma_cond)  # ascending
    evals = evals.flip(-1).numpy()
    R = evecs.flip(-1).numpy().copy()
    S = np.sqrt(np.maximum(evals, 0.0))
    sign = np.sign(np.linalg.det(R))
    R[:, :, 2] *= sign[:, None]
    return S, R


def densify_stats(mean7, L28, opacity, t: float, d, lambda_t: float, lambda_d: float, extent: float,
                  split_pt: float = 0.05, split_t: float = 0.25, prune_alpha: float = 0.01,
                  dir_mode: int = 0, center=None) -> dict:
    mean7 = torch.as_tensor(np.asarray(mean7), dtype=torch.float64)
    L28 = torch.as_tensor(np.asarray(L28), dtype=torch.float64)
    opacity = torch.as_tensor(np.asarray(opacity), dtype=torch.float64)
    sl = slicing.slice_gaussians(mean7, L28, opacity, t, d, lambda_t, lambda_d, dir_mode, center)
    S, R = scale_rotation(sl["Sigma_cond"])
    Sigma = sl["Sigma"].numpy()
    pt_norm = np.linalg.norm(Sigma[:, 0:3, 3], axis=1)
    t_scale = np.sqrt(Sigma[:, 3, 3])
    return dict(scale=S, rot=R, pt_norm=pt_norm, t_scale=t_scale,
                split=(pt_norm > split_pt * extent) & (t_scale > split_t),
                prune=opacity.numpy() < prune_alpha, Sigma_cond=sl["Sigma_cond"].numpy())
