"""Conditional slicing of 7D Gaussians into 3D Gaussians (oracle, float64).

Follows Sec. 4.1-4.2 literally:
  * Sigma = L L^T with L the 7x7 lower-triangular Cholesky factor (Sec. 4.1, Cholesky
    parameterisation; Algorithm 1 step 3).
  * Partition into Sigma_p (3x3), Sigma_{p,(t,d)} = [Sigma_pt Sigma_pd] (3x4) and
    Sigma_{(t,d)} = [[Sigma_t, Sigma_td], [Sigma_td^T, Sigma_d]] (4x4) (Sec. 4.2; Algorithm 1 step 4).
  * mu_cond = mu_p + Sigma_{p,(t,d)} Sigma_{(t,d)}^{-1} (t - mu_t, d - mu_d)   (Eq. cond_mean)
    Sigma_cond = Sigma_p - Sigma_{p,(t,d)} Sigma_{(t,d)}^{-1} Sigma_{p,(t,d)}^T  (Eq. cond_cov)
    (Algorithm 1 step 5).
  * f_temp = exp(-1/2 lambda_t (t - mu_t)^2 / Sigma_t)                          (Eq. temp_mod)
    f_dir  = exp(-1/2 lambda_d (d - mu_d)^T Sigma_d^{-1} (d - mu_d))             (Eq. dir_mod)
    alpha_cond = alpha f_temp f_dir                                              (Algorithm 1 step 6)
  The modulation uses the marginal Sigma_t and Sigma_d blocks of Sigma, exactly as printed.

The conditioning direction d is the request's view direction, or (dir_mode = 1, the 6DGS-style
reading of "view direction", Sec. 3) each Gaussian's own unit direction from the camera centre
to its spatial mean mu_p; then d depends on mu_p and gradients flow through it.  lambda_t and
lambda_d may be tensors that require gradients.
"""
from __future__ import annotations

import torch

F64 = torch.float64


def unpack_L(L28: torch.Tensor) -> torch.Tensor:
    """[N, 28] packed row-major lower triangle -> [N, 7, 7] (element (i, j) at i(i+1)/2 + j)."""
    n = L28.shape[0]
    rows, cols = torch.tril_indices(7, 7)
    # torch.tril_indices enumerates row by row, column ascending: the packed order.
    L = torch.zeros(n, 7, 7, dtype=L28.dtype)
    L = L.index_put((torch.arange(n).repeat_interleave(28), rows.repeat(n), cols.repeat(n)),
                    L28.reshape(-1))
    return L


def covariance(L: torch.Tensor) -> torch.Tensor:
    """Sigma = L L^T, the full 7x7 product."""
    return L @ L.transpose(-1, -2)


def partition(Sigma: torch.Tensor):
    """Blocks in the (p | t, d) order of Sec. 4.2."""
    S_p = Sigma[:, 0:3, 0:3]
    S_p_td = Sigma[:, 0:3, 3:7]
    S_td = Sigma[:, 3:7, 3:7]
    return S_p, S_p_td, S_td


def condition(mean7: torch.Tensor, Sigma: torch.Tensor, t: float, d) -> tuple[torch.Tensor, torch.Tensor]:
    """Eq. cond_mean and Eq. cond_cov with an explicit inverse of Sigma_{(t,d)}."""
    S_p, S_p_td, S_td = partition(Sigma)
    S_td_inv = torch.linalg.inv(S_td)
    d = torch.as_tensor(d, dtype=mean7.dtype).reshape(-1, 3)  # one direction, or one per Gaussian
    dev = torch.cat([t - mean7[:, 3:4], d - mean7[:, 4:7]], dim=1)  # (t - mu_t, d - mu_d)
    gain = S_p_td @ S_td_inv
    mu_cond = mean7[:, 0:3] + (gain @ dev.unsqueeze(-1)).squeeze(-1)
    Sigma_cond = S_p - gain @ S_p_td.transpose(-1, -2)
    return mu_cond, Sigma_cond


def modulation(mean7: torch.Tensor, Sigma: torch.Tensor, t: float, d, lambda_t: float,
               lambda_d: float) -> tuple[torch.Tensor, torch.Tensor]:
    """Eq. temp_mod and Eq. dir_mod with the marginal Sigma_t (scalar) and Sigma_d (3x3)."""
    S_t = Sigma[:, 3, 3]
    S_d = Sigma[:, 4:7, 4:7]
    dt = t - mean7[:, 3]
    f_temp = torch.exp(-0.5 * lambda_t * dt * dt / S_t)
    d = torch.as_tensor(d, dtype=mean7.dtype).reshape(-1, 3)
    dd = d - mean7[:, 4:7]
    q = (dd.unsqueeze(1) @ torch.linalg.inv(S_d) @ dd.unsqueeze(-1)).reshape(-1)
    f_dir = torch.exp(-0.5 * lambda_d * q)
    return f_temp, f_dir


def gaussian_directions(mean7: torch.Tensor, center) -> torch.Tensor:
    """Unit direction from the camera centre to each spatial mean mu_p (dir_mode = 1)."""
    w = mean7[:, 0:3] - torch.as_tensor(center, dtype=mean7.dtype).reshape(1, 3)
    return w / torch.linalg.norm(w, dim=1, keepdim=True)


def slice_gaussians(mean7, L28, opacity, t: float, d, lambda_t, lambda_d, dir_mode: int = 0,
                    center=None) -> dict:
    """Algorithm 1 steps 3-6 for every Gaussian (no adaptive refinement)."""
    if dir_mode == 1:
        d = gaussian_directions(mean7, center)
    elif dir_mode != 0:
        raise ValueError("dir_mode must be 0 or 1")
    Sigma = covariance(unpack_L(L28))
    mu_cond, Sigma_cond = condition(mean7, Sigma, t, d)
    f_temp, f_dir = modulation(mean7, Sigma, t, d, lambda_t, lambda_d)
    alpha_cond = opacity * f_temp * f_dir
    return dict(Sigma=Sigma, mu_cond=mu_cond, Sigma_cond=Sigma_cond, f_temp=f_temp, f_dir=f_dir,
                alpha_cond=alpha_cond)
