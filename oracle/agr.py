"""Adaptive Gaussian Refinement (oracle, float64; test infrastructure only -- the CUDA path never
imports it).

Sec. 4.3 and Algorithm 1 steps 1-2:
  f = mu_p (+) mu_t (+) mu_d (+) gamma(t)                                   (27 values)
  gamma(t) = (sin(2^0 pi t), cos(2^0 pi t), ..., sin(2^(K-1) pi t), cos(2^(K-1) pi t)), K = 10
  four two-layer MLPs C_in x 64 x C_out, C_out = 3, 1, 3, 28, give residuals
  mu_p^ = mu_p + phi_p(f), mu_t^ = mu_t + phi_t(f), mu_d^ = mu_d + phi_d(f), l^ = l + phi_l(f)
  with l the 28 packed lower-triangular entries of L (the same packing as L28).
Readings (the paper does not print them): each MLP is Linear(27, 64) -> ReLU -> Linear(64, C_out)
with biases in both layers.  Weights as stored: w1 [4, 64, 27] (MLPs in the order p, t, d, l),
b1 [4, 64], w2 [35, 64] (rows 0-2 phi_p, 3 phi_t, 4-6 phi_d, 7-34 phi_l; each row reads the 64
hidden units of its own MLP), b2 [35].
"""
from __future__ import annotations

import math

import torch

F64 = torch.float64
K_FREQ = 10
HIDDEN = 64
ROWS = ((0, 3), (3, 4), (4, 7), (7, 35))  # output rows of each MLP in w2 / b2


def temporal_encoding(t, K: int = K_FREQ) -> torch.Tensor:
    """gamma(t) as printed: sin and cos of 2^k pi t for k = 0 .. K-1, interleaved."""
    t = torch.as_tensor(t, dtype=F64)
    out = []
    for k in range(K):
        out.append(torch.sin((2.0 ** k) * math.pi * t))
        out.append(torch.cos((2.0 ** k) * math.pi * t))
    return torch.stack(out)


def features(mean7: torch.Tensor, t) -> torch.Tensor:
    g = temporal_encoding(t).reshape(1, -1).expand(mean7.shape[0], -1)
    return torch.cat([mean7[:, 0:3], mean7[:, 3:4], mean7[:, 4:7], g], dim=1)


def residuals(f: torch.Tensor, w: dict) -> torch.Tensor:
    """[N, 35]: the four MLPs' outputs stacked in the w2 row order."""
    outs = []
    for m, (r0, r1) in enumerate(ROWS):
        h = torch.relu(f @ w["w1"][m].T + w["b1"][m])
        outs.append(h @ w["w2"][r0:r1].T + w["b2"][r0:r1])
    return torch.cat(outs, dim=1)


def refine(mean7: torch.Tensor, L28: torch.Tensor, t, w: dict) -> tuple[torch.Tensor, torch.Tensor]:
    """(mean7^, L28^) = (mean7 + (phi_p, phi_t, phi_d), L28 + phi_l)."""
    r = residuals(features(mean7, t), w)
    return mean7 + r[:, 0:7], L28 + r[:, 7:35]


def weights_to_torch(w: dict, requires_grad: bool = False) -> dict:
    out = {k: torch.tensor(w[k], dtype=F64) for k in ("w1", "b1", "w2", "b2")}
    if requires_grad:
        for v in out.values():
            v.requires_grad_(True)
    return out
