"""Real spherical harmonics up to degree 3, built from the definition (oracle, float64).

The colour model c(d) = sum_{l<=3} sum_m beta_lm Y_lm(d) is the 3DGS one the paper keeps
(Sec. 3 "3D Gaussian Splatting", Sec. 4.1 colour representation).  The real basis is
    Y_l0      = N_l0 P_l(z)
    Y_lm      = sqrt(2) N_lm P_l^m(z) cos(m phi)        m > 0
    Y_l,-m    = sqrt(2) N_lm P_l^m(z) sin(m phi)        m > 0
with N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) and P_l^m the associated Legendre function
including the Condon-Shortley phase (-1)^m.  For a unit vector (x, y, z),
sin^m(theta) cos(m phi) = Re((x + i y)^m) and sin^m(theta) sin(m phi) = Im((x + i y)^m), so
P_l^m(z) cos(m phi) = (-1)^m [d^m P_l / dz^m](z) Re((x + i y)^m): a polynomial in x, y, z.
The Legendre polynomials come from the explicit sum
P_l(z) = 2^-l sum_k (-1)^k C(l, k) C(2l - 2k, l) z^(l - 2k), with exact rational coefficients.
Coefficients are indexed l*l + l + m.
"""
from __future__ import annotations

import math
from fractions import Fraction

import torch

DEGREE = 3
NCOEF = (DEGREE + 1) ** 2


def legendre_coeffs(l: int) -> list[Fraction]:
    """Coefficients c[k] of z^k in P_l(z)."""
    c = [Fraction(0)] * (l + 1)
    for k in range(l // 2 + 1):
        c[l - 2 * k] += Fraction((-1) ** k * math.comb(l, k) * math.comb(2 * l - 2 * k, l), 2 ** l)
    return c


def derivative(c: list[Fraction], m: int) -> list[Fraction]:
    for _ in range(m):
        c = [c[k] * k for k in range(1, len(c))] or [Fraction(0)]
    return c


def _poly(c: list[Fraction], z: torch.Tensor) -> torch.Tensor:
    out = torch.zeros_like(z)
    for k in reversed(range(len(c))):
        out = out * z + float(c[k])
    return out


def _xy_power(x: torch.Tensor, y: torch.Tensor, m: int):
    """Real and imaginary parts of (x + i y)^m."""
    re, im = torch.ones_like(x), torch.zeros_like(x)
    for _ in range(m):
        re, im = re * x - im * y, re * y + im * x
    return re, im


def basis(dirs: torch.Tensor, degree: int = DEGREE) -> torch.Tensor:
    """Y_lm at unit directions [N, 3] -> [N, (degree+1)^2]."""
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    cols = [None] * ((degree + 1) ** 2)
    for l in range(degree + 1):
        pl = legendre_coeffs(l)
        for m in range(0, l + 1):
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            dp = _poly(derivative(pl, m), z) * ((-1) ** m)
            if m == 0:
                cols[l * l + l] = norm * dp
            else:
                re, im = _xy_power(x, y, m)
                cols[l * l + l + m] = math.sqrt(2.0) * norm * dp * re
                cols[l * l + l - m] = math.sqrt(2.0) * norm * dp * im
    return torch.stack(cols, dim=1)


def colour(sh: torch.Tensor, dirs: torch.Tensor) -> torch.Tensor:
    """c = max(0, sum_lm beta_lm Y_lm(dir) + 1/2) per channel; sh is [N, 16, 3]."""
    Y = basis(dirs)
    return torch.clamp_min((Y.unsqueeze(-1) * sh).sum(dim=1) + 0.5, 0.0)
