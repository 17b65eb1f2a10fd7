"""Front-to-back alpha compositing of depth-sorted 2D Gaussians (oracle, float64).

The paper blends the projected Gaussians in depth order by opacity, with the 3DGS differentiable
rasteriser (Sec. 4.4).  The rules, fixed here as readings of that rasteriser:
  * a Gaussian is considered at a pixel iff the pixel's 16x16 tile lies in its tile rectangle
    (callers build the candidate lists; `render.composite_all` does so from the rectangles alone
    unless asked to apply the binning's reachability rule as well); candidates are visited in
    ascending (depth, id) order;
  * power = -1/2 (a dx^2 + c dy^2) - b dx dy with (dx, dy) = pixel centre - mean, conic [[a,b],[b,c]];
  * alpha_i = min(0.99, alpha_cond exp(power)); skip when power > 0 or alpha_i < 1/255;
  * T_next = T (1 - alpha_i); if T_next < 1e-4 stop *without* adding this Gaussian;
  * C += c_i alpha_i T; T = T_next; out = C + T_final bg.
  * n_contrib = 1 + position (in the tile list) of the last Gaussian added, 0 if none; last_id is
    that Gaussian's id (-1 if none), which does not depend on which skipped candidates a list holds.

`composite_tile` evaluates all candidates of one tile at once: the transmittance in front of
candidate k is the running product of (1 - alpha_j) over the candidates j < k that were not
skipped, and the stop position is the first candidate whose product drops below 1e-4.  This is
the same sequence of operations as the per-pixel loop in `composite_pixel_loop` (kept for tiny
cases and as its check).
"""
from __future__ import annotations

import torch

ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4
IMPACT = 5e-5  # colour change below which a flipped decision is harmless (tolerance 2e-4)


def composite_tile(pix: torch.Tensor, g: torch.Tensor, mean2d: torch.Tensor, conic: torch.Tensor,
                   alpha_cond: torch.Tensor, rgb: torch.Tensor, bg: torch.Tensor,
                   depth: torch.Tensor | None = None) -> dict:
    """pix [P, 2] pixel centres; g [n] candidate ids in (depth, id) order.

    Returns colour [P, 3], final_T [P], n_contrib [P] (int64), last_id [P] (int64, -1 if no
    Gaussian was added) and margin: a dict of [P] tensors
    with the smallest relative distance of the pixel's decisions to their thresholds (alpha vs
    1/255, T vs 1e-4, relative depth gap of neighbouring candidates up to the stop).
    """
    P = pix.shape[0]
    n = int(g.shape[0])
    dtype = mean2d.dtype
    if n == 0:
        inf = torch.full((P,), float("inf"), dtype=dtype)
        return dict(color=bg.expand(P, 3).clone(), final_T=torch.ones(P, dtype=dtype),
                    n_contrib=torch.zeros(P, dtype=torch.int64),
                    last_id=torch.full((P,), -1, dtype=torch.int64),
                    margin=dict(alpha=inf, T=inf.clone(), depth=inf.clone()))
    m = mean2d[g]
    q = conic[g]
    dx = pix[None, :, 0] - m[:, 0:1]
    dy = pix[None, :, 1] - m[:, 1:2]
    power = -0.5 * (q[:, 0:1] * dx * dx + q[:, 2:3] * dy * dy) - q[:, 1:2] * dx * dy
    alpha = torch.clamp_max(alpha_cond[g][:, None] * torch.exp(power), ALPHA_MAX)
    valid = (power <= 0) & (alpha >= ALPHA_MIN)
    a_eff = torch.where(valid, alpha, torch.zeros_like(alpha))
    T_incl = torch.cumprod(1.0 - a_eff, dim=0)
    T_excl = torch.cat([torch.ones(1, P, dtype=dtype), T_incl[:-1]], dim=0)
    with torch.no_grad():
        stop = valid & (T_incl < T_MIN)
        has_stop = stop.any(dim=0)
        s = torch.where(has_stop, torch.argmax(stop.to(torch.int8), dim=0), torch.full((P,), n))
        idx = torch.arange(n)[:, None]
        keep = valid & (idx < s[None, :])
        n_contrib = torch.where(keep.any(0), (idx.expand(n, P) * keep).max(0).values + 1,
                                torch.zeros(P, dtype=torch.int64))
        # Decision margins, counted only where flipping the decision could move the colour by
        # more than IMPACT: alpha vs 1/255 (impact ~ 2 T / 255), the stop test T_next < 1e-4
        # (impact ~ alpha T) and the order of neighbouring candidates (impact ~ alpha_k alpha_k+1 T).
        considered = idx <= s[None, :]
        big = torch.full_like(alpha, float("inf"))
        m_alpha = torch.where(considered & (power <= 0) & (2.0 * ALPHA_MIN * T_excl > IMPACT),
                              torch.abs(alpha - ALPHA_MIN) / ALPHA_MIN, big).min(0).values
        m_T = torch.where(considered & valid & (a_eff * T_excl > IMPACT),
                          torch.abs(T_incl - T_MIN) / T_MIN, big).min(0).values
        m_z = torch.full((P,), float("inf"), dtype=dtype)
        if depth is not None and n > 1:
            z = depth[g]
            gap = (torch.abs(z[1:] - z[:-1]) / torch.abs(z[:-1]))[:, None].expand(n - 1, P)
            pair = a_eff[1:] * a_eff[:-1] * T_excl[:-1]
            m_z = torch.where((idx[1:] <= s[None, :]) & (pair > IMPACT), gap, big[1:]).min(0).values
        margin = dict(alpha=m_alpha, T=m_T, depth=m_z)
    w = a_eff * T_excl * keep
    color = (w[:, :, None] * rgb[g][:, None, :]).sum(0)
    last = torch.clamp(s, max=n - 1)
    T_stop = torch.gather(T_excl, 0, last[None, :])[0]
    final_T = torch.where(has_stop, T_stop, T_incl[-1])
    color = color + final_T[:, None] * bg[None, :]
    last_id = torch.where(n_contrib > 0, g.to(torch.int64)[torch.clamp(n_contrib - 1, min=0)],
                          torch.full_like(n_contrib, -1))
    return dict(color=color, final_T=final_T, n_contrib=n_contrib, last_id=last_id, margin=margin)


def composite_pixel_loop(px: float, py: float, g, mean2d, conic, alpha_cond, rgb, bg):
    """The per-pixel loop, one candidate at a time (plain Python floats, tiny cases only)."""
    T = 1.0
    C = [0.0, 0.0, 0.0]
    last = 0
    for k, gi in enumerate(g):
        dx = px - float(mean2d[gi][0])
        dy = py - float(mean2d[gi][1])
        a, b, c = (float(v) for v in conic[gi])
        power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        if power > 0.0:
            continue
        alpha = min(ALPHA_MAX, float(alpha_cond[gi]) * float(torch.exp(torch.tensor(power, dtype=torch.float64))))
        if alpha < ALPHA_MIN:
            continue
        T_next = T * (1.0 - alpha)
        if T_next < T_MIN:
            break
        for ch in range(3):
            C[ch] += float(rgb[gi][ch]) * alpha * T
        T = T_next
        last = k + 1
    return [C[ch] + T * float(bg[ch]) for ch in range(3)], T, last
