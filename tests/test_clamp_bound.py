"""The rounding bound behind the forward rasteriser's clamp-free batches, checked on the CPU.

The forward rasteriser leaves out the 0.99 clamp of alpha for a batch when every staged Gaussian
has alpha_cond <= 0.98 and S = |qa| Dx^2 + |qb| Dx Dy + |qc| Dy^2 <= 6e4 (Dx, Dy: the largest
pixel-centre offsets over the tile, q: the conic scaled to log2 units).  The argument: for a
positive-definite conic the exact exponent at the rounded offsets is <= 0, and the kernel's FP32
evaluation (a = (qa dx) dx, bx = qb dx, t = fma(qc, dy, bx), p = fma(dy, t, a)) adds at most
gamma_3 S < 0.0108, so alpha_cond * 2^p <= 0.98 * 2^0.0108 < 0.99.  These tests evaluate the
exponent as the kernel does, in float32 with fused multiply-adds emulated in float64 (exact
products), at every pixel centre of a tile for random and adversarial positive-definite conics,
and check the bound wherever the S test passes."""
from __future__ import annotations

import numpy as np

NEG_HALF_LOG2E = np.float32(-0.72134752044448170)
NEG_LOG2E = np.float32(-1.4426950408889634)


def _fma32(a, b, c):
    """float32 fused multiply-add: the float64 product of two float32 values is exact."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _exponents(u, v, a, b, c, x0, y0):
    """The kernel's float32 exponent at the 256 pixel centres of the tile whose first centre is
    (x0, y0), for Gaussians with mean (u, v) and conic (a, b, c); shape [n, 256]."""
    qa = (NEG_HALF_LOG2E * a).astype(np.float32)[:, None]
    qb = (NEG_LOG2E * b).astype(np.float32)[:, None]
    qc = (NEG_HALF_LOG2E * c).astype(np.float32)[:, None]
    px, py = np.meshgrid(np.arange(16, dtype=np.float32) + np.float32(x0),
                         np.arange(16, dtype=np.float32) + np.float32(y0))
    dx = (px.reshape(1, -1) - u[:, None]).astype(np.float32)
    dy = (py.reshape(1, -1) - v[:, None]).astype(np.float32)
    aa = ((qa * dx).astype(np.float32) * dx).astype(np.float32)
    bx = (qb * dx).astype(np.float32)
    t = _fma32(qc, dy, bx)
    return _fma32(dy, t, aa), (qa, qb, qc)


def _s_test(u, v, q, x0, y0):
    """The kernel's S test, in float32 as written there."""
    qa, qb, qc = (x[:, 0] for x in q)
    f = np.float32
    Dx = (np.maximum(np.abs(f(x0) - u), np.abs(f(x0) + f(15) - u)) * f(1.0001)).astype(np.float32)
    Dy = (np.maximum(np.abs(f(y0) - v), np.abs(f(y0) + f(15) - v)) * f(1.0001)).astype(np.float32)
    S = ((np.abs(qa) * Dx * Dx + np.abs(qb) * Dx * Dy + np.abs(qc) * Dy * Dy) * f(1.0001)).astype(np.float32)
    return S <= f(6e4)


def _random_conics(rng, n):
    """Positive-definite conics of 2D covariances: scales from 0.3 px (the dilation's floor) to
    300 px, aspect ratios down to 1e-3 (close to singular), any orientation."""
    s1 = np.exp(rng.uniform(np.log(0.3), np.log(300.0), n))
    s2 = s1 * np.exp(rng.uniform(np.log(1e-3), 0.0, n))
    s2 = np.maximum(s2, 0.3)
    th = rng.uniform(0, np.pi, n)
    cs, sn = np.cos(th), np.sin(th)
    cxx = cs ** 2 * s1 ** 2 + sn ** 2 * s2 ** 2
    cyy = sn ** 2 * s1 ** 2 + cs ** 2 * s2 ** 2
    cxy = cs * sn * (s1 ** 2 - s2 ** 2)
    det = cxx * cyy - cxy ** 2
    a, b, c = cyy / det, -cxy / det, cxx / det
    return a.astype(np.float32), b.astype(np.float32), c.astype(np.float32)


def test_clamp_free_bound_holds_at_every_pixel_of_the_tile():
    rng = np.random.default_rng(2024)
    worst, passed = -np.inf, 0
    for trial in range(40):
        n = 2000
        x0, y0 = 16 * int(rng.integers(0, 60)) + 0.5, 16 * int(rng.integers(0, 60)) + 0.5
        # means near the tile (inside, at its edge) and far from it (large Gaussians)
        off = rng.choice([4.0, 20.0, 200.0, 1000.0])
        u = (x0 + 7.5 + rng.uniform(-off, off, n)).astype(np.float32)
        v = (y0 + 7.5 + rng.uniform(-off, off, n)).astype(np.float32)
        a, b, c = _random_conics(rng, n)
        pd = (a > 0) & ((a * c).astype(np.float32) - (b * b).astype(np.float32) > 0)
        p, q = _exponents(u, v, a, b, c, x0, y0)
        ok = _s_test(u, v, q, x0, y0) & pd
        passed += int(ok.sum())
        if ok.any():
            worst = max(worst, float(p[ok].max()))
    assert passed > 10000  # most random Gaussians pass the S test
    assert worst <= 0.0108, worst
    # and the opacity condition keeps alpha below the clamp with room to spare
    assert 0.98 * 2.0 ** 0.0108 * (1 + 1e-6) < 0.99


def test_clamp_free_bound_on_centred_near_singular_conics():
    """Pixel centres on or next to the Gaussian's centre, where the exact exponent is ~0 and
    rounding can make the computed one positive: the S test keeps it within the bound."""
    rng = np.random.default_rng(7)
    n = 20000
    x0, y0 = 400.5, 400.5
    u = (x0 + rng.integers(0, 16, n) + rng.uniform(-1e-3, 1e-3, n)).astype(np.float32)
    v = (y0 + rng.integers(0, 16, n) + rng.uniform(-1e-3, 1e-3, n)).astype(np.float32)
    # long thin Gaussians (aspect down to 1e-3) at every orientation
    s1 = np.exp(rng.uniform(np.log(1.0), np.log(300.0), n))
    s2 = np.full(n, 0.3)
    th = rng.uniform(0, np.pi, n)
    cs, sn = np.cos(th), np.sin(th)
    cxx = cs ** 2 * s1 ** 2 + sn ** 2 * s2 ** 2
    cyy = sn ** 2 * s1 ** 2 + cs ** 2 * s2 ** 2
    cxy = cs * sn * (s1 ** 2 - s2 ** 2)
    det = cxx * cyy - cxy ** 2
    a, b, c = (x.astype(np.float32) for x in (cyy / det, -cxy / det, cxx / det))
    pd = (a > 0) & ((a * c).astype(np.float32) - (b * b).astype(np.float32) > 0)
    p, q = _exponents(u, v, a, b, c, x0, y0)
    ok = _s_test(u, v, q, x0, y0) & pd
    assert ok.mean() > 0.9
    assert float(p[ok].max()) <= 0.0108


def _near_singular_along_diagonal(rng, n, x0, y0):
    """Conics k [[1, -(1 - e)], [-(1 - e), 1]] with e down to the float32 limit of positive
    definiteness, each centred on the tile's diagonal line at a distance d: along that line the
    exact exponent is -k e d^2 (tiny) while its terms are ~k d^2, so rounding can make the
    computed exponent positive."""
    k = np.exp(rng.uniform(np.log(1e-4), np.log(3.3), n)).astype(np.float32)
    e = rng.choice([6e-8, 1.2e-7, 1e-6, 1e-5], n)
    b = (-k * (1 - e)).astype(np.float32)
    d = rng.uniform(-3000, 3000, n).astype(np.float32)
    u = (np.float32(x0 + 7.5) - d).astype(np.float32)
    v = (np.float32(y0 + 7.5) - d).astype(np.float32)
    return u, v, k, b, k


def test_clamp_free_bound_on_adversarial_cancellation():
    """Near-singular conics along their degenerate direction: the computed exponent is positive at
    many pixels, the S test keeps it below the bound's 0.0108, and without the S test (a threshold
    100 times larger) the bound would fail."""
    rng = np.random.default_rng(11)
    worst, worst_loose, positive, passed = -np.inf, -np.inf, 0, 0
    x0 = y0 = 400.5
    for _ in range(30):
        u, v, a, b, c = _near_singular_along_diagonal(rng, 4000, x0, y0)
        pd = (a > 0) & ((a * c).astype(np.float32) - (b * b).astype(np.float32) > 0)
        p, q = _exponents(u, v, a, b, c, x0, y0)
        ok = _s_test(u, v, q, x0, y0) & pd
        passed += int(ok.sum())
        positive += int((p[ok] > 0).any(axis=1).sum())
        worst = max(worst, float(p[ok].max()))
        # the same Gaussians under a 100 times looser S threshold
        qa, qb, qc = (x[:, 0] for x in q)
        f = np.float32
        Dx = np.maximum(np.abs(f(x0) - u), np.abs(f(x0) + f(15) - u))
        Dy = np.maximum(np.abs(f(y0) - v), np.abs(f(y0) + f(15) - v))
        S = np.abs(qa) * Dx * Dx + np.abs(qb) * Dx * Dy + np.abs(qc) * Dy * Dy
        loose = (S <= 6e6) & pd
        worst_loose = max(worst_loose, float(p[loose].max()))
    assert passed > 50000 and positive > 5000  # the family does produce positive exponents
    assert worst <= 0.0108, worst
    assert worst_loose > 0.0108, worst_loose
