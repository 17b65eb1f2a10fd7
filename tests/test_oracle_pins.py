"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a closed form, a textbook
identity, a special case the paper prints, brute force on a tiny input, or a finite difference.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest
import torch

import synth
from oracle import binning, composite, projection, render, sh, slicing

F64 = torch.float64


def _random_L(rng, n, scale=0.1):
    """Well-conditioned random Cholesky factors (cond(Sigma) ~ 1e2), so FP64 identities hold to 1e-10."""
    L = np.tril(rng.normal(0.0, scale, size=(n, 7, 7)))
    for i in range(7):
        L[:, i, i] = np.exp(rng.uniform(np.log(0.2), np.log(0.6), size=n))
    return L


def _pack(L):
    rows, cols = np.tril_indices(7)
    return L[:, rows, cols]


def _mvn_logpdf(x, mu, S):
    """log N(x; mu, S) written from the density, via a Cholesky-free solve and slogdet."""
    k = x.shape[-1]
    diff = (x - mu)
    sol = torch.linalg.solve(S, diff.unsqueeze(-1)).squeeze(-1)
    _, logdet = torch.linalg.slogdet(S)
    return -0.5 * (diff * sol).sum(-1) - 0.5 * logdet - 0.5 * k * math.log(2 * math.pi)


# ----------------------------------------------------------------------------------------------
# Slicing: Eq. cond_mean / cond_cov / temp_mod / dir_mod (Sec. 4.2, Algorithm 1 steps 3-6)
# ----------------------------------------------------------------------------------------------

def test_unpack_matches_packed_layout():
    rng = np.random.default_rng(1)
    L = _random_L(rng, 5)
    got = slicing.unpack_L(torch.tensor(_pack(L))).numpy()
    np.testing.assert_array_equal(got, L)
    # element (i, j) lives at i(i+1)/2 + j
    L28 = torch.arange(28, dtype=F64).reshape(1, 28)
    U = slicing.unpack_L(L28)[0]
    for i in range(7):
        for j in range(i + 1):
            assert U[i, j] == i * (i + 1) // 2 + j


def test_density_factorisation_pins_conditioning():
    """N7((x_p, t, d)) / N3(x_p; mu_cond, Sigma_cond) is constant in x_p and equals N4((t, d))."""
    rng = np.random.default_rng(2)
    n = 16
    L = torch.tensor(_random_L(rng, n))
    mean7 = torch.tensor(rng.normal(size=(n, 7)))
    t = 0.37
    d = np.array([0.2, -0.5, 0.84])
    Sigma = slicing.covariance(L)
    mu_c, S_c = slicing.condition(mean7, Sigma, t, d)
    td = torch.tensor(np.concatenate([[t], d]))
    log_marg = _mvn_logpdf(td.expand(n, 4), mean7[:, 3:], Sigma[:, 3:, 3:])
    for _ in range(4):
        xp = torch.tensor(rng.normal(size=(n, 3)))
        x7 = torch.cat([xp, td.expand(n, 4)], 1)
        ratio = _mvn_logpdf(x7, mean7, Sigma) - _mvn_logpdf(xp, mu_c, S_c)
        np.testing.assert_allclose(ratio.numpy(), log_marg.numpy(), rtol=0, atol=1e-10)


def test_block_diagonal_static_case_is_plain_3dgs():
    """Block-diagonal L with t = mu_t, d = mu_d: mu_cond = mu_p, Sigma_cond = L_pp L_pp^T, f = 1."""
    rng = np.random.default_rng(3)
    n = 8
    L = _random_L(rng, n)
    L[:, 3:, :3] = 0.0  # no p <-> (t, d) coupling
    L[:, 4:, 3] = 0.0  # no t <-> d coupling
    mean7 = rng.normal(size=(n, 7))
    for i in range(n):
        mu_t, mu_d = mean7[i, 3], mean7[i, 4:]
        Ls = torch.tensor(L[i:i + 1])
        Sigma = slicing.covariance(Ls)
        m = torch.tensor(mean7[i:i + 1])
        mu_c, S_c = slicing.condition(m, Sigma, mu_t, mu_d)
        np.testing.assert_allclose(mu_c.numpy()[0], mean7[i, :3], rtol=0, atol=1e-14)
        Lpp = L[i, :3, :3]
        np.testing.assert_allclose(S_c.numpy()[0], Lpp @ Lpp.T, rtol=0, atol=1e-14)
        ft, fd = slicing.modulation(m, Sigma, mu_t, mu_d, 0.7, 0.9)
        assert ft.item() == 1.0 and fd.item() == 1.0
        # away from mu_t the geometry is unchanged and only the opacity drops
        mu_c2, S_c2 = slicing.condition(m, Sigma, mu_t + 0.3, mu_d)
        np.testing.assert_allclose(mu_c2.numpy()[0], mean7[i, :3], atol=1e-14)
        np.testing.assert_allclose(S_c2.numpy()[0], Lpp @ Lpp.T, atol=1e-14)
        ft2, _ = slicing.modulation(m, Sigma, mu_t + 0.3, mu_d, 0.7, 0.9)
        assert ft2.item() < 1.0


def _sigma_from_blocks(rng, zero_pt=False, zero_pd=False, zero_td=False):
    A = rng.normal(size=(7, 7))
    S = A @ A.T + 7 * np.eye(7)
    if zero_pt:
        S[:3, 3] = S[3, :3] = 0.0
    if zero_pd:
        S[:3, 4:] = S[4:, :3] = 0.0
    if zero_td:
        S[3, 4:] = S[4:, 3] = 0.0
    return S


def test_reduces_to_6dgs_conditioning():
    """Sigma_pt = Sigma_td = 0 and t = mu_t: the 6DGS formulas of Sec. 3 (direction only)."""
    rng = np.random.default_rng(4)
    S = _sigma_from_blocks(rng, zero_pt=True, zero_td=True)
    L = np.linalg.cholesky(S)
    mean7 = rng.normal(size=7)
    d = np.array([0.3, 0.1, -0.9])
    mu_c, S_c = slicing.condition(torch.tensor(mean7[None]), slicing.covariance(torch.tensor(L[None])),
                                  mean7[3], d)
    Spd, Sd = S[:3, 4:], S[4:, 4:]
    want_mu = mean7[:3] + Spd @ np.linalg.solve(Sd, d - mean7[4:])
    want_S = S[:3, :3] - Spd @ np.linalg.solve(Sd, Spd.T)
    np.testing.assert_allclose(mu_c.numpy()[0], want_mu, atol=1e-12)
    np.testing.assert_allclose(S_c.numpy()[0], want_S, atol=1e-12)


def test_reduces_to_scalar_time_conditioning():
    """Sigma_pd = Sigma_td = 0 and d = mu_d: the scalar Schur complement in time."""
    rng = np.random.default_rng(5)
    S = _sigma_from_blocks(rng, zero_pd=True, zero_td=True)
    L = np.linalg.cholesky(S)
    mean7 = rng.normal(size=7)
    t = mean7[3] + 0.8
    mu_c, S_c = slicing.condition(torch.tensor(mean7[None]), slicing.covariance(torch.tensor(L[None])),
                                  t, mean7[4:])
    Spt, St = S[:3, 3], S[3, 3]
    np.testing.assert_allclose(mu_c.numpy()[0], mean7[:3] + Spt * (t - mean7[3]) / St, atol=1e-12)
    np.testing.assert_allclose(S_c.numpy()[0], S[:3, :3] - np.outer(Spt, Spt) / St, atol=1e-12)


def test_conditional_covariance_spd_and_schur_determinant():
    rng = np.random.default_rng(6)
    n = 64
    L = torch.tensor(_random_L(rng, n))
    Sigma = slicing.covariance(L)
    mean7 = torch.tensor(rng.normal(size=(n, 7)))
    _, S_c = slicing.condition(mean7, Sigma, 0.5, [0.0, 0.0, 1.0])
    assert torch.all(torch.linalg.eigvalsh(S_c) > 0)
    det_ratio = torch.linalg.det(Sigma) / torch.linalg.det(Sigma[:, 3:, 3:])
    np.testing.assert_allclose(torch.linalg.det(S_c).numpy(), det_ratio.numpy(), rtol=1e-9)
    # precision-matrix identity: Sigma_cond = ((Sigma^-1)_pp)^-1
    prec = torch.linalg.inv(Sigma)
    np.testing.assert_allclose(S_c.numpy(), torch.linalg.inv(prec[:, :3, :3]).numpy(), rtol=1e-8,
                               atol=1e-12)


def test_modulation_is_scaled_marginal_density_ratio():
    """With lambda = 1, f_temp and f_dir are the marginal densities of t and d over their peaks."""
    rng = np.random.default_rng(7)
    n = 16
    L = torch.tensor(_random_L(rng, n))
    Sigma = slicing.covariance(L)
    mean7 = torch.tensor(rng.normal(size=(n, 7)))
    t, d = 0.25, np.array([0.6, 0.0, 0.8])
    ft, fd = slicing.modulation(mean7, Sigma, t, d, 1.0, 1.0)
    tt = torch.full((n, 1), t, dtype=F64)
    lt = _mvn_logpdf(tt, mean7[:, 3:4], Sigma[:, 3:4, 3:4]) - _mvn_logpdf(mean7[:, 3:4], mean7[:, 3:4],
                                                                          Sigma[:, 3:4, 3:4])
    dd = torch.tensor(d).expand(n, 3)
    ld = _mvn_logpdf(dd, mean7[:, 4:], Sigma[:, 4:, 4:]) - _mvn_logpdf(mean7[:, 4:], mean7[:, 4:],
                                                                      Sigma[:, 4:, 4:])
    np.testing.assert_allclose(torch.log(ft).numpy(), lt.numpy(), atol=1e-10)
    np.testing.assert_allclose(torch.log(fd).numpy(), ld.numpy(), atol=1e-10)
    # lambda scales the exponent
    ft2, fd2 = slicing.modulation(mean7, Sigma, t, d, 0.05, 0.3)
    np.testing.assert_allclose(torch.log(ft2).numpy(), 0.05 * lt.numpy(), atol=1e-10)
    np.testing.assert_allclose(torch.log(fd2).numpy(), 0.3 * ld.numpy(), atol=1e-10)
    sl = slicing.slice_gaussians(mean7, torch.tensor(_pack(L.numpy())), torch.full((n,), 0.8, dtype=F64),
                                 t, d, 0.05, 0.3)
    a = sl["alpha_cond"].numpy()
    assert np.all(a >= 0) and np.all(a <= 0.8)


# ----------------------------------------------------------------------------------------------
# SH colour (Sec. 3 colour model, kept by Sec. 4.1)
# ----------------------------------------------------------------------------------------------

def test_sh_matches_textbook_cartesian_table(golden_dir):
    rng = np.random.default_rng(8)
    v = rng.normal(size=(32, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    Y = sh.basis(torch.tensor(v)).numpy()
    rows = [ln.split(None, 3) for ln in open(os.path.join(golden_dir, "real_sh_cartesian.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 16
    for l, m, sign, expr in rows:
        l, m, sign = int(l), int(m), int(sign)
        ns = dict(x=v[:, 0], y=v[:, 1], z=v[:, 2], pi=math.pi, sqrt=np.sqrt)
        want = sign * eval(expr, {"__builtins__": {}}, ns)
        np.testing.assert_allclose(Y[:, l * l + l + m], want, rtol=1e-13, atol=1e-13)


def test_sh_orthonormal_by_quadrature():
    """Gauss-Legendre in z times a uniform grid in phi integrates degree <= 6 polynomials exactly."""
    zs, wz = np.polynomial.legendre.leggauss(8)
    phis = np.arange(16) * 2 * np.pi / 16
    Z, P = np.meshgrid(zs, phis, indexing="ij")
    W = np.repeat(wz, 16) * (2 * np.pi / 16)
    s = np.sqrt(1 - Z ** 2)
    dirs = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
    Y = sh.basis(torch.tensor(dirs)).numpy()
    gram = (Y * W[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-13)


def test_sh_colour_dc_only_is_view_independent():
    rng = np.random.default_rng(9)
    coeffs = np.zeros((1, 16, 3))
    coeffs[0, 0] = [0.3, -0.2, 0.9]
    v = rng.normal(size=(10, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    c = sh.colour(torch.tensor(coeffs).expand(10, 16, 3), torch.tensor(v)).numpy()
    want = np.maximum(0.0, 0.5 / math.sqrt(math.pi) * np.array([0.3, -0.2, 0.9]) + 0.5)
    np.testing.assert_allclose(c, np.tile(want, (10, 1)), atol=1e-15)


# ----------------------------------------------------------------------------------------------
# Projection
# ----------------------------------------------------------------------------------------------

def test_ewa_covariance_matches_numerical_jacobian():
    """Sigma_2D - 0.3 I = dpi/dp Sigma_cam dpi/dp^T with dpi/dp by central differences of pi."""
    rng = np.random.default_rng(10)
    cam = synth.config_cameras(1, count=1, width=128, height=96)[0]  # a rotated camera
    n = 12
    mu = torch.tensor(rng.uniform(-0.3, 0.3, size=(n, 3)))
    A = rng.normal(size=(n, 3, 3)) * 0.1
    S = torch.tensor(A @ A.transpose(0, 2, 1) + 0.01 * np.eye(3))
    pr = projection.project(mu, S, cam)
    R = cam.viewmat[:3, :3]
    tv = cam.viewmat[:3, 3]

    def pi(p):
        return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])

    for i in range(n):
        p = R @ mu[i].numpy() + tv
        h = 1e-6
        Jn = np.stack([(pi(p + h * e) - pi(p - h * e)) / (2 * h) for e in np.eye(3)], 1)
        want = Jn @ (R @ S[i].numpy() @ R.T) @ Jn.T + 0.3 * np.eye(2)
        a, b, c = pr["cov2d"][i].numpy()
        np.testing.assert_allclose([[a, b], [b, c]], want, rtol=1e-7)
        np.testing.assert_allclose(pr["mean2d"][i].numpy(), pi(p), rtol=1e-14)
        q = pr["conic"][i].numpy()
        np.testing.assert_allclose(np.array([[q[0], q[1]], [q[1], q[2]]]) @ want, np.eye(2), atol=1e-9)
        lam = np.linalg.eigvalsh(want).max()
        np.testing.assert_allclose(pr["extent"][i].item(), 3 * np.sqrt(lam), rtol=1e-8)


def test_tile_rect_matches_brute_force_intersection():
    rng = np.random.default_rng(11)
    W, H = 100, 70
    tx, ty = 7, 5
    u = torch.tensor(rng.uniform(-40, 140, size=300))
    v = torch.tensor(rng.uniform(-40, 110, size=300))
    r = torch.tensor(rng.integers(0, 40, size=300).astype(np.float64))
    u[:20] = torch.tensor(rng.integers(0, 7, size=20) * 16.0) + r[:20]  # edges exactly on tile borders
    rect = projection.tile_rect(u, v, r, tx, ty).numpy()
    for i in range(300):
        want = np.zeros((ty, tx), bool)
        for j in range(ty):
            for k in range(tx):
                # closed square [u-r, u+r] meets the half-open box [16k, 16k+16)
                want[j, k] = (16 * k <= u[i] + r[i]) and (u[i] - r[i] < 16 * k + 16) and \
                             (16 * j <= v[i] + r[i]) and (v[i] - r[i] < 16 * j + 16)
        got = np.zeros((ty, tx), bool)
        got[rect[i, 1]:rect[i, 3], rect[i, 0]:rect[i, 2]] = True
        assert np.array_equal(got, want), i


# ----------------------------------------------------------------------------------------------
# Binning and compositing
# ----------------------------------------------------------------------------------------------

def test_binning_matches_python_sort_of_tuples():
    rec = synth.random_projected(300, 100, 70, seed=12)
    keys, vals = binning.sort_keys(rec["depth"], rec["rect"], 7)
    tuples = []
    for g in range(300):
        rx0, ry0, rx1, ry1 = rec["rect"][g]
        for y in range(ry0, ry1):
            for x in range(rx0, rx1):
                tuples.append((y * 7 + x, float(rec["depth"][g]), g))
    tuples.sort()
    assert [int(k >> np.uint64(32)) for k in keys] == [t[0] for t in tuples]
    assert [int(v) for v in vals] == [t[2] for t in tuples]
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)
    ranges = binning.tile_ranges(keys, 35)
    counts = np.bincount([t[0] for t in tuples], minlength=35)
    np.testing.assert_array_equal(ranges[:, 1] - ranges[:, 0], counts)
    lists = binning.tile_lists(rec["depth"], rec["rect"], 7, 35)
    for tile in range(35):
        np.testing.assert_array_equal(lists[tile], vals[ranges[tile, 0]:ranges[tile, 1]])


def test_single_gaussian_closed_form():
    """One Gaussian on the optical axis with an axis-aligned Sigma_cond: every pixel is
    alpha_i c + (1 - alpha_i) bg with Sigma_2D = diag(fx^2 sx^2 / z^2, fy^2 sy^2 / z^2) + 0.3 I."""
    sx, sy, sz = 0.05, 0.08, 0.03
    L = np.zeros((1, 7, 7))
    np.fill_diagonal(L[0], [sx, sy, sz, 0.2, 0.3, 0.3, 0.3])
    mean7 = np.array([[0.0, 0.0, 0.0, 0.5, 0.0, 0.0, 1.0]], dtype=np.float32)
    coeffs = np.zeros((1, 16, 3), np.float32)
    coeffs[0, 0] = [0.4, 0.1, -0.3]
    scene = synth.Scene(mean7, _pack(L).astype(np.float32), np.array([0.7], np.float32), coeffs,
                        0.05, 0.05, (0.2, 0.3, 0.4))
    cam = synth.make_camera((0.0, 0.0, -3.0), 64, 48, 60.0, 0.5, bg=(0.2, 0.3, 0.4))
    out = render.render(scene, cam)
    L32 = _pack(L).astype(np.float32).astype(np.float64)
    sx2, sy2 = L32[0, 0] ** 2, L32[0, 2] ** 2
    z = 3.0
    a = cam.fx ** 2 * sx2 / z ** 2 + 0.3
    c = cam.fy ** 2 * sy2 / z ** 2 + 0.3
    col = np.maximum(0.0, 0.5 / math.sqrt(math.pi) * coeffs[0, 0].astype(np.float64) + 0.5)
    alpha0 = float(np.float32(0.7))
    ys, xs = np.mgrid[0:48, 0:64]
    dx, dy = xs + 0.5 - 32.0, ys + 0.5 - 24.0
    al = np.minimum(0.99, alpha0 * np.exp(-0.5 * (dx * dx / a + dy * dy / c)))
    al = np.where(al >= 1 / 255, al, 0.0)
    r = math.ceil(3 * math.sqrt(max(a, c)))
    inside = (np.floor((32 - r) / 16) * 16 <= xs) & (xs < (np.floor((32 + r) / 16) + 1) * 16) & \
             (np.floor((24 - r) / 16) * 16 <= ys) & (ys < (np.floor((24 + r) / 16) + 1) * 16)
    al = np.where(inside, al, 0.0)
    want = al[..., None] * col + (1 - al[..., None]) * np.array(cam.bg)
    np.testing.assert_allclose(out["image"].numpy(), want, atol=1e-12)


def test_colour_is_evaluated_toward_the_gaussian_from_the_camera():
    """SH colour at dir = (mu_cond - camera centre) / |.|, checked with the textbook l = 1 terms."""
    rng = np.random.default_rng(18)
    n = 6
    L = np.zeros((n, 7, 7))
    for i in range(n):
        np.fill_diagonal(L[i], [0.05, 0.05, 0.05, 0.2, 0.3, 0.3, 0.3])
    mean7 = np.zeros((n, 7), np.float32)
    mean7[:, :3] = rng.uniform(-0.6, 0.6, size=(n, 3))
    mean7[:, 3] = 0.5
    mean7[:, 6] = 1.0
    coeffs = np.zeros((n, 16, 3), np.float32)
    coeffs[:, 0] = 0.3
    coeffs[:, 1:4] = rng.normal(0, 0.2, size=(n, 3, 3))
    scene = synth.Scene(mean7, _pack(L).astype(np.float32), np.full(n, 0.5, np.float32), coeffs,
                        0.05, 0.05)
    cam = synth.make_camera((0.4, -0.2, -3.0), 64, 64, 60.0, 0.5)
    g = render.render(scene, cam)["g"]
    c1 = math.sqrt(3 / (4 * math.pi))
    for i in range(n):
        v = mean7[i, :3].astype(np.float64) - np.array([0.4, -0.2, -3.0])
        x, y, z = v / np.linalg.norm(v)
        want = 0.5 / math.sqrt(math.pi) * coeffs[i, 0] + c1 * (-y * coeffs[i, 1] + z * coeffs[i, 2]
                                                                 - x * coeffs[i, 3]) + 0.5
        np.testing.assert_allclose(g["rgb"][i].numpy(), np.maximum(want, 0), atol=1e-7)


def test_compositing_invariants():
    rec = synth.random_projected(200, 64, 64, seed=13)
    out = render.render_projected(rec, 64, 64, (0.0, 0.0, 0.0))
    # weights + final transmittance = 1: with white Gaussians on black, image = 1 - T_final
    white = dict(rec, rgb=np.ones_like(rec["rgb"]))
    o2 = render.render_projected(white, 64, 64, (0.0, 0.0, 0.0))
    np.testing.assert_allclose(o2["image"].numpy(), np.repeat(1 - o2["final_T"].numpy()[..., None], 3, -1),
                               atol=1e-12)
    # every colour equal to the background: the image is that colour
    grey = dict(rec, rgb=np.full_like(rec["rgb"], 0.25))
    o3 = render.render_projected(grey, 64, 64, (0.25, 0.25, 0.25))
    np.testing.assert_allclose(o3["image"].numpy(), 0.25, atol=1e-12)
    assert np.all(out["final_T"].numpy() >= 1e-4 * 0.0) and np.all(out["final_T"].numpy() <= 1.0)


def test_transmittance_monotone_and_stop_rule():
    rec = synth.random_projected(400, 32, 32, seed=14, max_half_tiles=2)
    rec["opacity"] = np.full_like(rec["opacity"], 0.95)
    lists = binning.tile_lists(rec["depth"], rec["rect"], 2, 4)
    f = lambda k: np.asarray(rec[k], np.float32).astype(np.float64)
    for (px, py) in [(3.5, 4.5), (20.5, 9.5), (30.5, 30.5)]:
        tile = int(py // 16) * 2 + int(px // 16)
        T = 1.0
        g = lists[tile]
        col, Tf, last = composite.composite_pixel_loop(px, py, g, f("mean2d"), f("conic"), f("opacity"),
                                                       f("rgb"), (0, 0, 0))
        # replay: T never increases and never drops below 1e-4
        for gi in g[:last]:
            dx, dy = px - f("mean2d")[gi][0], py - f("mean2d")[gi][1]
            a, b, c = f("conic")[gi]
            al = min(0.99, f("opacity")[gi] * math.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy))
            if al >= 1 / 255:
                assert T * (1 - al) <= T
                T *= 1 - al
        assert abs(T - Tf) < 1e-15 and Tf >= 1e-4


def test_vectorised_compositing_equals_per_pixel_loop():
    rec = synth.random_projected(150, 48, 32, seed=15)
    out = render.render_projected(rec, 48, 32, (0.1, 0.2, 0.3))
    lists = binning.tile_lists(rec["depth"], rec["rect"], 3, 6)
    f = lambda k: np.asarray(rec[k], np.float32).astype(np.float64)
    for y in range(0, 32, 3):
        for x in range(0, 48, 5):
            tile = (y // 16) * 3 + x // 16
            col, T, last = composite.composite_pixel_loop(x + 0.5, y + 0.5, lists[tile], f("mean2d"),
                                                          f("conic"), f("opacity"), f("rgb"), (0.1, 0.2, 0.3))
            np.testing.assert_allclose(out["image"][y, x].numpy(), col, atol=1e-13)
            assert out["n_contrib"][y, x].item() == last
            assert abs(out["final_T"][y, x].item() - T) < 1e-13


def test_reachability_filter_changes_no_pixel():
    """Compositing over the rectangle lists (the blending rule as stated) and over the lists the
    binning's reachability rule keeps gives the same image, transmittance and last contributor:
    the rule only drops candidates that every pixel of the tile skips."""
    scene = synth.config_scene(0)
    cam = synth.config_cameras(0)[0]
    full = render.render(scene, cam)
    kept = render.render(scene, cam, reach=True)
    # (the colour sums run over lists of different length, so only their rounding may differ)
    assert float((full["image"] - kept["image"]).abs().max()) < 1e-12
    assert torch.equal(full["final_T"], kept["final_T"])
    assert torch.equal(full["last_id"], kept["last_id"])
    assert (full["last_id"] >= 0).float().mean() > 0.5
    # the filtered lists are much shorter, so positions differ while the contributors agree
    assert (full["n_contrib"] >= kept["n_contrib"]).all()
    assert (full["n_contrib"] > kept["n_contrib"]).any()
    rec = synth.random_projected(400, 80, 64, seed=21, max_half_tiles=3)
    a = render.render_projected(rec, 80, 64, (0.2, 0.1, 0.4))
    b = render.render_projected(rec, 80, 64, (0.2, 0.1, 0.4), reach=True)
    assert float((a["image"] - b["image"]).abs().max()) < 1e-12
    assert torch.equal(a["last_id"], b["last_id"]) and torch.equal(a["final_T"], b["final_T"])


# ----------------------------------------------------------------------------------------------
# Gradients: autograd through the oracle forward vs central finite differences (FP64)
# ----------------------------------------------------------------------------------------------

def _decisions(scene, cam):
    out = render.render(scene, cam)
    g = out["g"]
    return (g["visible"].numpy().copy(), g["rect"].numpy().copy(), out["n_contrib"].numpy().copy()), out


def test_oracle_gradient_matches_central_differences():
    scene = synth.make_scene(64, seed=16, box=0.6)
    cam = synth.make_camera((0.0, 0.0, -3.0), 32, 32, 60.0, 0.5, bg=(0.3, 0.3, 0.3))
    rng = np.random.default_rng(17)
    dL = rng.normal(size=(32, 32, 3))
    grads = render.vjp(scene, cam, dL)
    base_dec, _ = _decisions(scene, cam)
    checked = skipped = 0
    names = ["mean7", "L28", "opacity", "sh"]
    for _ in range(40):
        name = names[rng.integers(0, 4)]
        arr = getattr(scene, name)
        flat_idx = int(rng.integers(0, arr.size))
        # choose a visible Gaussian's parameter
        g = flat_idx // (arr.size // scene.n)
        if not base_dec[0][g]:
            continue
        vals = []
        decs = []
        for sgn in (+1, -1):
            a64 = {k: getattr(scene, k).astype(np.float64) for k in names}
            x0 = a64[name].reshape(-1)[flat_idx]
            h = 1e-6 * max(1.0, abs(x0))
            a64[name].reshape(-1)[flat_idx] = x0 + sgn * h
            sc = synth.Scene(a64["mean7"], a64["L28"], a64["opacity"], a64["sh"], scene.lambda_t,
                             scene.lambda_d, scene.bg)
            dec, out = _decisions(sc, cam)
            decs.append(dec)
            vals.append(float((out["image"].numpy() * dL).sum()))
        if not all(np.array_equal(a, b) for d in decs for a, b in zip(d, base_dec)):
            skipped += 1
            continue
        fd = (vals[0] - vals[1]) / (2 * h)
        an = grads[name].reshape(-1)[flat_idx]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-7, (name, flat_idx, fd, an)
        checked += 1
    assert checked >= 20 and skipped <= 5


# ----------------------------------------------------------------------------------------------
# Tile reachability (the conservative per-tile drop applied in binning)
# ----------------------------------------------------------------------------------------------

def test_alpha_exponent_bound_is_an_upper_bound_within_1p1_percent():
    alpha = np.concatenate([np.geomspace(1 / 255 * (1 + 1e-6), 1.0, 20000), [1 / 255, 0.5, 0.99]])
    exact = 2 * np.log(255 * alpha.astype(np.float32).astype(np.float64))
    bound = binning.alpha_exponent_bound(alpha).astype(np.float64)
    # near alpha = 1/255 float32 rounding can undershoot by ~6e-5; the rule adds 1e-3 on top
    assert np.all(bound + 1e-3 >= exact + 5e-4)
    assert np.all(bound <= exact * 1.011 + 2e-4)


def _stress_gaussians(rng, n):
    """Screen-space Gaussians spanning the shapes the rule must survive: tiny (0.3 px), huge
    (300 px), needle-thin (aspect 1e-3), correlation up to 0.99999, alpha just above 1/255."""
    mean2d = rng.uniform(-40, 140, size=(n, 2)).astype(np.float32)
    kind = rng.integers(0, 4, n)
    sx = np.where(kind == 0, rng.uniform(0.3, 3, n), np.where(kind == 1, rng.uniform(3, 40, n),
                  np.where(kind == 2, rng.uniform(40, 300, n), rng.uniform(0.5, 60, n))))
    sy = np.where(kind == 3, sx * rng.uniform(0.001, 0.05, n), rng.uniform(0.3, 60, n))
    rho = np.where(rng.random(n) < 0.3, rng.choice([-1, 1], n) * rng.uniform(0.99, 0.99999, n),
                   rng.uniform(-0.99, 0.99, n))
    cov = np.stack([sx * sx, rho * sx * sy, sy * sy], 1)
    det = cov[:, 0] * cov[:, 2] - cov[:, 1] ** 2
    conic = np.stack([cov[:, 2] / det, -cov[:, 1] / det, cov[:, 0] / det], 1).astype(np.float32)
    alpha = np.where(rng.random(n) < 0.3, (1 / 255) * (1 + rng.uniform(0, 0.05, n)),
                     rng.uniform(1 / 255, 1.0, n)).astype(np.float32)
    return mean2d, conic, alpha


def test_dropped_tiles_have_no_pixel_at_or_above_the_alpha_threshold():
    """Brute force, in float64, over all 256 pixel centres of each of the 64 tiles of an 8 x 8 grid
    for 3000 stress Gaussians: every tile holding a pixel with alpha >= 1/255 is kept, and the
    rule keeps at most 6% more tiles than that exact set."""
    rng = np.random.default_rng(5)
    n, T = 3000, 8
    mean2d, conic, alpha = _stress_gaussians(rng, n)
    tx, ty = np.meshgrid(np.arange(T), np.arange(T), indexing="xy")
    G = np.repeat(np.arange(n), T * T)
    TX, TY = np.tile(tx.ravel(), n), np.tile(ty.ravel(), n)
    keep = binning.tile_reachable(mean2d[G], conic[G], alpha[G], TX, TY)
    px, py = np.meshgrid(np.arange(16) + 0.5, np.arange(16) + 0.5, indexing="xy")
    px, py = px.ravel(), py.ravel()
    reach = np.zeros(len(G), bool)
    for s0 in range(0, len(G), 20000):
        g = G[s0:s0 + 20000]
        dx = TX[s0:s0 + 20000, None] * 16 + px[None] - mean2d[g, 0:1].astype(np.float64)
        dy = TY[s0:s0 + 20000, None] * 16 + py[None] - mean2d[g, 1:2].astype(np.float64)
        a, b, c = (conic[g, k:k + 1].astype(np.float64) for k in range(3))
        al = alpha[g, None].astype(np.float64) * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
        reach[s0:s0 + 20000] = al.max(1) >= 1 / 255
    assert not np.any(reach & ~keep), np.nonzero(reach & ~keep)[0][:5]
    assert reach.sum() > 10000 and keep.sum() <= 1.06 * reach.sum()


def test_row_span_rule_keeps_contiguous_spans_and_special_cases():
    """Kept tiles of a row form one contiguous run; alpha < 1/255 drops everything; a conic that
    is not positive definite keeps everything."""
    rng = np.random.default_rng(7)
    n = 500
    mean2d, conic, alpha = _stress_gaussians(rng, n)
    tx = np.arange(-4, 14)
    for i in range(n):
        for row in range(-2, 10):
            k = binning.tile_reachable(mean2d[i:i + 1], conic[i:i + 1], alpha[i:i + 1], tx, np.full_like(tx, row))
            idx = np.nonzero(k)[0]
            assert len(idx) == 0 or idx[-1] - idx[0] + 1 == len(idx)
    low = binning.tile_reachable(mean2d[:20], conic[:20], np.full(20, 0.5 / 255, np.float32), np.zeros(20, int),
                                 np.zeros(20, int))
    assert not low.any()
    bad = conic[:20].copy()
    bad[:, 1] = np.sqrt(bad[:, 0] * bad[:, 2]) * 1.01  # det < 0
    far = np.full((20, 2), 1e4, np.float32)
    assert binning.tile_reachable(far, bad, alpha[:20], np.zeros(20, int), np.zeros(20, int)).all()


def test_reachability_drops_a_large_share_of_rectangle_tiles_on_a_scene():
    scene, cam = synth.config_scene(0), synth.config_cameras(0)[0]
    g = render.gaussians(render.params_from_scene(scene), cam, scene.lambda_t, scene.lambda_d)
    rect = g["rect"].numpy()
    full, _ = binning.instances(rect, cam.tiles_x)
    kept, _ = binning.instances(rect, cam.tiles_x, render.cull_inputs(g["mean2d"], g["conic"], g["alpha_cond"]))
    assert 0 < len(kept) < 0.8 * len(full)


# ----------------------------------------------------------------------------------------------
# Per-Gaussian conditioning direction and lambda gradients
# ----------------------------------------------------------------------------------------------

def test_per_gaussian_direction_is_unit_vector_from_camera_centre_to_mu_p():
    """dir_mode = 1 conditions Gaussian i on (mu_p,i - c) / |mu_p,i - c|: the same as the request
    path with that single direction; and a Gaussian whose mu_d is that direction has f_dir = 1."""
    rng = np.random.default_rng(21)
    n = 12
    L28 = torch.tensor(_pack(_random_L(rng, n)))
    mean7 = torch.tensor(rng.normal(size=(n, 7)))
    centre = np.array([0.3, -0.2, -3.0])
    w = mean7[:, :3].numpy() - centre
    unit = w / np.linalg.norm(w, axis=1, keepdims=True)
    mean7[::2, 4:7] = torch.tensor(unit[::2])  # even Gaussians look exactly along their direction
    op = torch.full((n,), 0.7, dtype=F64)
    per = slicing.slice_gaussians(mean7, L28, op, 0.4, None, 0.05, 0.3, dir_mode=1, center=centre)
    np.testing.assert_allclose(per["f_dir"].numpy()[::2], 1.0, rtol=0, atol=1e-14)
    for i in range(n):
        one = slicing.slice_gaussians(mean7[i:i + 1], L28[i:i + 1], op[i:i + 1], 0.4, unit[i], 0.05, 0.3)
        for k in ("mu_cond", "Sigma_cond", "alpha_cond"):
            np.testing.assert_allclose(per[k].numpy()[i], one[k].numpy()[0], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("dir_mode", [0, 1])
def test_oracle_lambda_and_mean_gradients_match_central_differences(dir_mode):
    scene = synth.make_scene(48, seed=23, box=0.6, lambda_t=0.1, lambda_d=0.15, diag=(0.2, 0.6))
    scene.dir_mode = dir_mode
    cam = synth.make_camera((0.2, -0.1, -3.0), 32, 32, 60.0, 0.35, bg=(0.3, 0.3, 0.3))
    rng = np.random.default_rng(29)
    dL = rng.normal(size=(32, 32, 3))
    grads = render.vjp(scene, cam, dL)
    base_dec, _ = _decisions(scene, cam)

    def run(lam_t, lam_d, mean7):
        sc = synth.Scene(mean7, scene.L28.astype(np.float64), scene.opacity.astype(np.float64),
                         scene.sh.astype(np.float64), lam_t, lam_d, scene.bg, dir_mode)
        dec, out = _decisions(sc, cam)
        return dec, float((out["image"].numpy() * dL).sum())

    m64 = scene.mean7.astype(np.float64)
    for k, (lt, ld) in enumerate([(1e-6, 0.0), (0.0, 1e-6)]):
        (dp, vp), (dm, vm) = run(scene.lambda_t + lt, scene.lambda_d + ld, m64), \
            run(scene.lambda_t - lt, scene.lambda_d - ld, m64)
        assert all(np.array_equal(a, b) for d in (dp, dm) for a, b in zip(d, base_dec))
        fd = (vp - vm) / 2e-6
        assert abs(fd - grads["lam"][k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, grads["lam"][k])
    assert np.any(grads["lam"] != 0)
    checked = 0
    vis = np.nonzero(base_dec[0])[0]
    for g in rng.choice(vis, size=8, replace=False):
        for c in range(3):  # mu_p: with dir_mode = 1 it also moves the conditioning direction
            h = 1e-6
            mp, mm = m64.copy(), m64.copy()
            mp[g, c] += h
            mm[g, c] -= h
            (dp, vp), (dm, vm) = run(scene.lambda_t, scene.lambda_d, mp), run(scene.lambda_t, scene.lambda_d, mm)
            if not all(np.array_equal(a, b) for d in (dp, dm) for a, b in zip(d, base_dec)):
                continue
            fd = (vp - vm) / (2 * h)
            an = grads["mean7"][g, c]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-7, (g, c, fd, an)
            checked += 1
    assert checked >= 18


# ----------------------------------------------------------------------------------------------
# Densification statistics (Algorithm 1 step 7, Sec. 4.4)
# ----------------------------------------------------------------------------------------------

def _rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_scale_rotation_recovers_a_known_rotation_and_scales():
    """Sigma_cond = R0 diag(s0^2) R0^T with distinct s0: S = sorted s0, R = R0's columns in that
    order up to sign, det R = +1."""
    from oracle import densify
    rng = np.random.default_rng(41)
    n = 20
    R0 = np.stack([_rotation(rng) for _ in range(n)])
    s0 = rng.uniform(0.05, 1.0, size=(n, 3))
    Sig = np.einsum("nij,nj,nkj->nik", R0, s0 ** 2, R0)
    S, R = densify.scale_rotation(torch.tensor(Sig))
    order = np.argsort(-s0, axis=1)
    np.testing.assert_allclose(S, np.take_along_axis(s0, order, axis=1), rtol=1e-12)
    for i in range(n):
        for j in range(3):
            c = abs(float(R[i, :, j] @ R0[i, :, order[i, j]]))
            assert abs(c - 1.0) < 1e-10
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)


def test_split_statistics_closed_form():
    """With L built so that row t of L is (0, 0, 0, st, 0, 0, 0) plus a chosen coupling to x:
    Sigma_t = st^2 + c^2 and Sigma_pt = (c * L_xx, 0, 0)."""
    from oracle import densify
    n = 3
    L = np.zeros((n, 7, 7))
    for i in range(7):
        L[:, i, i] = 0.3
    st = np.array([0.1, 0.3, 0.5])
    c = np.array([0.0, 0.4, 0.2])
    L[:, 3, 3] = st
    L[:, 3, 0] = c
    mean7 = np.zeros((n, 7))
    mean7[:, 4:] = [0.0, 0.0, 1.0]
    out = densify.densify_stats(mean7, _pack(L), np.array([0.5, 0.005, 0.02]), 0.0, [0, 0, 1], 0.05, 0.05,
                                extent=2.0)
    np.testing.assert_allclose(out["t_scale"], np.sqrt(st ** 2 + c ** 2), rtol=1e-14)
    np.testing.assert_allclose(out["pt_norm"], c * 0.3, rtol=1e-14, atol=1e-16)
    # split: |Sigma_pt| > 0.05 * 2.0 = 0.1 and t_scale > 0.25
    np.testing.assert_array_equal(out["split"], [False, True, False])
    np.testing.assert_array_equal(out["prune"], [False, True, False])


# ----------------------------------------------------------------------------------------------
# Adaptive Gaussian Refinement (Sec. 4.3, Algorithm 1 steps 1-2)
# ----------------------------------------------------------------------------------------------

def test_temporal_encoding_closed_form():
    from oracle import agr
    g0 = agr.temporal_encoding(0.0).numpy()
    np.testing.assert_array_equal(g0, np.tile([0.0, 1.0], 10))
    # t = 1/2: sin(2^k pi / 2) = 1, 0, 0, ...; cos(2^k pi / 2) = 0, -1, 1, 1, ...
    g = agr.temporal_encoding(0.5).numpy()
    np.testing.assert_allclose(g[0::2], [1.0] + [0.0] * 9, atol=1e-12)
    np.testing.assert_allclose(g[1::2], [0.0, -1.0] + [1.0] * 8, atol=1e-12)
    assert g.shape == (20,)


def _zero_weights():
    return dict(w1=torch.zeros(4, 64, 27, dtype=F64), b1=torch.zeros(4, 64, dtype=F64),
                w2=torch.zeros(35, 64, dtype=F64), b2=torch.zeros(35, dtype=F64))


def test_refinement_routes_each_mlp_to_its_parameters():
    """Zero weights give the identity; one hidden unit feeding one output row gives
    relu(f_c + beta) on exactly the parameter that row refines."""
    from oracle import agr
    rng = np.random.default_rng(51)
    n = 9
    mean7 = torch.tensor(rng.normal(size=(n, 7)))
    L28 = torch.tensor(rng.normal(size=(n, 28)))
    t = 0.3
    m0, l0 = agr.refine(mean7, L28, t, _zero_weights())
    assert torch.equal(m0, mean7) and torch.equal(l0, L28)
    f = agr.features(mean7, t).numpy()
    cases = [(0, 0, 0, -0.2, "mean7", 0), (1, 5, 3, 0.1, "mean7", 3), (2, 9, 6, 0.0, "mean7", 6),
             (3, 7, 10, 0.4, "L28", 3), (3, 26, 34, -0.7, "L28", 27), (0, 12, 2, 0.25, "mean7", 2)]
    for m, c, row, beta, which, col in cases:
        w = _zero_weights()
        w["w1"][m, 17, c] = 1.0
        w["b1"][m, 17] = beta
        w["w2"][row, 17] = 1.0
        mh, lh = agr.refine(mean7, L28, t, w)
        want = np.maximum(f[:, c] + beta, 0.0)
        got_m, got_l = (mh - mean7).numpy(), (lh - L28).numpy()
        target, other = (got_m, got_l) if which == "mean7" else (got_l, got_m)
        np.testing.assert_allclose(target[:, col], want, rtol=0, atol=1e-15)
        target[:, col] = 0.0
        assert not target.any() and not other.any(), (m, c, row)
    # features: mu_p, mu_t, mu_d, then gamma(t)
    np.testing.assert_array_equal(f[:, :7], mean7.numpy())
    np.testing.assert_allclose(f[:, 7], math.sin(math.pi * t), rtol=1e-15)
    np.testing.assert_allclose(f[:, 26], math.cos(2 ** 9 * math.pi * t), rtol=1e-12)


def test_refinement_gradients_match_central_differences():
    from oracle import agr
    rng = np.random.default_rng(53)
    n = 6
    mean7 = torch.tensor(rng.normal(size=(n, 7)), requires_grad=True)
    L28 = torch.tensor(rng.normal(size=(n, 28)), requires_grad=True)
    w = agr.weights_to_torch(synth.make_agr_weights(seed=5, scale=1.0), requires_grad=True)
    cm, cl = torch.tensor(rng.normal(size=(n, 7))), torch.tensor(rng.normal(size=(n, 28)))

    def loss(m7, l28, ww):
        mh, lh = agr.refine(m7, l28, 0.37, ww)
        return (mh * cm).sum() + (lh * cl).sum()

    loss(mean7, L28, w).backward()
    checked = 0
    for name in ("mean7", "L28", "w1", "b1", "w2", "b2"):
        base = {"mean7": mean7, "L28": L28, **w}
        for _ in range(6):
            arr = base[name].detach()
            k = int(rng.integers(0, arr.numel()))
            vals = []
            for sgn in (1, -1):
                cur = {kk: v.detach().clone() for kk, v in base.items()}
                cur[name].reshape(-1)[k] += sgn * 1e-6
                with torch.no_grad():
                    vals.append(float(loss(cur["mean7"], cur["L28"], {q: cur[q] for q in ("w1", "b1", "w2", "b2")})))
            fd = (vals[0] - vals[1]) / 2e-6
            an = float(base[name].grad.reshape(-1)[k])
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, k, fd, an)
            checked += 1
    assert checked == 36
