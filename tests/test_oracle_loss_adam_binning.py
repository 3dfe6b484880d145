"""Pins of the oracle's loss (Eq. 5), Adam, binning definition (Eq. 1, the
per-column test) and the end-to-end chain of gradients."""
import math
from pathlib import Path

import numpy as np
import pytest
import torch

import synth
from oracle import adam, binning, loss, preprocess, render, step


# --------------------------------------------------------------------- loss

def _ssim_bruteforce(x, y):
    """SSIM by explicit loops over pixels and the 11 x 11 window (zero padding)."""
    g1 = np.exp(-((np.arange(11) - 5.0) ** 2) / (2 * 1.5 ** 2))
    g1 /= g1.sum()
    w = np.outer(g1, g1)
    C, H, W = x.shape
    tot = 0.0
    for c in range(C):
        for j in range(H):
            for i in range(W):
                mx = my = sxx = syy = sxy = 0.0
                for v in range(11):
                    for u in range(11):
                        jj, ii = j + v - 5, i + u - 5
                        if 0 <= jj < H and 0 <= ii < W:
                            a, b = x[c, jj, ii], y[c, jj, ii]
                            mx += w[v, u] * a
                            my += w[v, u] * b
                            sxx += w[v, u] * a * a
                            syy += w[v, u] * b * b
                            sxy += w[v, u] * a * b
                sxx -= mx * mx
                syy -= my * my
                sxy -= mx * my
                c1, c2 = 0.01 ** 2, 0.03 ** 2
                tot += ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return tot / (C * H * W)


def test_ssim_matches_bruteforce_loops():
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(2, 7, 9))
    y = rng.uniform(size=(2, 7, 9))
    got = float(loss.ssim(torch.as_tensor(x), torch.as_tensor(y)))
    np.testing.assert_allclose(got, _ssim_bruteforce(x, y), rtol=1e-12)


def test_ssim_of_identical_images_is_one_with_zero_gradient():
    x = synth.target_uniform(3, 20, 14).astype(np.float64)
    L, g = loss.photometric(x, x, lam=1.0)
    assert abs(L) < 1e-12
    assert np.abs(g).max() < 1e-12


def test_photometric_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(3, 6, 8))
    y = x + rng.choice([-0.3, 0.3], size=x.shape)  # keep |x - y| away from the L1 kink
    _, g = loss.photometric(x, y, lam=0.2)
    fd = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        h = 1e-6
        xp = x.copy()
        xm = x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd[idx] = (loss.photometric(xp, y, 0.2)[0] - loss.photometric(xm, y, 0.2)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_l1_closed_form():
    x = np.array([[[0.2, 0.9]]])
    y = np.array([[[0.5, 0.4]]])
    L, g = loss.photometric(x, y, lam=0.0)
    assert abs(L - 0.4) < 1e-15
    np.testing.assert_allclose(g, [[[-0.5, 0.5]]])


def test_window_is_normalised_gaussian():
    w = loss.gaussian_window().numpy()
    np.testing.assert_allclose(w.sum(), 1.0, rtol=1e-14)
    np.testing.assert_allclose(w[5, 5] / w[5, 6], math.exp(1 / (2 * 1.5 ** 2)), rtol=1e-12)


# --------------------------------------------------------------------- adam

def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = adam.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # m_hat = g, v_hat = g^2  ->  update = lr * g / (|g| + eps)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-9)


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(2)
    p0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(4)]
    pt = torch.nn.Parameter(torch.as_tensor(p0.copy()))
    opt = torch.optim.Adam([pt], lr=3e-3, betas=(0.9, 0.999), eps=1e-15)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for k, g in enumerate(grads, start=1):
        pt.grad = torch.as_tensor(g)
        opt.step()
        p, m, v = adam.adam_step(p, g, m, v, k, lr=3e-3)
    np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_visible_adam_matches_torch_sparse_adam():
    """torch.optim.SparseAdam updates only the rows present in a sparse
    gradient, with the global step count: the same rule, up to where eps
    enters the denominator (negligible at eps = 1e-30, where both coincide)."""
    rng = np.random.default_rng(4)
    n, d = 40, 3
    p0 = rng.standard_normal((n, d))
    pt = torch.nn.Parameter(torch.as_tensor(p0.copy()))
    opt = torch.optim.SparseAdam([pt], lr=2e-3, betas=(0.9, 0.999), eps=1e-30)
    p, m, v = p0.copy(), np.zeros((n, d)), np.zeros((n, d))
    for k in range(1, 6):
        vis = rng.uniform(size=n) < 0.6
        g = rng.standard_normal((n, d)) * vis[:, None]
        rows = np.nonzero(vis)[0]
        pt.grad = torch.sparse_coo_tensor(torch.as_tensor(rows[None]), torch.as_tensor(g[rows]), (n, d))
        opt.step()
        p, m, v = adam.adam_step_visible(p, g, m, v, k, lr=2e-3, visible=vis, eps=1e-30)
    np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_visible_adam_special_cases():
    rng = np.random.default_rng(5)
    p0, g = rng.standard_normal((9, 4)), rng.standard_normal((9, 4))
    m0, v0 = rng.standard_normal((9, 4)), rng.uniform(0.1, 1.0, (9, 4))
    everyone = adam.adam_step_visible(p0, g, m0, v0, 3, 1e-2, np.ones(9, bool))
    for a, b in zip(everyone, adam.adam_step(p0, g, m0, v0, 3, 1e-2)):
        np.testing.assert_array_equal(a, b)
    nobody = adam.adam_step_visible(p0, g, m0, v0, 3, 1e-2, np.zeros(9, bool))
    for a, b in zip(nobody, (p0, m0, v0)):
        np.testing.assert_array_equal(a, b)


# ------------------------------------------------------------------ binning

def test_min_q_over_rectangle_matches_dense_sampling():
    rng = np.random.default_rng(3)
    for _ in range(200):
        L = rng.standard_normal((2, 2))
        A = L @ L.T + 0.05 * np.eye(2)
        a, b, c = A[0, 0], A[0, 1], A[1, 1]
        mx, my = rng.uniform(-20, 20, 2)
        x0, y0 = rng.uniform(-20, 20, 2)
        x1, y1 = x0 + rng.uniform(0, 15), y0 + rng.uniform(0, 15)
        got = binning.min_q_rect(mx, my, a, b, c, x0, x1, y0, y1)
        xs, ys = np.meshgrid(np.linspace(x0, x1, 301), np.linspace(y0, y1, 301))
        dx, dy = xs - mx, ys - my
        dense = (a * dx * dx + 2 * b * dx * dy + c * dy * dy).min()
        assert got <= dense + 1e-12
        assert dense - got <= 1e-3 * max(1.0, dense) + 0.01 * (a + abs(b) + c)


def test_level_set_extent_is_the_corrected_eq2():
    # Eq. 2 prints b^2 - ac under the root; for a positive-definite conic the
    # tangent points are x_d = +-sqrt(b^2 t / (a (ac - b^2))) and the y-extent
    # is sqrt(t a / (ac - b^2)) = sqrt(t Syy).  Check against the ellipse.
    rng = np.random.default_rng(4)
    for _ in range(50):
        L = rng.standard_normal((2, 2))
        A = L @ L.T + 0.1 * np.eye(2)
        a, b, c = A[0, 0], A[0, 1], A[1, 1]
        t = rng.uniform(0.5, 11)
        th = np.linspace(0, 2 * np.pi, 200001)
        # boundary points: q(x, y) = t
        Lc = np.linalg.cholesky(np.linalg.inv(A))
        pts = math.sqrt(t) * (Lc @ np.stack([np.cos(th), np.sin(th)]))
        ymax = pts[1].max()
        xd_at_ymax = pts[0, pts[1].argmax()]
        np.testing.assert_allclose(ymax, math.sqrt(t * a / (a * c - b * b)), rtol=1e-6)
        np.testing.assert_allclose(abs(xd_at_ymax), math.sqrt(b * b * t / (a * (a * c - b * b))),
                                   rtol=1e-3, atol=1e-3)
        np.testing.assert_allclose(pts[0].max(), math.sqrt(t * c / (a * c - b * b)), rtol=1e-6)


def test_tile_min_q_on_config1_covers_every_blended_pixel():
    sc = synth.scene_c1(1)
    cam = synth.camera_c1()
    pr = preprocess.project(preprocess.params_from_scene(sc), cam, 0)
    r = preprocess.pack_for_render(pr)
    tiles = binning.tile_min_q(r, 256, 256)
    for gid in range(0, sc.n, 97):
        if gid not in tiles:
            continue
        ids, mq, t = tiles[gid]
        touched = set(ids[mq <= t].tolist())
        single = r.copy()
        single[np.arange(sc.n) != gid, 11] = 0.0
        f = render.render_fwd(single, (0, 0, 0), (0, 0, 256, 256), amb=None)
        ys, xs = np.nonzero(f["count"])
        blended_tiles = set((ys // 16 * 16 + xs // 16).tolist())
        assert blended_tiles <= touched


GOLDEN = Path(__file__).parent / "golden"


def _golden_snugbox_cases():
    cases = []
    for line in (GOLDEN / "snugbox_tiles.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        lhs, rhs = line.split(":")
        w, h, mx, my, a, b, c, t = (float(x) for x in lhs.split())
        want = set() if rhs.strip() == "-" else {int(x) for x in rhs.split()}
        cases.append((int(w), int(h), mx, my, a, b, c, t, want))
    return cases


def test_golden_snugbox_tiles_worked_by_hand():
    """Sec. 2.1, Eq. 1-2: the tile sets of tests/golden/snugbox_tiles.txt,
    derived by hand there, from the oracle's tile test and from dense sampling
    of every tile rectangle (which shares nothing with the oracle's
    edge-minimum search)."""
    cases = _golden_snugbox_cases()
    assert len(cases) == 4
    for w, h, mx, my, a, b, c, t, want in cases:
        rec = np.zeros((1, 12))
        rec[0, 0:5] = (mx, my, a, b, c)
        rec[0, 5] = math.exp(t / 2.0) / 255.0  # Eq. 1 solved for o
        rec[0, 10] = t
        rec[0, 11] = 1.0
        tiles = binning.tile_min_q(rec, w, h)
        got = set()
        if 0 in tiles:
            ids, mq, tt = tiles[0]
            got = set(ids[mq <= tt].tolist())
        assert got == want, (w, h, mx, my, got, want)
        # dense sampling of each tile's pixel-centre rectangle
        tw, th = -(-w // 16), -(-h // 16)
        dense = set()
        for ty in range(th):
            for tx in range(tw):
                xs = np.linspace(tx * 16 + 0.5, min(tx * 16 + 15, w - 1) + 0.5, 241)
                ys = np.linspace(ty * 16 + 0.5, min(ty * 16 + 15, h - 1) + 0.5, 241)
                dx, dy = np.meshgrid(xs - mx, ys - my)
                if t > 0 and (a * dx * dx + 2 * b * dx * dy + c * dy * dy).min() <= t:
                    dense.add(ty * tw + tx)
        assert dense == want, (w, h, mx, my, dense, want)


def test_stable_sort_definition():
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 50, size=1000).astype(np.uint32)
    vals = np.arange(1000, dtype=np.uint32)
    k, v = binning.stable_sort_pairs(keys, vals)
    want = sorted(zip(keys.tolist(), vals.tolist()))
    assert list(zip(k.tolist(), v.tolist())) == want


# -------------------------------------------------------- end to end chain

def test_full_step_gradient_matches_finite_differences():
    """Loss(preprocess -> blend -> SSIM/L1) vs the chained oracle backward."""
    cam = synth.camera_tiny(16, 16)
    sc = synth.scene_tiny(4, seed=32, sh_degree=1)
    sc64 = synth.Scene(*(a.astype(np.float64) for a in sc.arrays()), sh_degree=1)
    # target far from the image keeps L1 on one side of its kink
    target = np.full((3, 16, 16), 2.0)
    bg = (0.1, 0.2, 0.3)

    def L(scene):
        return step.forward_backward(scene, cam, target, bg=bg, lam=0.2)[0]

    _, grads, f = step.forward_backward(sc64, cam, target, bg=bg, lam=0.2)
    amb = render.render_fwd(preprocess.pack_for_render(preprocess.project(
        preprocess.params_from_scene(sc64), cam, 1)), bg, (0, 0, 16, 16), amb=(1e-3, 1e-3, 1e-3, 1e-6))["amb"]
    assert not amb.any(), "choose a seed whose pixels are away from the thresholds"
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        arr = getattr(sc64, name)
        for idx in np.ndindex(arr.shape):
            h = 1e-6
            old = arr[idx]
            arr[idx] = old + h
            fp = L(sc64)
            arr[idx] = old - h
            fm = L(sc64)
            arr[idx] = old
            fd = (fp - fm) / (2 * h)
            assert abs(grads[name][idx] - fd) <= 2e-5 * max(1e-3, abs(fd)), (name, idx, grads[name][idx], fd)


def test_batch_loss_is_pixel_weighted_and_matches_finite_differences():
    """A batch of views of unequal size: the batch gradient is the gradient
    of the pooled per-pixel mean, and two copies of one view give exactly
    that view's loss and gradient."""
    sc = synth.scene_tiny(4, seed=32, sh_degree=1)
    sc64 = synth.Scene(*(a.astype(np.float64) for a in sc.arrays()), sh_degree=1)
    cams = [synth.camera_tiny(16, 16), synth.camera_tiny(24, 12)]
    rng = np.random.default_rng(3)
    targets = [rng.uniform(1.5, 2.0, size=(3, c.height, c.width)) for c in cams]
    dts = [rng.uniform(0.0, 0.05, size=(c.height, c.width)) for c in cams]
    kw = dict(bg=(0.1, 0.2, 0.3), lam=0.2, disp_targets=dts, disp_weight=0.1)
    L, g = step.forward_backward_batch(sc64, cams, targets, **kw)
    for c in cams:
        amb = render.render_fwd(preprocess.pack_for_render(preprocess.project(
            preprocess.params_from_scene(sc64), c, 1)), kw["bg"], (0, 0, c.width, c.height),
            amb=(1e-3, 1e-3, 1e-3, 1e-6))["amb"]
        assert not amb.any()
    for name, idx in (("means", (1, 0)), ("log_scales", (2, 1)), ("opacity_logits", (3,)), ("sh", (0, 1, 2))):
        arr = getattr(sc64, name)
        h = 1e-6
        old = arr[idx]
        arr[idx] = old + h
        fp = step.forward_backward_batch(sc64, cams, targets, **kw)[0]
        arr[idx] = old - h
        fm = step.forward_backward_batch(sc64, cams, targets, **kw)[0]
        arr[idx] = old
        fd = (fp - fm) / (2 * h)
        assert abs(g[name][idx] - fd) <= 2e-5 * max(1e-3, abs(fd)), (name, idx, g[name][idx], fd)
    # the pooled mean differs from the plain mean of the two views' losses
    L0 = step.forward_backward(sc64, cams[0], targets[0], bg=kw["bg"], lam=0.2, disp_target=dts[0],
                               disp_weight=0.1)
    L1 = step.forward_backward(sc64, cams[1], targets[1], bg=kw["bg"], lam=0.2, disp_target=dts[1],
                               disp_weight=0.1)
    assert abs(L - (256 * L0[0] + 288 * L1[0]) / 544) < 1e-12
    L2, g2 = step.forward_backward_batch(sc64, [cams[0], cams[0]], [targets[0]] * 2, bg=kw["bg"], lam=0.2,
                                         disp_targets=[dts[0]] * 2, disp_weight=0.1)
    assert abs(L2 - L0[0]) < 1e-12
    for k in g2:
        np.testing.assert_allclose(g2[k], L0[1][k], rtol=1e-12, atol=1e-15)
