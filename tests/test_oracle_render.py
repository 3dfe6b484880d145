"""Pins of the oracle's per-pixel blend and backward (Sec. 2.1 renderCUDA,
Sec. 2.2): closed forms, invariants, threshold cases, finite differences and
an independent autograd evaluation of the same definition."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import preprocess, render

BLACK = (0.0, 0.0, 0.0)


def rec(mx, my, a, b, c, o, rgb, z, valid=1.0):
    t = 2.0 * math.log(255.0 * o) if o > 0 else -1.0
    return [mx, my, a, b, c, o, rgb[0], rgb[1], rgb[2], z, t, valid]


def records(rows):
    return np.array(rows, dtype=np.float64)


def test_single_gaussian_pixels_match_closed_form():
    var = 9.0
    o = 0.8
    bg = (0.1, 0.2, 0.3)
    rgb = (0.9, 0.4, 0.2)
    r = records([rec(16.2, 15.7, 1 / var, 0.0, 1 / var, o, rgb, 2.5)])
    f = render.render_fwd(r, bg, (0, 0, 32, 32))
    i, j = np.meshgrid(np.arange(32) + 0.5, np.arange(32) + 0.5)
    q = ((i - 16.2) ** 2 + (j - 15.7) ** 2) / var
    a = np.minimum(0.99, o * np.exp(-0.5 * q))
    a = np.where(a < 1 / 255, 0.0, a)
    for ch in range(3):
        np.testing.assert_allclose(f["rgb"][ch], rgb[ch] * a + (1 - a) * bg[ch], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(f["T"], 1 - a, rtol=1e-13)
    np.testing.assert_allclose(f["disp"], a / 2.5, rtol=1e-13, atol=1e-16)
    # the level set of Eq. 1 is where alpha reaches 1/255: radius sqrt(t * var)
    radius = math.sqrt(2 * math.log(255 * o) * var)
    d = np.sqrt((i - 16.2) ** 2 + (j - 15.7) ** 2)
    assert np.all(f["count"][d < radius - 1e-9] == 1)
    assert np.all(f["count"][d > radius + 1e-9] == 0)


def test_three_gaussian_compositing_closed_form_and_depth_order():
    # co-centred Gaussians, listed out of depth order on purpose
    o = [0.6, 0.5, 0.7]
    z = [3.0, 1.5, 2.0]
    col = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    var = [4.0, 9.0, 16.0]
    r = records([rec(8.5, 8.5, 1 / v, 0, 1 / v, oo, cc, zz) for oo, cc, zz, v in zip(o, col, z, var)])
    bg = (0.2, 0.2, 0.2)
    f = render.render_fwd(r, bg, (0, 0, 17, 17))
    # pixel (9, 8): centre (9.5, 8.5), r^2 = 1
    al = [oo * math.exp(-0.5 / v) for oo, v in zip(o, var)]
    order = np.argsort(z)
    T = 1.0
    C = np.zeros(3)
    D = 0.0
    for k in order:
        C += np.array(col[k]) * al[k] * T
        D += al[k] * T / z[k]
        T *= 1 - al[k]
    C += T * np.array(bg)
    np.testing.assert_allclose(f["rgb"][:, 8, 9], C, rtol=1e-13)
    np.testing.assert_allclose(f["T"][8, 9], T, rtol=1e-13)
    np.testing.assert_allclose(f["disp"][8, 9], D, rtol=1e-13)


def test_transmittance_stop_blends_exactly_three_of_four():
    # four splats with alpha = 0.95 at the pixel centre: T = 0.05, 0.0025,
    # 1.25e-4; the 4th would give 6.25e-6 < 1e-4 and is not blended
    rows = [rec(4.5, 4.5, 1.0, 0.0, 1.0, 0.95, (0.1 * (k + 1), 0.0, 1.0), 1.0 + k) for k in range(4)]
    f = render.render_fwd(records(rows), BLACK, (0, 0, 9, 9))
    assert f["count"][4, 4] == 3
    np.testing.assert_allclose(f["T"][4, 4], 0.05 ** 3, rtol=1e-12)
    want_r = 0.95 * (0.1 + 0.2 * 0.05 + 0.3 * 0.0025)
    np.testing.assert_allclose(f["rgb"][0, 4, 4], want_r, rtol=1e-12)
    np.testing.assert_allclose(f["rgb"][2, 4, 4], 1 - 0.05 ** 3, rtol=1e-12)


def test_golden_one_pixel_blend_worked_by_hand():
    """tests/golden/blend_one_pixel.txt: five splats on one pixel, given out of
    depth order, exercising the sort by depth, the 1/255 skip, the 0.99
    clamp, the transmittance stop without blending, the background and the
    disparity channel; the expected values are derived by hand in the file."""
    from pathlib import Path

    rows, want = [], {}
    for line in (Path(__file__).parent / "golden" / "blend_one_pixel.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "splat":
            z, o, r, g, b = (float(v) for v in vals)
            rows.append(rec(0.5, 0.5, 1.0, 0.0, 1.0, o, (r, g, b), z))
        else:
            want[key] = [float(v) for v in vals]
    assert len(rows) == 5
    f = render.render_fwd(records(rows), tuple(want["bg"]), (0, 0, 1, 1))
    np.testing.assert_allclose(f["rgb"][:, 0, 0], want["rgb"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(f["disp"][0, 0], want["disp"][0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(f["T"][0, 0], want["T"][0], rtol=0, atol=1e-15)
    assert f["count"][0, 0] == int(want["blended"][0])
    assert f["last"][0, 0] == int(want["last"][0])


def test_alpha_cutoff_either_side_of_one_over_255():
    o = 0.5
    for sign, blended in ((+1, 1), (-1, 0)):
        target = (1.0 / 255.0) * (1 + sign * 1e-3)
        d = math.sqrt(2 * math.log(o / target))
        r = records([rec(10.5 + d, 10.5, 1.0, 0.0, 1.0, o, (1, 1, 1), 2.0)])
        f = render.render_fwd(r, BLACK, (10, 10, 11, 11))
        assert f["count"][0, 0] == blended
        np.testing.assert_allclose(f["rgb"][0, 0, 0], blended * target, rtol=1e-9)


def test_alpha_clamp_at_099():
    r = records([rec(3.5, 3.5, 1.0, 0.0, 1.0, 0.999, (1, 1, 1), 2.0)])
    f = render.render_fwd(r, BLACK, (3, 3, 4, 4))
    np.testing.assert_allclose(f["T"][0, 0], 0.01, rtol=1e-12)


def _c1_records(seed=0, rgb_one=False, same_z=None):
    sc = synth.scene_c1(seed)
    pr = preprocess.project(preprocess.params_from_scene(sc), synth.camera_c1(), 0)
    r = preprocess.pack_for_render(pr)
    if rgb_one:
        r[:, 6:9] = 1.0
    if same_z is not None:
        r[:, 9] = same_z
    return r


def test_invariants_on_config1_scene():
    r = _c1_records(rgb_one=True, same_z=3.0)
    f = render.render_fwd(r, BLACK, (0, 0, 256, 256), amb=None)
    # telescoping: sum_i alpha_i T_i + T_final = 1
    np.testing.assert_allclose(f["rgb"][0], 1.0 - f["T"], atol=1e-12)
    # all at one depth z: blended disparity = (1 - T_final) / z
    np.testing.assert_allclose(f["disp"], (1.0 - f["T"]) / 3.0, atol=1e-12)
    # every blended splat kept T >= 1e-4, so the final T does too
    assert f["T"].min() >= 1e-4
    assert f["count"].max() > 20  # the stop actually triggered somewhere
    # colours lie within [0, max rgb] on a black background
    r2 = _c1_records()
    f2 = render.render_fwd(r2, BLACK, (0, 0, 256, 256), amb=None)
    assert f2["rgb"].min() >= 0 and f2["rgb"].max() <= r2[:, 6:9].max() + 1e-12


def test_transmittance_never_increases_with_more_splats():
    r = _c1_records()
    order = np.argsort(r[:, 9], kind="stable")
    prev = None
    for k in (0, 512, 1024, 2048, 4096):
        sub = r.copy()
        sub[order[k:], 11] = 0.0  # only the k nearest Gaussians exist
        T = render.render_fwd(sub, BLACK, (0, 0, 256, 256), amb=None)["T"]
        if prev is not None:
            assert np.all(T <= prev + 1e-15)
        prev = T


def _tiny_records(seed, n=6):
    sc = synth.scene_tiny(n, seed=seed, sh_degree=1)
    pr = preprocess.project(preprocess.params_from_scene(sc), synth.camera_tiny(), 1)
    return preprocess.pack_for_render(pr)


def _objective(r, g, gd, bg, win):
    f = render.render_fwd(r, bg, win, amb=None)
    return float((f["rgb"] * g).sum() + (f["disp"] * gd).sum())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_render_backward_matches_finite_differences(seed):
    r = _tiny_records(seed)
    win = (0, 0, 16, 16)
    bg = (0.3, 0.1, 0.6)
    g, gd = synth.upstream_grads(seed + 100, 16, 16)
    g = g.astype(np.float64)
    gd = gd.astype(np.float64)
    # drop pixels where a threshold is within reach of the FD step
    amb = render.render_fwd(r, bg, win, amb=(1e-4, 1e-4, 1e-4, 1e-6))["amb"]
    g[:, amb] = 0.0
    gd[amb] = 0.0
    got = render.render_bwd(r, bg, win, g, gd)
    cols = {0: 0, 1: 1, 2: 2, 3: 3, 4: 4, 5: 5, 6: 6, 7: 7, 8: 8}
    for i in range(r.shape[0]):
        for col, out in cols.items():
            h = 1e-7 * max(1.0, abs(r[i, col]))
            rp = r.copy()
            rm = r.copy()
            rp[i, col] += h
            rm[i, col] -= h
            if col == 5:  # the level set moves with o; keep the record consistent
                rp[i, 10] = 2 * math.log(255 * rp[i, 5])
                rm[i, 10] = 2 * math.log(255 * rm[i, 5])
            fd = (_objective(rp, g, gd, bg, win) - _objective(rm, g, gd, bg, win)) / (2 * h)
            assert abs(got[i, out] - fd) <= 1e-5 * max(1.0, abs(fd)), (i, col, got[i, out], fd)
        # depth enters through the disparity weight 1/z only
        h = 1e-7 * r[i, 9]
        rp = r.copy()
        rm = r.copy()
        rp[i, 9] += h
        rm[i, 9] -= h
        fd = (_objective(rp, g, gd, bg, win) - _objective(rm, g, gd, bg, win)) / (2 * h)
        want = got[i, 9] * (-1.0 / r[i, 9] ** 2)
        assert abs(want - fd) <= 1e-5 * max(1.0, abs(fd)), (i, "z", want, fd)


def _torch_blend(r, bg, w, h):
    """The same per-pixel definition evaluated with torch autograd (tiny sizes)."""
    rt = torch.as_tensor(r[:, :10], dtype=torch.float64).requires_grad_(True)
    outs = []
    order = sorted(range(r.shape[0]), key=lambda k: (r[k, 9], k))
    for j in range(h):
        for i in range(w):
            px, py = i + 0.5, j + 0.5
            T = torch.ones((), dtype=torch.float64)
            C = torch.zeros(3, dtype=torch.float64)
            D = torch.zeros((), dtype=torch.float64)
            for k in order:
                if r[k, 11] == 0 or not r[k, 10] > 0:
                    continue
                mx, my, a, b, c, o = rt[k, 0], rt[k, 1], rt[k, 2], rt[k, 3], rt[k, 4], rt[k, 5]
                dx, dy = px - mx, py - my
                power = -0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy)
                if power.item() > 0:
                    continue
                al = torch.clamp(o * torch.exp(power), max=0.99)
                if al.item() < 1 / 255:
                    continue
                tt = T * (1 - al)
                if tt.item() < 1e-4:
                    break
                C = C + rt[k, 6:9] * al * T
                D = D + al * T / rt[k, 9]
                T = tt
            outs.append(torch.cat([C + T * torch.as_tensor(bg, dtype=torch.float64), D[None]]))
    return rt, torch.stack(outs).reshape(h, w, 4)


def test_render_backward_matches_autograd_of_the_definition():
    r = _tiny_records(4, n=5)
    bg = (0.2, 0.5, 0.1)
    g, gd = synth.upstream_grads(9, 16, 16)
    rt, out = _torch_blend(r, bg, 16, 16)
    gt = torch.as_tensor(np.concatenate([np.moveaxis(g, 0, -1), gd[..., None]], -1), dtype=torch.float64)
    (out * gt).sum().backward()
    ag = rt.grad.numpy()
    got = render.render_bwd(r, bg, (0, 0, 16, 16), g.astype(np.float64), gd.astype(np.float64))
    np.testing.assert_allclose(got[:, 0:9], ag[:, 0:9], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(got[:, 9] * (-1.0 / r[:, 9] ** 2), ag[:, 9], rtol=1e-10, atol=1e-12)
    # and the forward agrees with the oracle's
    f = render.render_fwd(r, bg, (0, 0, 16, 16), amb=None)
    np.testing.assert_allclose(np.moveaxis(out.detach().numpy()[..., :3], -1, 0), f["rgb"], atol=1e-14)


def test_windowed_render_equals_crop_of_full_render():
    r = _c1_records(seed=2)
    full = render.render_fwd(r, BLACK, (0, 0, 256, 256), amb=None)
    part = render.render_fwd(r, BLACK, (40, 72, 105, 130), amb=None)
    np.testing.assert_array_equal(part["rgb"], full["rgb"][:, 72:130, 40:105])
    np.testing.assert_array_equal(part["count"], full["count"][72:130, 40:105])


def test_threads_do_not_change_results():
    r = _c1_records(seed=3)
    g, gd = synth.upstream_grads(5, 256, 256)
    a = render.render_bwd(r, BLACK, (0, 0, 256, 256), g, gd, n_threads=1)
    b = render.render_bwd(r, BLACK, (0, 0, 256, 256), g, gd, n_threads=4)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# Where float32 may decide a branch: flags, alternatives and slack.

F32 = render.float32_bands()


def _stack_rows(alphas, z0=1.0):
    """Splats centred on pixel (0, 0) with the given alphas (power = 0), at
    increasing depths, colours distinct per splat."""
    return [rec(0.5, 0.5, 1.0, 0.0, 1.0, a, (0.1 * (k + 1), 1.0 - 0.1 * k, 0.5), z0 + k) for k, a in enumerate(alphas)]


def _blend_by_hand(alphas, bg, rows):
    T, C, D = 1.0, np.zeros(3), 0.0
    for a, r in zip(alphas, rows):
        C += np.array(r[6:9]) * a * T
        D += a * T / r[9]
        T *= 1.0 - a
    return C + T * np.array(bg), D, T


def test_alternatives_at_the_cut_the_clamp_and_the_stop():
    """A splat whose alpha sits just above 1/255, one just above the 0.99
    clamp, and a stop whose T (1 - alpha) lies just above 1e-4: each decision
    is flagged, and each alternative (the decision taken the other way) is the
    hand-computed blend of that branch."""
    bg = (0.2, 0.3, 0.4)
    # the cut: alpha = (1/255)(1 + 1e-9)
    a_cut = (1 / 255) * (1 + 1e-9)
    rows = _stack_rows([0.3, a_cut, 0.5])
    f = render.render_fwd(records(rows), bg, (0, 0, 1, 1), amb=F32)
    assert f["flags"][0, 0] & render.F_CUT
    C, D, T = _blend_by_hand([0.3, a_cut, 0.5], bg, rows)
    np.testing.assert_allclose(f["rgb"][:, 0, 0], C, rtol=1e-13)
    assert len(f["alts"]["pix"]) == 1
    C2, D2, T2 = _blend_by_hand([0.3, 0.5], bg, [rows[0], rows[2]])
    np.testing.assert_allclose(f["alts"]["val"][0], [*C2, D2, T2], rtol=1e-13)
    assert f["alts"]["last"][0] == 2
    # the clamp: o = 0.99 (1 + 1e-9) blends 0.99 (no gradient); the
    # alternative blends o itself
    o = 0.99 * (1 + 1e-9)
    rows = _stack_rows([0.4, o])
    f = render.render_fwd(records(rows), bg, (0, 0, 1, 1), amb=F32)
    assert f["flags"][0, 0] & render.F_CLAMP
    C, D, T = _blend_by_hand([0.4, 0.99], bg, rows)
    np.testing.assert_allclose(f["T"][0, 0], T, rtol=1e-13)
    C2, D2, T2 = _blend_by_hand([0.4, o], bg, rows)
    np.testing.assert_allclose(f["alts"]["val"][0], [*C2, D2, T2], rtol=1e-12)
    # the stop: after three splats of alpha 0.9 (T = 1e-3), a fourth with
    # T (1 - alpha) = 1e-4 (1 + 1e-9) is blended; the alternative stops
    # there (three splats blended, last id 2)
    a4 = 1.0 - 0.1 * (1 + 1e-9)
    rows = _stack_rows([0.9, 0.9, 0.9, a4, 0.3])
    f = render.render_fwd(records(rows), bg, (0, 0, 1, 1), amb=F32)
    assert f["flags"][0, 0] & render.F_STOP
    assert f["count"][0, 0] == 4 and f["last"][0, 0] == 3  # the fifth would stop
    C2, D2, T2 = _blend_by_hand([0.9, 0.9, 0.9], bg, rows[:3])
    alt = [k for k in range(len(f["alts"]["pix"])) if f["alts"]["last"][k] == 2]
    assert len(alt) == 1
    np.testing.assert_allclose(f["alts"]["val"][alt[0]], [*C2, D2, T2], rtol=1e-12)
    # far from every threshold: nothing flagged, no alternative
    rows = _stack_rows([0.3, 0.2, 0.5])
    f = render.render_fwd(records(rows), bg, (0, 0, 1, 1), amb=F32)
    assert f["flags"][0, 0] == 0 and len(f["alts"]["pix"]) == 0


def test_slack_is_the_change_of_each_gaussians_gradient_under_the_other_branch():
    """At a flagged cut, the slack of every Gaussian is the largest change of
    its 2D gradient between the two branches, which equals the difference of
    the oracle's own backward on records nudged to either side of the cut."""
    bg = (0.2, 0.3, 0.4)
    a_cut = (1 / 255) * (1 + 1e-9)
    base = _stack_rows([0.3, a_cut, 0.5])
    g = np.array([0.7, -0.4, 0.9]).reshape(3, 1, 1)
    gd = np.array([[0.3]])
    grad, slack = render.render_bwd(records(base), bg, (0, 0, 1, 1), g, gd, amb=F32, with_slack=True)
    below = [list(r) for r in base]
    below[1][5] = (1 / 255) * (1 - 1e-9)
    below[1][10] = 2 * math.log(255 * below[1][5])
    g_below = render.render_bwd(records(below), bg, (0, 0, 1, 1), g, gd)
    np.testing.assert_allclose(slack, np.abs(g_below - grad), rtol=1e-6, atol=1e-12)
    assert slack[1].max() > 0 and slack[2].max() > 0 and slack[0].max() > 0


def test_depth_order_is_the_float32_depth_ties_by_index():
    """Two splats whose depths differ by less than half a float32 ulp round
    to the same float32 depth: they blend in index order, although the
    float64 depths would put the second one first."""
    z = 3.0
    rows = [rec(0.5, 0.5, 1.0, 0.0, 1.0, 0.6, (1, 0, 0), z + 1e-9),
            rec(0.5, 0.5, 1.0, 0.0, 1.0, 0.5, (0, 1, 0), z)]
    assert np.float32(z + 1e-9) == np.float32(z)
    f = render.render_fwd(records(rows), BLACK, (0, 0, 1, 1))
    want = 0.6 * np.array([1, 0, 0]) + 0.5 * 0.4 * np.array([0, 1, 0])
    np.testing.assert_allclose(f["rgb"][:, 0, 0], want, rtol=1e-13)
    assert f["last"][0, 0] == 1
    # one float32 ulp apart: depth order
    rows[0][9] = float(np.nextafter(np.float32(z), np.float32(np.inf)))
    f = render.render_fwd(records(rows), BLACK, (0, 0, 1, 1))
    want = 0.5 * np.array([0, 1, 0]) + 0.6 * 0.5 * np.array([1, 0, 0])
    np.testing.assert_allclose(f["rgb"][:, 0, 0], want, rtol=1e-13)
    assert f["last"][0, 0] == 0


def test_value_bound_of_one_splat():
    """With only the fixed band eps of ln alpha and the rounding t of T, a
    pixel under one splat (alpha, colour c, background b) has the bounds
    alpha |c - b| eps + b (1 - alpha) t for a colour channel,
    alpha eps / z for the disparity and alpha eps + (1 - alpha) t for T."""
    eps, t = 1e-6, 2e-7
    amb = (eps, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, t, 0.0)
    a, z = 0.6, 2.0
    bg = (0.2, 0.3, 0.4)
    col = (0.9, 0.1, 0.5)
    f = render.render_fwd(records([rec(0.5, 0.5, 1.0, 0.0, 1.0, a, col, z)]), bg, (0, 0, 1, 1), amb=amb)
    want = [a * abs(c - b) * eps + b * (1 - a) * t for c, b in zip(col, bg)] + [a * eps / z, a * eps + (1 - a) * t]
    np.testing.assert_allclose(f["bound"][:, 0, 0], want, rtol=1e-12)
