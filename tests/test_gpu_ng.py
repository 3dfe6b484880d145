"""Parity of the tensor-core neural-Gaussian decoder (Sec. 2.3) with the
float64 oracle that rounds to bfloat16 at the same points.

A value the method rounds to bfloat16 is computed in float32 on the GPU and
in float64 by the oracle; when it lies closer to a bfloat16 rounding midpoint
than the float32 rounding error can reach, the two sides may round it
differently.  The bound on that error: a few float32 ulps for the view
direction and dL/dy (a handful of operations), and K float32 ulps of the sum
of |terms| for a K-term tensor-core sum (h: K = 48, dL/dh: K = 144).  Anchors
with such a value are compared with a loose bound; all others strictly."""
import numpy as np
import pytest
import torch

import synth
from oracle import ng as ong
from tests.parity import grad_mismatch, to_np

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _setup(n_anchors, seed):
    pts = synth.scene_clustered(max(4 * n_anchors, 4000), seed=seed, sh_degree=0).means
    d = synth.ng_anchors(pts, n_anchors, seed=seed)
    cam = synth.ring_cameras(8, 640, 360)[seed % 8]
    return d, cam


def _oracle(d, cam):
    R = cam.w2c()[:, :3].astype(np.float64)
    t = cam.w2c()[:, 3].astype(np.float64)
    campos = -(R.T @ t)
    out, cache = ong.decode_forward(d["anchor_xyz"], d["feat"], d["anchor_ls"], d["w1"], d["b1"], d["w2"], d["b2"],
                                    campos)
    xd = cache["x"].numpy()[:, 32:35]
    hp = cache["h_pre"].numpy()
    risky = (ong.bf16_midpoint_distance(xd) < 8 * U32 * np.abs(xd)).any(1)
    err_h = 48 * U32 * cache["h_absum"].numpy()
    risky |= ((ong.bf16_midpoint_distance(hp) < err_h) & (hp > 0)).any(1)
    risky |= (np.abs(hp) < err_h).any(1)  # the ReLU's side may differ
    return out, cache, risky


@pytest.mark.parametrize("n_anchors", [1000, 128, 4177])
def test_ng_decode_forward_matches_oracle(gs, n_anchors):
    from paper_2601_19489_gb300 import api

    d, cam = _setup(n_anchors, seed=n_anchors % 7)
    ng = api.NgParams.from_dict(d)
    ws = api.gs_ng_workspace(n_anchors)
    ch = api.ng_children(n_anchors)
    api.gs_ng_decode_fwd(ng, cam, ch, ws)
    assert api.gs_ng_status(ws) == 0
    out, cache, risky = _oracle(d, cam)
    assert risky.mean() < 0.5
    ok = np.repeat(~risky, 10)
    got = {"means": ch.means, "log_scales": ch.log_scales, "quats": ch.quats, "opacity_logits": ch.opacity_logits,
           "sh": ch.sh}
    for k, t in got.items():
        g = to_np(t).reshape(ok.size, -1).astype(np.float64)
        r = out[k].numpy().reshape(ok.size, -1)
        err = np.abs(g - r)
        tol = 1e-4 * np.abs(r) + 2e-5
        assert np.all(err[ok] <= tol[ok]), (k, err[ok].max(), np.argwhere(err > tol)[:3])
        # anchors next to a rounding midpoint differ by at most a bfloat16 step of h or x
        assert np.all(err <= 0.05 * np.abs(r) + 0.05), (k, err.max())


@pytest.mark.parametrize("n_anchors", [1000, 4177])
def test_ng_decode_backward_matches_oracle(gs, n_anchors):
    from paper_2601_19489_gb300 import api

    d, cam = _setup(n_anchors, seed=n_anchors % 5 + 1)
    out, cache, risky = _oracle(d, cam)
    assert risky.mean() < 0.5
    # an anchor whose forward may round differently has an uncertain y, hence
    # uncertain dL/dy: its children get zero upstream gradient, so that it
    # adds exactly nothing to any gradient on either side
    rng = np.random.default_rng(n_anchors)
    n = n_anchors * 10
    keep = np.repeat(~risky, 10)
    cg_np = {"means": rng.standard_normal((n, 3)), "log_scales": rng.standard_normal((n, 3)),
             "quats": rng.standard_normal((n, 4)), "opacity_logits": rng.standard_normal(n) * 0.1,
             "sh": rng.standard_normal((n, 1, 3))}
    cg_np = {k: (v * keep.reshape((-1,) + (1,) * (v.ndim - 1))).astype(np.float32) for k, v in cg_np.items()}
    ng = api.NgParams.from_dict(d)
    ws = api.gs_ng_workspace(n_anchors)
    ch = api.ng_children(n_anchors)
    api.gs_ng_decode_fwd(ng, cam, ch, ws)
    cg = api.Gaussians(*(torch.from_numpy(cg_np[k]).cuda() for k in
                         ("means", "log_scales", "quats", "opacity_logits", "sh")), 0)
    grads = ng.zeros_like()
    api.gs_ng_decode_bwd(ng, cam, cg, grads, ws)
    assert api.gs_ng_status(ws) == 0
    ref = ong.decode_backward(cache, {k: v.astype(np.float64) for k, v in cg_np.items()})
    # backward roundings: a dL/dy element within the float32 error of a
    # bfloat16 midpoint may round one step differently; that step moves dL/dh
    # by at most step * |W2|, and a dL/dh element within that plus the K = 144
    # tensor-core sum's error of a midpoint may round one step differently too
    dy, dh = ref["_dy"], ref["_dh_pre"]
    w1r, w2r = np.abs(cache["w1r"].numpy()), np.abs(cache["w2r"].numpy())
    ulp = lambda v: np.where(v != 0, np.ldexp(1.0, np.frexp(v)[1] - 8), 0.0)
    flip_dy = np.where(ong.bf16_midpoint_distance(dy) < 8 * U32 * np.abs(dy), ulp(dy), 0.0)
    moved_dh = flip_dy @ w2r
    flip_dh = np.where(ong.bf16_midpoint_distance(dh) < 144 * U32 * ref["_dh_absum"] + moved_dh, ulp(dh), 0.0)
    assert not np.any(ref["feat"][risky]) and not np.any(ref["anchor_ls"][risky])
    # the anchor log-scale gradients involve no bfloat16 rounding
    bad = grad_mismatch(to_np(grads.anchor_ls), ref["anchor_ls"])
    assert bad.sum() == 0, ("anchor_ls", bad.sum())
    # dL/dfeat = W1^T (rounded dL/dh): widened by the flipped steps through |W1|
    g = to_np(grads.feat).astype(np.float64)
    r = ref["feat"]
    tol = 1e-3 * np.maximum(np.abs(r), 1e-3 * np.abs(r).max()) + flip_dh @ w1r[:, :32]
    bad = np.abs(g - r) > tol
    assert bad.sum() == 0, ("feat", bad.sum(), np.argwhere(bad)[:3])
    # the weight and bias gradients sum over all anchors; elementwise they are
    # widened by the worst case of the flipped steps (each flipped operand
    # moves its one product term by its step), and as whole tensors they
    # must agree to 1e-3 in the Frobenius norm
    x = np.abs(cache["x"].numpy())
    h = np.abs(cache["h"].numpy())
    widen_w = {"w1": flip_dh.T @ x, "w2": flip_dy.T @ h, "b1": moved_dh.sum(0), "b2": 0.0}
    for k in ("w1", "b1", "w2", "b2"):
        g = to_np(getattr(grads, k)).astype(np.float64)
        r = ref[k]
        tol = 1e-3 * np.maximum(np.abs(r), 1e-3 * np.abs(r).max()) + widen_w[k]
        bad = np.abs(g - r) > tol
        assert bad.sum() == 0, (k, bad.sum(), np.abs(g - r).max(), np.abs(r).max())
        assert np.linalg.norm(g - r) <= 1e-3 * np.linalg.norm(r), (k, np.linalg.norm(g - r), np.linalg.norm(r))
