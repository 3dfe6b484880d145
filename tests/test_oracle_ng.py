"""Pins of the neural-Gaussian decoder oracle (Sec. 2.3): bfloat16 rounding
against torch's conversion, the explicit backward against autograd of the
forward (rounding off), finite differences, and closed-form children."""
import math

import numpy as np
import torch

import synth
from oracle import ng

CAM = np.array([0.3, -0.2, 4.0])


def _anchors(n=40, seed=0):
    pts = synth.scene_clustered(2000, seed=seed, sh_degree=0).means
    return synth.ng_anchors(pts, n, seed=seed)


def test_bf16_round_matches_torch_on_float32_values():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-10, 10, 20000))).astype(np.float32)
    want = torch.as_tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = ng.bf16_round(torch.as_tensor(x.astype(np.float64))).numpy()
    np.testing.assert_array_equal(got, want)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    np.testing.assert_array_equal(ng.bf16_round(torch.tensor([1 + 2 ** -8, 1 + 3 * 2 ** -8])).numpy(),
                                  [1.0, 1 + 2 ** -6])


def test_explicit_backward_equals_autograd_without_rounding():
    p = _anchors(30, seed=1)
    T = {k: torch.as_tensor(v.astype(np.float64)).requires_grad_(k != "anchor_xyz") for k, v in p.items()}
    out, cache = ng.decode_forward(T["anchor_xyz"], T["feat"], T["anchor_ls"], T["w1"], T["b1"], T["w2"],
                                   T["b2"], CAM, bf16=False)
    rng = np.random.default_rng(2)
    gout = {k: torch.as_tensor(rng.standard_normal(v.shape)) for k, v in out.items()}
    # opacity <= 0 children have no gradient path: their logit is a constant
    total = sum((out[k] * gout[k]).sum() for k in out)
    total.backward()
    got = ng.decode_backward(cache, {k: v.numpy() for k, v in gout.items()}, bf16=False)
    for k in ("feat", "anchor_ls", "w1", "b1", "w2", "b2"):
        np.testing.assert_allclose(got[k], T[k].grad.numpy(), rtol=1e-10, atol=1e-12, err_msg=k)


def test_forward_finite_differences_of_one_feature():
    p = _anchors(8, seed=3)
    rng = np.random.default_rng(4)
    gout = None
    base = {k: v.astype(np.float64) for k, v in p.items()}

    def L(q):
        out, cache = ng.decode_forward(q["anchor_xyz"], q["feat"], q["anchor_ls"], q["w1"], q["b1"], q["w2"],
                                       q["b2"], CAM, bf16=False)
        return out, cache

    out, cache = L(base)
    gout = {k: rng.standard_normal(v.shape) for k, v in out.items()}
    g = ng.decode_backward(cache, gout, bf16=False)
    for (a, j) in [(0, 0), (3, 17), (7, 31)]:
        h = 1e-6
        qp = {k: v.copy() for k, v in base.items()}
        qm = {k: v.copy() for k, v in base.items()}
        qp["feat"][a, j] += h
        qm["feat"][a, j] -= h
        fp = sum(float((L(qp)[0][k].numpy() * gout[k]).sum()) for k in gout)
        fm = sum(float((L(qm)[0][k].numpy() * gout[k]).sum()) for k in gout)
        np.testing.assert_allclose(g["feat"][a, j], (fp - fm) / (2 * h), rtol=1e-6, atol=1e-9)


def test_children_closed_form_with_constant_mlp():
    p = _anchors(5, seed=5)
    p["w2"][:] = 0.0  # y = b2 for every anchor
    b2 = np.zeros(140)
    u = b2.reshape(10, 14)
    u[:, 0:3] = math.atanh(0.5)
    u[:, 3] = math.atanh(0.25)
    u[:, 4:7] = 0.0
    u[:, 7:10] = math.log(3.0)  # sigmoid = 3/4
    u[:, 10:14] = [0.5, 0.5, 0.5, 0.5]
    u[2, 3] = -1.0  # a child with negative opacity
    out, _ = ng.decode_forward(p["anchor_xyz"], p["feat"], p["anchor_ls"], p["w1"], p["b1"], p["w2"], b2, CAM,
                               bf16=False)
    xyz = p["anchor_xyz"].astype(np.float64)
    ls = p["anchor_ls"].astype(np.float64)
    means = out["means"].numpy().reshape(5, 10, 3)
    want = np.broadcast_to(xyz[:, None, :] + 0.5 * np.exp(ls[:, None, 0:3]), means.shape)
    np.testing.assert_allclose(means, want, rtol=1e-9)
    logit = out["opacity_logits"].numpy().reshape(5, 10)
    np.testing.assert_allclose(logit[:, 0], math.log(0.25 / 0.75), rtol=1e-12)
    assert np.all(logit[:, 2] == ng.LOGIT_FLOOR)
    np.testing.assert_allclose(out["sh"].numpy(), 0.0, atol=1e-15)  # colour 0.5 -> DC 0
    np.testing.assert_allclose(out["log_scales"].numpy().reshape(5, 10, 3),
                               np.broadcast_to(ls[:, None, 3:6] + math.log(0.75), (5, 10, 3)), rtol=1e-12)
    np.testing.assert_allclose(out["quats"].numpy(), 0.5)


def test_rounding_points_change_results_only_at_bf16_level():
    p = _anchors(64, seed=6)
    a, _ = ng.decode_forward(p["anchor_xyz"], p["feat"], p["anchor_ls"], p["w1"], p["b1"], p["w2"], p["b2"], CAM)
    b, _ = ng.decode_forward(p["anchor_xyz"], p["feat"], p["anchor_ls"], p["w1"], p["b1"], p["w2"], p["b2"], CAM,
                             bf16=False)
    d = np.abs(a["quats"].numpy() - b["quats"].numpy()).max()
    assert 1e-6 < d < 5e-2
