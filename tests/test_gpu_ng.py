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
    cg2 = api.Gaussians(*(t.clone() for t in cg.tensors()), 0)
    api.gs_ng_decode_bwd(ng, cam, cg, grads, ws)
    assert api.gs_ng_status(ws) == 0
    # the sums over anchors run in a fixed order: a second run is bit-identical
    grads2 = ng.zeros_like()
    api.gs_ng_decode_bwd(ng, cam, cg2, grads2, ws)
    for k in ("feat", "anchor_ls", "w1", "b1", "w2", "b2"):
        assert torch.equal(getattr(grads, k), getattr(grads2, k)), k
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


def _tiny_chain(seed=3, W=48, H=48):
    """Six anchors in front of a 48 x 48 camera, children a few pixels wide;
    seed 3: no decoder value near a bfloat16 midpoint and no pixel near a
    float32 blend threshold."""
    cam = synth.camera_tiny(W, H)
    pts = synth.scene_tiny(6, seed=seed, sh_degree=0, width=W, height=H).means
    d = synth.ng_anchors(pts, 6, seed=seed)
    d["anchor_ls"][:, 0:3] = np.log(0.15)
    d["anchor_ls"][:, 3:6] = np.log(0.25)
    target = np.random.default_rng(seed).uniform(2.0, 2.5, size=(3, H, W))
    return cam, d, target


def test_ng_training_step_chain_matches_oracle(gs):
    """decode -> splat -> loss -> splat backward -> decode backward, the
    decoder gradients against the oracle's chain.  The children's gradients
    reaching the decoder carry the splatting backward's float32 error
    (within 1e-3 relative, the splatting parity bar), which the bfloat16
    rounding of dL/dy may turn into one bfloat16 step (2^-8 relative) per
    element; the decoder gradients are compared at 1e-2 of their scale."""
    from oracle import step as ostep
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import NgTrainer

    cam, d, target = _tiny_chain()
    out, cache = ong.decode_forward(d["anchor_xyz"], d["feat"], d["anchor_ls"], d["w1"], d["b1"], d["w2"],
                                    d["b2"], np.zeros(3))
    sc = synth.Scene(out["means"].numpy(), out["log_scales"].numpy(), out["quats"].numpy(),
                     out["opacity_logits"].numpy(), out["sh"].numpy(), 0)
    ref_L, g, _ = ostep.forward_backward(sc, cam, target, lam=0.2)
    ref = ong.decode_backward(cache, g)

    ng = api.NgParams.from_dict(d)
    tr = NgTrainer(ng, cam.width, cam.height, lam=0.2, inst_capacity=1 << 16)
    tgt = torch.from_numpy(target.reshape(-1).astype(np.float32)).cuda()
    # the stages of NgTrainer.step up to (not including) its Adam update
    s = torch.cuda.current_stream().cuda_stream
    tr._decode(cam, s)
    tr._splat_stages([cam], tgt, None, s, lambda i: None, 0)
    import ctypes
    from paper_2601_19489_gb300 import _lib as L
    L.check(L.lib().gs_ng_decode_bwd(ctypes.byref(tr._ngp), tr._cam([cam]), ctypes.byref(tr._gstruct), 1,
                                     ctypes.byref(tr._ngg), tr.ng_ws.data_ptr(), s), "gs_ng_decode_bwd")
    assert tr.status() == 0 and tr.plan.status()["rc"] == 0
    np.testing.assert_allclose(tr.loss.item(), ref_L, rtol=1e-5)
    for t in tr.grads.tensors():  # consumed by the decoder backward
        assert float(t.abs().max()) == 0.0
    for k in ("feat", "anchor_ls", "w1", "b1", "w2", "b2"):
        got = to_np(getattr(tr.ng_grads, k)).astype(np.float64).reshape(ref[k].shape)
        r = ref[k]
        assert np.linalg.norm(got - r) <= 1e-2 * np.linalg.norm(r), (k, np.linalg.norm(got - r), np.linalg.norm(r))
        assert np.abs(got - r).max() <= 1e-2 * np.abs(r).max(), (k, np.abs(got - r).max(), np.abs(r).max())


def test_ng_trainer_learns_and_replays_as_a_graph(gs):
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import NgTrainer

    cam, d, target = _tiny_chain()
    target = np.clip(target - 1.8, 0.0, 1.0)  # reachable colours
    tgt = torch.from_numpy(target.reshape(-1).astype(np.float32)).cuda()
    runs = []
    for graphed in (False, True):
        ng = api.NgParams.from_dict(d)
        xyz0 = ng.anchor_xyz.clone()
        tr = NgTrainer(ng, cam.width, cam.height, lam=0.2, inst_capacity=1 << 16)
        tr.ensure_capacity([cam])
        losses = []
        tr.step(cam, tgt)
        losses.append(tr.loss.item())
        g = tr.capture(cam, tgt) if graphed else None
        for _ in range(29):
            g.replay() if graphed else tr.step(cam, tgt)
            losses.append(tr.loss.item())
        torch.cuda.synchronize()
        assert tr.status() == 0 and tr.plan.status()["rc"] == 0
        assert int(tr.d_step.item()) == 30
        assert torch.equal(ng.anchor_xyz, xyz0)  # anchors stay where they are
        runs.append(losses)
    assert runs[0][-1] < 0.9 * runs[0][0], runs[0]
    np.testing.assert_allclose(runs[1], runs[0], rtol=1e-3)


@pytest.mark.parametrize("n_anchors,box3", [(1000, 0), (4177, 0), (1000, 1)])
def test_fused_decode_preprocess_equals_two_launches(gs, n_anchors, box3):
    """gs_ng_decode_preprocess against gs_ng_decode_fwd + gs_preprocess on
    the same anchors and camera: the children's parameters, blend records,
    level sets, tile counts and rectangles are bit-identical, and so are the
    tile lists after the binning (so the depth keys are too)."""
    from paper_2601_19489_gb300 import _lib as L
    from paper_2601_19489_gb300 import api

    d, cam = _setup(n_anchors, seed=n_anchors % 5 + 1)
    ng = api.NgParams.from_dict(d)
    out = []
    for fused in (False, True):
        ws = api.gs_ng_workspace(n_anchors)
        ch = api.ng_children(n_anchors)
        plan = api.Plan(ch.n, 0, [(cam.width, cam.height)], 1 << 22, tuning={"bbox_3sigma": box3})
        if fused:
            api.gs_ng_decode_preprocess(ng, cam, ch, ws, plan)
        else:
            api.gs_ng_decode_fwd(ng, cam, ch, ws)
            api.gs_preprocess(plan, ch, [cam])
        bufs = [to_np(plan.view(w, torch.int32)).copy() for w in (L.GS_WS_RECORDS, L.GS_WS_BIN,
                                                                 L.GS_WS_TILES_TOUCHED, L.GS_WS_RECTS)]
        api.gs_bin_sort(plan, True)
        st = plan.status()
        assert st["rc"] == 0 and st["n_instances"] > 0, st
        ranges = to_np(plan.view(L.GS_WS_TILE_RANGES, torch.int32)).reshape(-1, 2).copy()
        items = to_np(plan.view(L.GS_WS_INST_GID, torch.int32))[: st["n_instances"]].copy()
        assert api.gs_ng_status(ws) == 0
        out.append(([to_np(t).copy() for t in ch.tensors()], bufs, ranges, items))
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][2], out[1][2]) and np.array_equal(out[0][3], out[1][3])


def test_fused_decode_trainer_step_equals_unfused(gs):
    """The neural-Gaussian training step with the fused decode + preprocess:
    the first step's loss is bit-identical to the two-launch step, and both
    keep training to the same losses (float32 atomics order aside)."""
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import NgTrainer

    cam, d, target = _tiny_chain()
    tgt = torch.from_numpy(np.clip(target - 1.8, 0.0, 1.0).reshape(-1).astype(np.float32)).cuda()
    runs = []
    for fused in (False, True):
        tr = NgTrainer(api.NgParams.from_dict(d), cam.width, cam.height, lam=0.2, inst_capacity=1 << 16,
                       fused_decode=fused)
        tr.ensure_capacity([cam])
        losses = []
        for _ in range(10):
            tr.step(cam, tgt)
            losses.append(tr.loss.item())
        torch.cuda.synchronize()
        assert tr.status() == 0 and tr.plan.status()["rc"] == 0
        runs.append(losses)
    assert runs[0][0] == runs[1][0]
    np.testing.assert_allclose(runs[1], runs[0], rtol=1e-3)


@pytest.mark.slow
def test_ng_decode_forward_at_full_size_on_sampled_anchors(gs):
    """The decoder at the benchmark's size (104,857 anchors -> 1,048,570
    children, a 1080p ring view): the children of 512 sampled anchors,
    spread over every CTA tile, against the oracle (each anchor's decode
    depends only on its own inputs and the shared MLP)."""
    from paper_2601_19489_gb300 import api

    n = (1 << 20) // 10
    pts = synth.scene_clustered(1 << 20, seed=0, sh_degree=0).means
    d = synth.ng_anchors(pts, n, seed=0)
    cam = synth.ring_cameras(16, 1920, 1080)[0]
    ng = api.NgParams.from_dict(d)
    ws = api.gs_ng_workspace(n)
    ch = api.ng_children(n)
    api.gs_ng_decode_fwd(ng, cam, ch, ws)
    assert api.gs_ng_status(ws) == 0
    pick = np.sort(np.random.default_rng(8).choice(n, size=512, replace=False))
    pick[-1] = n - 1  # the ragged last tile
    sub = {k: (v[pick] if k in ("anchor_xyz", "feat", "anchor_ls") else v) for k, v in d.items()}
    out, cache, risky = _oracle(sub, cam)
    assert risky.mean() < 0.5
    rows = (pick[:, None] * 10 + np.arange(10)[None]).reshape(-1)
    ok = np.repeat(~risky, 10)
    got = {"means": ch.means, "log_scales": ch.log_scales, "quats": ch.quats, "opacity_logits": ch.opacity_logits,
           "sh": ch.sh}
    for k, t in got.items():
        g = to_np(t).reshape(n * 10, -1)[rows].astype(np.float64)
        r = out[k].numpy().reshape(ok.size, -1)
        err = np.abs(g - r)
        tol = 1e-4 * np.abs(r) + 2e-5
        assert np.all(err[ok] <= tol[ok]), (k, err[ok].max())
        assert np.all(err <= 0.05 * np.abs(r) + 0.05), (k, err.max())


def test_bounded_wait_runs_out_and_reports_a_timeout(gs):
    """Failure detection without a GPU fault: the decoder's bounded mbarrier
    wait, on a barrier nothing arrives on (no copy and no MMA in flight),
    gives up after its try limit and records GS_ERR_TIMEOUT; the launch
    returns and the context stays usable.  With an arrival first, the same
    wait succeeds and records nothing."""
    import time

    from paper_2601_19489_gb300 import _lib as L

    lib = L.load()
    s = torch.cuda.current_stream().cuda_stream
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    assert lib.gs_ng_wait_probe(err.data_ptr(), 1000, 0, s) == 0
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 5.0
    assert int(err.item()) == L.GS_ERR_TIMEOUT
    err.zero_()
    assert lib.gs_ng_wait_probe(err.data_ptr(), 1000, 1, s) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    # the context is still usable after the timed-out wait
    x = torch.arange(1000, device="cuda", dtype=torch.float32)
    assert float(x.sum().item()) == 499500.0
    # arguments outside the stated range are refused before any launch
    assert lib.gs_ng_wait_probe(err.data_ptr(), 0, 0, s) == L.GS_ERR_ARG
    assert lib.gs_ng_wait_probe(err.data_ptr(), (1 << 22) + 1, 0, s) == L.GS_ERR_ARG
    assert lib.gs_ng_wait_probe(None, 10, 0, s) == L.GS_ERR_ARG
