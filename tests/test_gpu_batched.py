"""The batched multi-view training step (several views of uneven resolution
per launch, gradients summed, one Adam update) against the oracle, and its
CUDA-graph replay against eager execution."""
import numpy as np
import pytest
import torch

import synth
from oracle import adam as oadam
from oracle import step as ostep
from tests.parity import grad_mismatch, to_np

pytestmark = pytest.mark.gpu

SIZES = [(96, 54), (128, 72), (160, 90)]
BG = (0.0, 0.0, 0.0)


def _batch():
    # 400 Gaussians, seed 1: the oracle flags no pixel of these three views
    # as near a float32 branch threshold, so every pixel is compared
    scene = synth.scene_clustered(400, seed=1, sh_degree=1)
    cams = [synth.ring_cameras(5, w, h)[i] for i, (w, h) in enumerate(SIZES)]
    rng = np.random.default_rng(7)
    # targets beyond every rendered value keep the L1 terms off their kinks
    targets = [rng.uniform(2.0, 2.5, size=(3, h, w)) for (w, h) in SIZES]
    dts = [rng.uniform(-0.1, -0.05, size=(h, w)) for (w, h) in SIZES]
    return scene, cams, targets, dts


def _flat(arrs, planar=True):
    return torch.from_numpy(np.concatenate([a.reshape(-1) for a in arrs]).astype(np.float32)).cuda()


@pytest.mark.parametrize("betas", [(0.9, 0.999), (0.9 ** 8, 0.999 ** 8)])
def test_adam_device_step_matches_oracle(gs, betas):
    """Default betas and the batch-scaled ones of an 8-view batch (beta^8:
    beta1 below 0.5, where b - 1 in the bias correction rounds)."""
    from paper_2601_19489_gb300 import api

    b1, b2 = betas

    rng = np.random.default_rng(11)
    n = 5003
    p0 = rng.standard_normal(n).astype(np.float32)
    q0 = rng.standard_normal(96).astype(np.float32)
    p, q = torch.from_numpy(p0.copy()).cuda(), torch.from_numpy(q0.copy()).cuda()
    mp, vp, mq, vq = (torch.zeros_like(t) for t in (p, p, q, q))
    d_step = torch.zeros(1, dtype=torch.int32, device="cuda")
    ref = {"p": p0.astype(np.float64), "mp": np.zeros(n), "vp": np.zeros(n),
           "q": q0.astype(np.float64), "mq": np.zeros(96), "vq": np.zeros(96)}
    for step in range(1, 5):
        gp0 = rng.standard_normal(n).astype(np.float32)
        gq0 = rng.standard_normal(96).astype(np.float32)
        gp, gq = torch.from_numpy(gp0.copy()).cuda(), torch.from_numpy(gq0.copy()).cuda()
        api.gs_adam_step_multi_dev([{"p": p, "g": gp, "m": mp, "v": vp, "lr": 1e-2},
                                    {"p": q, "g": gq, "m": mq, "v": vq, "lr": 3e-3, "period": 48, "head": 3,
                                     "lr_head": 5e-2}], d_step, b1=b1, b2=b2)
        ref["p"], ref["mp"], ref["vp"] = oadam.adam_step(ref["p"], gp0, ref["mp"], ref["vp"], step, lr=1e-2,
                                                         b1=b1, b2=b2)
        lr_q = np.where(np.arange(96) % 48 < 3, 5e-2, 3e-3)
        ref["q"], ref["mq"], ref["vq"] = oadam.adam_step(ref["q"], gq0, ref["mq"], ref["vq"], step, lr=lr_q,
                                                         b1=b1, b2=b2)
        assert float(gp.abs().max()) == 0.0 and float(gq.abs().max()) == 0.0
    assert int(d_step.item()) == 4
    np.testing.assert_allclose(to_np(p), ref["p"], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(to_np(q), ref["q"], rtol=1e-5, atol=1e-6)


def test_batched_step_gradients_match_oracle(gs):
    from paper_2601_19489_gb300 import api

    scene, cams, targets, dts = _batch()
    plan = api.Plan(scene.n, scene.sh_degree, SIZES, 1 << 20)
    params = api.Gaussians.from_scene(scene)
    P = plan.pixels
    rgb, disp, T = (torch.empty(k * P, device="cuda") for k in (3, 1, 1))
    dL, dLd = torch.empty(3 * P, device="cuda"), torch.empty(P, device="cuda")
    loss = torch.zeros(1, device="cuda")
    api.gs_preprocess(plan, params, cams)
    api.gs_bin_sort(plan, True)
    api.gs_render_fwd(plan, BG, rgb, disp, T)
    api.gs_loss(plan, rgb, _flat(targets), 0.2, dL, loss, api.gs_loss_scratch(plan), disp=disp,
                target_disp=_flat(dts), disp_weight=0.1, dL_ddisp=dLd)
    grads = params.zeros_like()
    api.gs_render_bwd(plan, params, cams, BG, rgb, disp, dL, dLd, grads)
    assert plan.status()["rc"] == 0
    sc64 = synth.Scene(*(a.astype(np.float64) for a in scene.arrays()), sh_degree=scene.sh_degree)
    ref_L, ref = ostep.forward_backward_batch(sc64, cams, targets, bg=BG, lam=0.2, disp_targets=dts,
                                              disp_weight=0.1)
    np.testing.assert_allclose(loss.item(), ref_L, rtol=1e-5)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        got = to_np(getattr(grads, k)).reshape(ref[k].shape)
        bad = grad_mismatch(got, ref[k])
        assert bad.sum() == 0, (k, int(bad.sum()), np.abs(got - ref[k]).max(), np.abs(ref[k]).max())


def test_graph_replay_matches_eager_steps(gs):
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer

    scene, cams, targets, dts = _batch()
    tgt, tdisp = _flat(targets), _flat(dts)
    trainers = []
    for _ in range(2):
        tr = Trainer(api.Gaussians.from_scene(scene), lam=0.2, disp_weight=0.1, inst_capacity=1 << 20)
        tr.ensure_capacity([cams])
        trainers.append(tr)
    eager, graphed = trainers
    losses = ([], [])
    for i in range(5):
        eager.step(cams, tgt, tdisp)
        losses[0].append(eager.loss.item())
    graphed.step(cams, tgt, tdisp)  # the first step eagerly: loads every kernel before capture
    losses[1].append(graphed.loss.item())
    g = graphed.capture(cams, tgt, tdisp)
    for i in range(4):
        g.replay()
        losses[1].append(graphed.loss.item())
    torch.cuda.synchronize()
    assert int(eager.d_step.item()) == 5 and int(graphed.d_step.item()) == 5
    assert graphed.step_count == 5
    np.testing.assert_allclose(losses[1], losses[0], rtol=1e-4)
    assert losses[0][-1] < losses[0][0]
    # Adam's first steps move a parameter by about its learning rate whatever
    # the gradient's size, so a gradient that cancels to nearly zero may take
    # either sign under a different atomic order; all but a few elements agree
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        a = to_np(getattr(eager.params, k))
        b = to_np(getattr(graphed.params, k))
        off = np.abs(a - b) > 1e-6 * np.maximum(1.0, np.abs(a))
        assert off.mean() < 0.01, (k, off.mean())
    assert graphed.slot_for(cams).plan.status()["rc"] == 0


def test_per_view_graphs_round_robin_match_eager_steps(gs):
    """The benchmark's step loop: one captured graph per view on one trainer
    (the views share its plan and buffers), replayed round robin, each view's
    target refilled from pinned host memory on a side stream before its
    replay, against the same single-view steps launched eagerly."""
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer

    W, H = 160, 90
    scene = synth.scene_clustered(400, seed=1, sh_degree=1)
    cams = synth.ring_cameras(5, W, H)[:3]
    rng = np.random.default_rng(8)
    tgt_h = [torch.from_numpy(rng.uniform(2.0, 2.5, size=3 * W * H).astype(np.float32)).pin_memory()
             for _ in cams]
    order = [0, 1, 2, 0, 1, 2, 0]
    eager, graphed = (Trainer(api.Gaussians.from_scene(scene), W, H, lam=0.2, inst_capacity=1 << 20)
                      for _ in range(2))
    for tr in (eager, graphed):
        tr.ensure_capacity(cams)
    tgt_e = [t.cuda() for t in tgt_h]
    losses = ([], [])
    for v in order:
        eager.step(cams[v], tgt_e[v])
        losses[0].append(eager.loss.item())
    # the graphs' target buffers start empty: every replay sees the refill
    tgt_g = [torch.zeros_like(t) for t in tgt_e]
    tgt_g[order[0]].copy_(tgt_h[order[0]])
    graphed.step(cams[order[0]], tgt_g[order[0]])  # eager first: loads every kernel before capture
    losses[1].append(graphed.loss.item())
    graphs = [graphed.capture([c], t) for c, t in zip(cams, tgt_g)]
    stream, side = torch.cuda.current_stream(), torch.cuda.Stream()
    for v in order[1:]:
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            tgt_g[v].copy_(tgt_h[v], non_blocking=True)
        stream.wait_stream(side)
        graphs[v].replay()
        losses[1].append(graphed.loss.item())
    torch.cuda.synchronize()
    assert graphed.step_count == len(order) and int(graphed.d_step.item()) == len(order)
    np.testing.assert_allclose(losses[1], losses[0], rtol=1e-4)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        a = to_np(getattr(eager.params, k))
        b = to_np(getattr(graphed.params, k))
        off = np.abs(a - b) > 1e-6 * np.maximum(1.0, np.abs(a))
        assert off.mean() < 0.01, (k, off.mean())
    assert graphed.plan.status()["rc"] == 0


def test_fused_preprocess_backward_adam_equals_unfused(gs):
    """The fused preprocess backward + Adam against the separate kernels on
    the same blend gradients, over three updates (moments evolving)."""
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer, default_lrs

    scene, cams, targets, dts = _batch()
    tr = Trainer(api.Gaussians.from_scene(scene), lam=0.2, disp_weight=0.1, inst_capacity=1 << 20)
    tr.ensure_capacity([cams])
    sl = tr.slot_for(cams)
    lrs = default_lrs()
    # parameters, first and second moments of each side
    fused = [api.Gaussians(*(t.clone() for t in tr.params.tensors()), scene.sh_degree)]
    fused += [tr.params.zeros_like(), tr.params.zeros_like()]
    unf = [api.Gaussians(*(t.clone() for t in tr.params.tensors()), scene.sh_degree)]
    unf += [tr.params.zeros_like(), tr.params.zeros_like()]
    step_f = torch.zeros(1, dtype=torch.int32, device="cuda")
    step_u = torch.zeros(1, dtype=torch.int32, device="cuda")
    grads = tr.params.zeros_like()
    tgt, tdisp = _flat(targets), _flat(dts)
    for it in range(3):
        # blend gradients of the current (fused) parameters, shared by both
        tr.params = fused[0]
        tr._build_adam()
        tr._splat_stages(cams, tgt, tdisp, torch.cuda.current_stream().cuda_stream, lambda i: None, 0,
                         with_pbwd=False)
        api.gs_preprocess_bwd_adam(sl.plan, fused[0], cams, fused[1], fused[2], lrs, step_f)
        for t in grads.tensors():
            t.zero_()
        from paper_2601_19489_gb300 import _lib as L
        import ctypes
        p, g = unf[0].struct(), grads.struct()
        L.check(L.lib().gs_preprocess_bwd(sl.plan.handle, sl.plan.ws.data_ptr(), ctypes.byref(p),
                                          api.cameras_array(cams), ctypes.byref(g),
                                          torch.cuda.current_stream().cuda_stream), "gs_preprocess_bwd")
        groups = []
        for name in ("means", "log_scales", "quats", "opacity_logits"):
            groups.append({"p": getattr(unf[0], name), "g": getattr(grads, name), "m": getattr(unf[1], name),
                           "v": getattr(unf[2], name), "lr": lrs[name]})
        K = (scene.sh_degree + 1) ** 2
        groups.append({"p": unf[0].sh, "g": grads.sh, "m": unf[1].sh, "v": unf[2].sh, "lr": lrs["sh_rest"],
                       "period": 3 * K, "head": 3, "lr_head": lrs["sh_dc"]})
        api.gs_adam_step_multi_dev(groups, step_u)
        torch.cuda.synchronize()
        assert int(step_f.item()) == int(step_u.item()) == it + 1
        for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            a, b = to_np(getattr(fused[0], name)), to_np(getattr(unf[0], name))
            off = np.abs(a - b) > 1e-6 * np.maximum(1.0, np.abs(b))
            # a gradient that cancels to a few ulps may take either sign
            assert off.mean() < 1e-3, (name, it, off.mean())
            assert np.abs(a - b).max() <= 2.5 * max(lrs.values()) * (it + 1), (name, it)
            # and both copies stay in step from here on
            getattr(unf[0], name).copy_(getattr(fused[0], name))
        for k in range(1, 3):
            for t_u, t_f in zip(unf[k].tensors(), fused[k].tensors()):
                t_u.copy_(t_f)


def test_visible_only_adam_matches_oracle(gs):
    """The fused update in its visible-only form against the oracle's sparse
    Adam over two steps: a third of the Gaussians sit far above the ring of
    views, so they touch no tile and must keep their parameters and moments
    bit for bit; the others follow the oracle's Adam."""
    from oracle import binning as obin
    from oracle import preprocess as opre
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer, default_lrs

    scene, cams, targets, dts = _batch()
    scene = scene.copy()
    scene.means[::3] += np.array([0.0, -60.0, 0.0], dtype=np.float32)
    tgt, tdisp = _flat(targets), _flat(dts)
    lrs = default_lrs()
    tr = Trainer(api.Gaussians.from_scene(scene), lam=0.2, disp_weight=0.1, lrs=lrs, inst_capacity=1 << 20,
                 visible_adam=True)
    tr.ensure_capacity([cams])
    names = ("means", "log_scales", "quats", "opacity_logits", "sh")
    p0 = {k: to_np(getattr(tr.params, k)).copy() for k in names}
    st = ostep.new_state(synth.Scene(*(a.astype(np.float64) for a in scene.arrays()), sh_degree=scene.sh_degree))
    for it in range(2):
        sc = ostep.scene_from_state(st, scene)
        # visibility as the binning defines it: some tile of some view within
        # the level set; Gaussians within the binning's widening of it are
        # ambiguous and compared loosely
        vis, amb = np.zeros(scene.n, bool), np.zeros(scene.n, bool)
        for cam in cams:
            rec = opre.pack_for_render(opre.project(opre.params_from_scene(sc), cam, sc.sh_degree))
            for gid, (ids, mq, t) in obin.tile_min_q(rec, cam.width, cam.height).items():
                vis[gid] |= bool(np.any(mq <= t))
                amb[gid] |= bool(np.any(mq <= t * (1 + 2.0 ** -9) + 2.0 ** -11)) and not np.any(mq <= t)
        _, g = ostep.forward_backward_batch(sc, cams, targets, bg=BG, lam=0.2, disp_targets=dts, disp_weight=0.1)
        st["step"] += 1
        gsplit = ostep._split(g)
        for k in ostep.GROUPS:
            st["params"][k], st["m"][k], st["v"][k] = oadam.adam_step_visible(
                st["params"][k], gsplit[k], st["m"][k], st["v"][k], st["step"], lrs[k], vis)
        tr.step(cams, tgt, tdisp)
    torch.cuda.synchronize()
    assert tr.slot_for(cams).plan.status()["rc"] == 0
    hidden = ~vis & ~amb
    assert hidden.sum() >= scene.n // 3 - 2
    ref = {"means": st["params"]["means"], "log_scales": st["params"]["log_scales"], "quats": st["params"]["quats"],
           "opacity_logits": st["params"]["opacity_logits"],
           "sh": np.concatenate([st["params"]["sh_dc"], st["params"]["sh_rest"]], axis=1)}
    for k in names:
        got = to_np(getattr(tr.params, k)).reshape(ref[k].shape)
        base = p0[k].reshape(ref[k].shape)
        # never-visible Gaussians: untouched, bit for bit, moments still zero
        np.testing.assert_array_equal(got[hidden], base[hidden], err_msg=k)
        for mom in (tr.m, tr.v):
            assert not np.any(to_np(getattr(mom, k)).reshape(ref[k].shape)[hidden]), k
        # the others follow the oracle (a gradient that cancels to a few ulps
        # may take either sign in Adam's first steps)
        live = vis & ~amb
        off = np.abs(got[live] - ref[k][live]) > 1e-5 * np.maximum(1.0, np.abs(ref[k][live]))
        assert off.mean() < 0.01, (k, off.mean())
        assert np.abs(got[live] - ref[k][live]).max() <= 2.5 * max(lrs.values()) * 2, k


@pytest.mark.slow
def test_visible_only_adam_at_1m_1080p(gs):
    """At the full size (1M clustered Gaussians, 1080p views from a ring of
    radius 2.2 that leaves about half of them outside each view), two steps
    on two views, visible-only against dense Adam: a Gaussian outside the
    second view keeps its first-step state bit for bit under the visible-only
    update while the dense update keeps moving it (momentum); Gaussians inside
    the second view get the same update from both."""
    from paper_2601_19489_gb300 import _lib as L
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer

    scene = synth.scene_clustered(1 << 20, seed=0, sh_degree=3)
    ring = synth.ring_cameras(16, 1920, 1080, radius=2.2)
    views = [ring[2], ring[6]]  # a quarter turn apart: each sees Gaussians the other does not
    tgt = [torch.from_numpy(synth.target_uniform(12 + i, 1920, 1080).reshape(-1)).cuda() for i in range(2)]
    names = ("means", "log_scales", "quats", "opacity_logits", "sh")
    tr = {}
    for vis in (False, True):
        t = Trainer(api.Gaussians.from_scene(scene), 1920, 1080, visible_adam=vis)
        t.ensure_capacity([[c] for c in views])
        t.step([views[0]], tgt[0])
        tr[vis] = t
    s1 = {k: (getattr(tr[True].params, k).clone(), getattr(tr[True].m, k).clone(), getattr(tr[True].v, k).clone())
          for k in names}
    d1 = {k: getattr(tr[False].params, k).clone() for k in names}
    for t in tr.values():
        t.step([views[1]], tgt[1])
    torch.cuda.synchronize()
    sl = tr[True].slot_for([views[1]])
    assert sl.plan.status()["rc"] == 0
    seen = sl.plan.view(L.GS_WS_TILES_TOUCHED, torch.int32)[: scene.n] > 0
    assert 0.2 < float(seen.float().mean()) < 0.9
    hidden = ~seen
    for k in names:
        p, m, v = (getattr(g, k) for g in (tr[True].params, tr[True].m, tr[True].v))
        assert torch.equal(p[hidden], s1[k][0][hidden]), k
        assert torch.equal(m[hidden], s1[k][1][hidden]) and torch.equal(v[hidden], s1[k][2][hidden]), k
        # the dense update moves the hidden Gaussians that carry momentum
        mom = (s1[k][1][hidden] != 0).reshape(int(hidden.sum()), -1).any(1)
        assert int(mom.sum()) > 1000, k
        dense_moved = (getattr(tr[False].params, k)[hidden] != d1[k][hidden]).reshape(int(hidden.sum()), -1).any(1)
        assert float(dense_moved[mom].float().mean()) > 0.9, k
        # inside the second view both take the same update (up to the order
        # of the gradient's atomic sums)
        a, b = p[seen], getattr(tr[False].params, k)[seen]
        off = (a - b).abs() > 1e-6 * torch.clamp(b.abs(), min=1.0)
        assert float(off.float().mean()) < 0.01, k
