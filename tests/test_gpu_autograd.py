"""The blend backward behind torch.autograd: gradients through GsRender
against the oracle's exact gradient, and against float32 central finite
differences of the CUDA forward itself."""
import numpy as np
import pytest
import torch

import synth
from oracle import preprocess as opre
from oracle import render as oren
from tests.parity import block_mismatch, to_np

pytestmark = pytest.mark.gpu

BG = (0.1, 0.2, 0.3)
NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _leaf_params(scene):
    from paper_2601_19489_gb300 import api

    p = api.Gaussians.from_scene(scene)
    return api.Gaussians(*(t.clone().requires_grad_(True) for t in p.tensors()), p.sh_degree)


def test_autograd_gradient_matches_oracle(gs):
    """Per Gaussian, each parameter's gradient (a 3-vector for the mean, the
    SH block, ...) is compared as a whole against 1e-3 of its largest entry:
    a component that is small only because of the world axes' orientation
    carries the float32 error of the vector's large components."""
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.autograd import render

    scene = synth.scene_clustered(3000, seed=5, sh_degree=2)
    cam = synth.ring_cameras(4, 160, 96)[1]
    W, H = cam.width, cam.height
    plan = api.Plan(scene.n, scene.sh_degree, [(W, H)], 1 << 20)
    params = _leaf_params(scene)
    rgb, disp, T = render(params, plan, [cam], BG)
    rec = opre.pack_for_render(opre.project(opre.params_from_scene(scene), cam, scene.sh_degree))
    g, gd = synth.upstream_grads(21, W, H)
    loss = (rgb * torch.from_numpy(g.reshape(-1)).cuda()).sum() + (disp * torch.from_numpy(gd.reshape(-1)).cuda()).sum()
    loss.backward()
    ref2d, slack = oren.render_bwd(rec, BG, (0, 0, W, H), g.astype(np.float64), gd.astype(np.float64),
                                   amb=oren.float32_bands(), with_slack=True)
    ref = opre.preprocess_backward(scene, cam, ref2d)
    slack_p = opre.preprocess_backward_abs(scene, cam, slack)
    from paper_2601_19489_gb300 import _lib as L

    g2d = to_np(plan.view(L.GS_WS_GRAD2D, torch.float32)).reshape(-1, 12)
    gpu10 = g2d[:, [0, 1, 2, 3, 4, 5, 8, 9, 10, 6]]
    for name, t in zip(NAMES, params.tensors()):
        got = to_np(t.grad)
        bad = block_mismatch(got.reshape(got.shape[0], -1), ref[name].reshape(got.shape[0], -1),
                             slack=slack_p[name].reshape(got.shape[0], -1))
        rows = np.nonzero(bad)[0][:4]
        assert bad.sum() == 0, (name, int(bad.sum()), rows, got[rows], ref[name][rows],
                                np.abs(ref[name]).max(), gpu10[rows], ref2d[rows])


def test_autograd_gradient_matches_finite_differences(gs):
    """Central differences of the CUDA forward in float32 (h = 1e-4) on a
    six-Gaussian scene: agreement to 2e-2 of each gradient's scale, the
    accuracy float32 differences of this size allow.  A perturbation that
    moves a pixel across the 1/255 cut-off or the transmittance stop makes
    the loss jump (by about 1/255 of a pixel's weight); such an element shows
    as a disagreement between the differences at h and 2h and is left out
    (at most a quarter of them)."""
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.autograd import render

    cam = synth.camera_tiny(16, 16)
    scene = synth.scene_tiny(6, seed=32, sh_degree=1)
    plan = api.Plan(scene.n, scene.sh_degree, [(16, 16)], 1 << 12)
    rng = np.random.default_rng(2)
    w = torch.from_numpy(rng.uniform(0.5, 1.5, size=3 * 256).astype(np.float32)).cuda()
    wd = torch.from_numpy(rng.uniform(0.5, 1.5, size=256).astype(np.float32)).cuda()
    params = _leaf_params(scene)
    rgb, disp, _ = render(params, plan, [cam], BG)
    ((rgb * w).sum() + (disp * wd).sum()).backward()

    def L(p):
        with torch.no_grad():
            r, d, _ = render(p, plan, [cam], BG)
            return float(((r.double() * w.double()).sum() + (d.double() * wd.double()).sum()).item())

    base = api.Gaussians(*(t.detach().clone() for t in params.tensors()), params.sh_degree)
    h = 1e-4
    for name, t in zip(NAMES, params.tensors()):
        arr = getattr(base, name)
        flat = arr.view(-1)
        fd = np.zeros((2, flat.numel()))
        for i in range(flat.numel()):
            old = float(flat[i])
            for j, hh in enumerate((h, 2 * h)):
                flat[i] = old + hh
                fp = L(base)
                flat[i] = old - hh
                fm = L(base)
                flat[i] = old
                fd[j, i] = (fp - fm) / (2 * hh)
        got = to_np(t.grad).reshape(-1)
        scale = max(np.abs(fd[0]).max(), 1e-6)
        smooth = np.abs(fd[0] - fd[1]) <= 1e-2 * scale
        assert smooth.mean() >= 0.75, (name, smooth.mean())
        err = np.abs(got - fd[0])[smooth]
        assert np.all(err <= 2e-2 * scale), (name, err.max(), scale)
