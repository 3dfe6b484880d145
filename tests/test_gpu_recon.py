"""The timed reconstruction harness on a small scene: every method raises
the held-out PSNR within a few seconds of training."""
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", ["plain", "densify", "batched_graph", "ng"])
def test_short_reconstruction_improves_heldout_psnr(gs, method):
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.recon import reconstruct, render_views
    from paper_2601_19489_gb300.trainer import Trainer

    W, H = 320, 212
    gt = synth.scene_clustered(20000, seed=100, sh_degree=1)
    cams = synth.orbit_cameras(24, W, H)
    gt_tr = Trainer(api.Gaussians.from_scene(gt), W, H)
    gt_tr.ensure_capacity([[c] for c in cams])
    views = render_views(gt_tr, cams)
    del gt_tr
    ev = [i for i in range(24) if i % 6 == 0]
    tr_ix = [i for i in range(24) if i % 6 != 0]
    init = synth.recon_init(gt, 4000, seed=1, sh_degree=1)
    r = reconstruct(method, init, [cams[i] for i in tr_ix], [views[i][0] for i in tr_ix],
                    [views[i][1] for i in tr_ix], [cams[i] for i in ev], [views[i][0] for i in ev],
                    budget_s=3.0, eval_every_s=1.0)
    torch.cuda.synchronize()
    assert len(r["curve"]) == 4 and r["steps"] > 0
    assert r["psnr_final"] > r["psnr_start"] + 0.5, r["curve"]
