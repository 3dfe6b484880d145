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


def test_trained_decoder_gains_over_a_frozen_one_at_equal_wall_time(gs):
    """What the trained network gains (Sec. 2.3): the decoder maps an anchor's
    feature and the view direction to its children, so a trained decoder can
    give them view-dependent appearance.  On a ground truth whose colour
    depends on the view (SH degree 3, higher coefficients N(0, 0.4)) the
    neural-Gaussian model is trained for a fixed wall time against the same
    anchors and children with the decoder's MLP frozen at its
    initialisation (features and anchor scales still trained); held-out PSNR
    decides.  Explicit 3DGS from the same starting points (DC colour only,
    like the decoded children) runs beside them and is printed."""
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.recon import reconstruct, render_views
    from paper_2601_19489_gb300.trainer import Trainer

    W, H = 320, 212
    gt = synth.scene_clustered(20000, seed=100, sh_degree=3, rest_std=0.4)
    cams = synth.orbit_cameras(48, W, H)
    gt_tr = Trainer(api.Gaussians.from_scene(gt), W, H)
    gt_tr.ensure_capacity([[c] for c in cams])
    views = render_views(gt_tr, cams)
    del gt_tr
    ev = [i for i in range(48) if i % 6 == 0]
    tr_ix = [i for i in range(48) if i % 6 != 0]
    init = synth.recon_init(gt, 4000, seed=1, sh_degree=0)
    res = {}
    for method in ("ng", "ng_frozen", "plain"):
        res[method] = reconstruct(method, init, [cams[i] for i in tr_ix], [views[i][0] for i in tr_ix],
                                  [views[i][1] for i in tr_ix], [cams[i] for i in ev], [views[i][0] for i in ev],
                                  budget_s=8.0, eval_every_s=4.0)
    torch.cuda.synchronize()
    print({m: (round(r["psnr_final"], 2), r["steps"]) for m, r in res.items()})
    assert res["ng"]["psnr_final"] > res["ng_frozen"]["psnr_final"] + 0.2, res
