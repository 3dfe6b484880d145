"""Three whole training steps of the CUDA path (preprocess through the fused
Adam update, one view per step) against three steps of the oracle's
training loop, on the small parity configuration (4096 Gaussians, 256 x 256):
the parameters after each step agree; after the first step, every element
whose gradient is not within the tolerance of zero took exactly the oracle's
step."""
import numpy as np
import pytest
import torch

import synth
from oracle import step as ostep
from tests.parity import to_np

pytestmark = pytest.mark.gpu


def test_three_training_steps_match_the_oracle(gs):
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer, default_lrs

    scene = synth.scene_c1(0)
    cam = synth.camera_c1()
    # a target beyond every rendered value keeps the L1 term off its kink
    target = np.random.default_rng(3).uniform(2.0, 2.5, size=(3, 256, 256))
    lrs = default_lrs(2.0)
    tr = Trainer(api.Gaussians.from_scene(scene), 256, 256, lam=0.2, lrs=lrs)
    tgt = torch.from_numpy(target.reshape(-1).astype(np.float32)).cuda()
    st = ostep.new_state(synth.Scene(*(a.astype(np.float64) for a in scene.arrays()), sh_degree=0))
    for it in range(1, 4):
        tr.step([cam], tgt)
        L_ref, g_ref, _ = ostep.train_step(st, scene, cam, target, lrs, lam=0.2)
        torch.cuda.synchronize()
        np.testing.assert_allclose(tr.loss.item(), L_ref, rtol=1e-4)
        ref = dict(st["params"])
        ref["sh"] = np.concatenate([ref.pop("sh_dc"), ref.pop("sh_rest")], axis=1)
        rate = {"means": lrs["means"], "log_scales": lrs["log_scales"], "quats": lrs["quats"],
                "opacity_logits": lrs["opacity_logits"], "sh": lrs["sh_dc"]}
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            got = to_np(getattr(tr.params, k)).reshape(ref[k].shape)
            err = np.abs(got - ref[k])
            if it == 1:
                # Adam's first step moves an element by its rate times the
                # sign of its gradient: wherever the oracle's gradient is not
                # within the gradient tolerance of zero (1e-3 of the tensor's
                # largest), the GPU must take the same step, to the float32
                # rounding of the parameter
                g = np.abs(g_ref[k]).reshape(ref[k].shape)
                decisive = g > 1e-3 * g.max()
                ulp = np.spacing(np.abs(ref[k]).astype(np.float32)).astype(np.float64)
                bad = decisive & (err > 2.0 * ulp + 1e-6 * rate[k])
                assert decisive.sum() >= 100, (k, int(decisive.sum()))
                assert not bad.any(), (k, int(bad.sum()), float(err[bad].max()) if bad.any() else 0.0)
            # An Adam step moves a parameter by at most about its rate, and by
            # a ratio of its gradients: where successive gradients nearly
            # cancel (or one is a few float32 ulps), float32 noise moves that
            # ratio a lot.  So: every element within two rates per step, the
            # typical one within 1e-3 of a rate, and few beyond 1e-2 of one.
            assert err.max() <= 2.0 * rate[k] * it, (k, it, err.max())
            assert np.median(err) <= 1e-3 * rate[k], (k, it, np.median(err))
            off = err > 1e-2 * rate[k] * it
            assert off.mean() < 0.02, (k, it, off.mean())
    assert tr.plan.status()["rc"] == 0
