"""Checkpoint and resume of a training run: a run restored from a saved
state continues with the losses of the uninterrupted run."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_resume_continues_the_same_run(gs, tmp_path):
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer

    scene = synth.scene_clustered(5000, seed=3, sh_degree=1)
    cams = synth.ring_cameras(4, 128, 96)
    tgts = [torch.from_numpy(synth.target_uniform(50 + i, 128, 96).reshape(-1)).cuda() for i in range(4)]
    a = Trainer(api.Gaussians.from_scene(scene), 128, 96, inst_capacity=1 << 20)
    for i in range(3):
        a.step(cams[i % 4], tgts[i % 4])
    a.save(str(tmp_path / "ckpt.pt"))
    la = []
    for i in range(3, 8):
        a.step(cams[i % 4], tgts[i % 4])
        la.append(a.loss.item())
    b = Trainer(api.Gaussians.from_scene(synth.scene_clustered(5000, seed=4, sh_degree=1)), 128, 96,
                inst_capacity=1 << 20)
    b.load(str(tmp_path / "ckpt.pt"))
    assert b.step_count == 3 and int(b.d_step.item()) == 3
    lb = []
    for i in range(3, 8):
        b.step(cams[i % 4], tgts[i % 4])
        lb.append(b.loss.item())
    np.testing.assert_allclose(lb, la, rtol=1e-4)


def test_ng_resume(gs, tmp_path):
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import NgTrainer

    pts = synth.scene_clustered(8000, seed=2, sh_degree=0).means
    d = synth.ng_anchors(pts, 500, seed=2)
    cams = synth.ring_cameras(4, 128, 96)
    tgts = [torch.from_numpy(synth.target_uniform(70 + i, 128, 96).reshape(-1)).cuda() for i in range(4)]
    a = NgTrainer(api.NgParams.from_dict(d), 128, 96, inst_capacity=1 << 18)
    for i in range(3):
        a.step(cams[i % 4], tgts[i % 4])
    st = a.state_dict()
    la = []
    for i in range(3, 7):
        a.step(cams[i % 4], tgts[i % 4])
        la.append(a.loss.item())
    b = NgTrainer(api.NgParams.from_dict(synth.ng_anchors(pts, 500, seed=9)), 128, 96, inst_capacity=1 << 18)
    b.load_state_dict(st)
    lb = []
    for i in range(3, 7):
        b.step(cams[i % 4], tgts[i % 4])
        lb.append(b.loss.item())
    np.testing.assert_allclose(lb, la, rtol=1e-4)


def test_host_feeder_delivers_each_step_its_own_input(gs):
    """Prefetched host inputs arrive intact and in order: each step's loss
    equals the loss of the same step fed synchronously."""
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import HostFeeder, Trainer

    scene = synth.scene_clustered(3000, seed=6, sh_degree=0)
    cams = synth.ring_cameras(3, 96, 64)
    host = [torch.from_numpy(synth.target_uniform(90 + i, 96, 64).reshape(-1)).pin_memory() for i in range(3)]
    runs = []
    for prefetch in (False, True):
        tr = Trainer(api.Gaussians.from_scene(scene), 96, 64, inst_capacity=1 << 18)
        feeder = HostFeeder(host[0].cuda())
        dev = host[0].cuda()
        losses = []
        for s in range(9):
            if prefetch:
                x = feeder.get(host[s % 3], host[(s + 1) % 3] if s < 8 else None)
            else:
                dev.copy_(host[s % 3])
                x = dev
            tr.step(cams[s % 3], x)
            if prefetch:
                feeder.done()
            losses.append(tr.loss.item())
        runs.append(losses)
    np.testing.assert_allclose(runs[1], runs[0], rtol=1e-4)
