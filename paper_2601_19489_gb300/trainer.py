"""The 3DGS training step through the C ABI: preprocess -> bin/sort ->
forward blend -> loss -> per-Gaussian backward (+ preprocess backward) ->
Adam, all enqueued on one CUDA stream with no host synchronisation.

A step takes one view or a batch of views of uneven resolution; a batch goes
through every stage as one launch (the plan lays the views' tiles and pixels
end to end), its gradients sum over the views, and one Adam update follows.
The Adam step count lives on the device, so a step can be captured once in a
CUDA graph (``Trainer.capture``) and replayed.

With ``pose`` set, the global pose refinement of Sec. 2.5 runs alongside: one
camera-side correction shared by every view (training and evaluation), its
gradient accumulated by every step's preprocess backward and applied by an
Adam step every ``every`` steps (300 in the paper).

Learning rates default to the 3DGS values the paper trains with (its Sec. 4
builds on 3DGS and names no optimiser settings); SH DC coefficients and the
higher SH coefficients get different rates inside one Adam group.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .api import (Gaussians, NgParams, Plan, PoseState, adam_groups_array, adam_hparams, camera_struct,
                  gs_densify_apply, gs_densify_plan, gs_densify_score, gs_densify_scratch, gs_ng_workspace,
                  gs_pose_step, ng_children, pose_hparams)


def default_lrs(extent: float = 1.0) -> dict:
    return {"means": 1.6e-4 * extent, "log_scales": 5e-3, "quats": 1e-3, "opacity_logits": 0.05,
            "sh_dc": 2.5e-3, "sh_rest": 2.5e-3 / 20.0}


def default_pose(extent: float = 1.0) -> dict:
    """Pose-refinement settings: an update every 300 steps (Sec. 2.5); the
    paper gives no rates, these move the correction by at most about 1 mrad
    and 0.1 % of the scene extent per update."""
    return {"every": 300, "lr_rot": 1e-3, "lr_trans": 1e-3 * extent}


def _as_list(cams):
    return list(cams) if isinstance(cams, (list, tuple)) else [cams]


class _Slot:
    """Plan and image buffers for one tuple of view sizes."""

    def __init__(self, params: Gaussians, sizes, cap: int, device, tuning=None):
        self.sizes = sizes
        self.plan = Plan(params.n, params.sh_degree, list(sizes), cap, device=device, tuning=tuning)
        P = self.plan.pixels
        self.rgb = torch.empty(3 * P, device=device)
        self.disp = torch.empty(P, device=device)
        self.T = torch.empty(P, device=device)
        self.dL_drgb = torch.empty(3 * P, device=device)
        self.dL_ddisp = torch.empty(P, device=device)
        self.scratch = torch.empty(int(L.lib().gs_loss_scratch_floats(self.plan.handle)), device=device)


class Trainer:
    """Explicit-3DGS trainer.  ``Trainer(params, W, H)`` prepares single views
    of W x H; other sizes and batches get their own plan on first use (or in
    ``ensure_capacity``, which should see every batch before timing or
    capture)."""

    STAGES_UNFUSED = ("preprocess", "bin_sort", "render_fwd", "loss", "render_bwd_blend", "preprocess_bwd",
                      "adam")
    STAGES_FUSED = ("preprocess", "bin_sort", "render_fwd", "loss", "render_bwd_blend", "preprocess_bwd_adam")

    def __init__(self, params: Gaussians, width: int | None = None, height: int | None = None, *,
                 lam: float = 0.2, bg=(0.0, 0.0, 0.0), lrs: dict | None = None,
                 inst_capacity: int | None = None, load_balanced: bool = True, disp_weight: float = 0.0,
                 tuning: dict | None = None, fused_adam: bool = True, pose: dict | None = None,
                 visible_adam: bool = False, betas=(0.9, 0.999), device="cuda"):
        """tuning: launch shapes of the plans ({"bucket": 32 | 64,
        "bwd_warps": 2 | 4 | 8}), e.g. from autotune.autotune.
        fused_adam: apply Adam inside the preprocess backward
        (gs_preprocess_bwd_adam) instead of storing the gradient and running
        a separate Adam pass; self.grads then stays zero.
        visible_adam: with fused_adam, the sparse Adam that updates only the
        Gaussians that touched a tile in the step's views (the others keep
        their parameters and moments).
        pose: enable the global pose refinement ({"every", "lr_rot",
        "lr_trans"}, missing keys from default_pose()); the correction is in
        self.pose (a PoseState) and applies to every view this trainer
        renders.
        betas: Adam's (beta1, beta2)."""
        self.params = params
        self.fused_adam = bool(fused_adam)
        self.visible_adam = bool(visible_adam)
        if self.visible_adam and not self.fused_adam:
            raise ValueError("visible-only Adam runs inside the fused preprocess backward")
        self.STAGES = self.STAGES_FUSED if self.fused_adam else self.STAGES_UNFUSED
        self.tuning = dict(tuning or {})
        self.betas = (float(betas[0]), float(betas[1]))
        self.grads = params.zeros_like()
        self.lam = float(lam)
        self.disp_weight = float(disp_weight)
        self.bg = tuple(float(b) for b in bg)
        self.lrs = dict(lrs or default_lrs())
        self.load_balanced = bool(load_balanced)
        self.device = device
        self.step_count = 0
        self.d_step = torch.zeros(1, dtype=torch.int32, device=device)
        self.loss = torch.zeros(1, device=device)
        self.cap = int(inst_capacity) if inst_capacity is not None else max(1 << 20, 16 * params.n)
        self._bg = (ctypes.c_float * 3)(*self.bg)
        self.pose_cfg = None
        self.pose = None
        self._capturing = False
        if pose is not None:
            self.pose_cfg = {**default_pose(), **pose}
            self.pose = PoseState(device)
            self._pose_hp = pose_hparams(self.pose_cfg["lr_rot"], self.pose_cfg["lr_trans"])
        self._slots: dict = {}
        self._default = None
        if width is not None:
            self._default = self._slot(((int(width), int(height)),))
        self._build_adam()
        self._cam_cache = {}

    # ------------------------------------------------------------ set-up
    def _slot(self, sizes) -> _Slot:
        s = self._slots.get(sizes)
        if s is None:
            s = _Slot(self.params, sizes, self.cap, self.device, self.tuning)
            if self.pose is not None:
                s.plan.set_pose(self.pose)
            self._slots[sizes] = s
        return s

    @property
    def plan(self) -> Plan:
        return self._default.plan

    @property
    def rgb(self):
        return self._default.rgb

    @property
    def disp(self):
        return self._default.disp

    @property
    def T(self):
        return self._default.T

    def slot_for(self, cams) -> _Slot:
        return self._slot(tuple((int(c.width), int(c.height)) for c in _as_list(cams)))

    def _build_adam(self) -> None:
        if not hasattr(self, "m"):
            self.m = self.params.zeros_like()
            self.v = self.params.zeros_like()
        K = (self.params.sh_degree + 1) ** 2
        p, g, m, v = self.params, self.grads, self.m, self.v
        groups = []
        for name in ("means", "log_scales", "quats", "opacity_logits"):
            groups.append({"p": getattr(p, name), "g": getattr(g, name), "m": getattr(m, name),
                           "v": getattr(v, name), "lr": self.lrs[name]})
        groups.append({"p": p.sh, "g": g.sh, "m": m.sh, "v": v.sh, "lr": self.lrs["sh_rest"],
                       "period": 3 * K, "head": 3, "lr_head": self.lrs["sh_dc"]})
        self._adam = adam_groups_array(groups)
        self._hp = adam_hparams(self.lrs, b1=self.betas[0], b2=self.betas[1],
                                visible_only=getattr(self, "visible_adam", False))
        self._pstruct = p.struct()
        self._gstruct = g.struct()
        self._mstruct = m.struct()
        self._vstruct = v.struct()

    def set_lr(self, name: str, lr: float) -> None:
        """Change one learning rate (takes effect for eager steps; a captured
        graph keeps the rates it was captured with)."""
        self.lrs[name] = float(lr)
        self._build_adam()

    def set_pose_lr(self, lr_rot: float, lr_trans: float) -> None:
        """Change the pose-refinement rates (for the following updates)."""
        self.pose_cfg.update(lr_rot=float(lr_rot), lr_trans=float(lr_trans))
        self._pose_hp = pose_hparams(self.pose_cfg["lr_rot"], self.pose_cfg["lr_trans"])

    def _pose_tick(self, s) -> None:
        """After a step: every `every` steps, fold the accumulated pose
        gradient into the correction (one launch, on the step's stream)."""
        if self.pose is not None and not self._capturing and self.step_count % self.pose_cfg["every"] == 0:
            L.check(L.lib().gs_pose_step(self.pose.buf.data_ptr(), ctypes.byref(self._pose_hp), s),
                    "gs_pose_step")

    def _cam(self, cams):
        cams = _as_list(cams)
        key = tuple(id(c) for c in cams)
        c = self._cam_cache.get(key)
        if c is None:
            arr = (L.GsCamera * len(cams))(*[camera_struct(x) for x in cams])
            self._cam_cache[key] = (arr, cams)
            return arr
        return c[0]

    def ensure_capacity(self, batches, slack: float = 1.25) -> int:
        """Bin every camera or batch once and grow the instance capacity to
        fit the largest with `slack` to spare (all plans are rebuilt then).
        Synchronises; call outside timed regions and before any capture.
        Returns the largest instance count seen."""
        worst = 0
        for cams in batches:
            self.forward(cams)
            st = self.slot_for(cams).plan.status()
            if st["error"]:
                raise L.GsError(st["error"], "device status")
            worst = max(worst, st["n_instances"])
        if worst * slack > self.cap:
            self.cap = int(worst * slack) + 1024
            sizes = list(self._slots)
            default = self._default.sizes if self._default is not None else None
            self._slots = {}
            for sz in sizes:
                self._slot(sz)
            if default is not None:
                self._default = self._slots[default]
        return worst

    # ------------------------------------------------------------ step
    def forward(self, cams, stream=None) -> _Slot:
        lib = L.lib()
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        sl = self.slot_for(cams)
        h, ws = sl.plan.handle, sl.plan.ws.data_ptr()
        c = self._cam(cams)
        L.check(lib.gs_preprocess(h, ws, ctypes.byref(self._pstruct), c, s), "gs_preprocess")
        L.check(lib.gs_bin_sort(h, ws, int(self.load_balanced), s), "gs_bin_sort")
        L.check(lib.gs_render_fwd(h, ws, self._bg, sl.rgb.data_ptr(), sl.disp.data_ptr(), sl.T.data_ptr(), s),
                "gs_render_fwd")
        return sl

    def step(self, cams, target: torch.Tensor, target_disp: torch.Tensor | None = None, stream=None,
             events=None) -> None:
        """One full training step on a view or a batch of views against
        `target` (flat planar colour, the views end to end, float32 on the
        device) and optionally `target_disp` (disparity, weighted by
        disp_weight).  The loss lands in self.loss.

        events: optional list of len(STAGES) + 1 CUDA events recorded on the
        stream around the stages, for per-stage timing."""
        st = stream if stream is not None else torch.cuda.current_stream()
        s = st.cuda_stream
        ev = (lambda i: events[i].record(st)) if events is not None else (lambda i: None)
        ev(0)
        self.step_count += 1
        if self.fused_adam:
            self._splat_stages(cams, target, target_disp, s, ev, 1, with_pbwd=False)
            sl = self.slot_for(cams)
            L.check(L.lib().gs_preprocess_bwd_adam(sl.plan.handle, sl.plan.ws.data_ptr(), ctypes.byref(self._pstruct),
                                                   self._cam(cams), ctypes.byref(self._mstruct),
                                                   ctypes.byref(self._vstruct), ctypes.byref(self._hp),
                                                   self.d_step.data_ptr(), s), "gs_preprocess_bwd_adam")
            ev(6)
            self._pose_tick(s)
            return
        self._splat_stages(cams, target, target_disp, s, ev, 1)
        L.check(L.lib().gs_adam_step_multi_dev(self._adam, len(self._adam), self.betas[0], self.betas[1], 1e-15,
                                               self.d_step.data_ptr(), s), "gs_adam_step_multi_dev")
        ev(7)
        self._pose_tick(s)

    def _splat_stages(self, cams, target, target_disp, s, ev, e0: int, with_pbwd: bool = True,
                      with_pre: bool = True) -> None:
        """preprocess .. preprocess backward of self.params on `cams`; the
        parameter gradients accumulate into self.grads.  Records events
        e0 .. e0 + 5 after each stage (without the preprocess backward:
        stops after the blend backward, e0 + 4).  with_pre=False: the
        preprocess already ran (fused into the neural-Gaussian decode)."""
        lib = L.lib()
        sl = self.slot_for(cams)
        h, ws = sl.plan.handle, sl.plan.ws.data_ptr()
        c = self._cam(cams)
        use_disp = target_disp is not None and self.disp_weight > 0.0
        if with_pre:
            L.check(lib.gs_preprocess(h, ws, ctypes.byref(self._pstruct), c, s), "gs_preprocess")
        ev(e0)
        L.check(lib.gs_bin_sort(h, ws, int(self.load_balanced), s), "gs_bin_sort")
        ev(e0 + 1)
        L.check(lib.gs_render_fwd(h, ws, self._bg, sl.rgb.data_ptr(), sl.disp.data_ptr(), sl.T.data_ptr(), s),
                "gs_render_fwd")
        ev(e0 + 2)
        L.check(lib.gs_loss(h, sl.rgb.data_ptr(), target.data_ptr(), self.lam,
                            sl.disp.data_ptr() if use_disp else None,
                            target_disp.data_ptr() if use_disp else None, self.disp_weight if use_disp else 0.0,
                            sl.dL_drgb.data_ptr(), sl.dL_ddisp.data_ptr() if use_disp else None,
                            self.loss.data_ptr(), sl.scratch.data_ptr(), s), "gs_loss")
        ev(e0 + 3)
        L.check(lib.gs_render_bwd_blend(h, ws, sl.rgb.data_ptr(), sl.disp.data_ptr(), sl.dL_drgb.data_ptr(),
                                        sl.dL_ddisp.data_ptr() if use_disp else None, s), "gs_render_bwd_blend")
        ev(e0 + 4)
        if not with_pbwd:
            return
        L.check(lib.gs_preprocess_bwd(h, ws, ctypes.byref(self._pstruct), c, ctypes.byref(self._gstruct), s),
                "gs_preprocess_bwd")
        ev(e0 + 5)

    # ------------------------------------------------------------ densify
    def densify(self, cams, targets, tau: float = 0.3, rules: dict | None = None, seed: int = 0,
                max_gaussians: int | None = None) -> dict:
        """One densify-and-prune stage (Sec. 3.2): score every Gaussian on the
        given views (single-view forwards against their targets, flat planar
        colour on the device), then clone, split or prune it by the rules and
        rebuild the parameter set with its Adam moments.  Plans are rebuilt
        for the new count; captured graphs must be captured again.
        rules: tau_plus, tau_minus, min_opacity, percent_dense, extent.
        max_gaussians: if the result would exceed it, no Gaussian is added
        (pruning still happens).  Returns before / after counts and actions."""
        import numpy as np

        lib = L.lib()
        r = {"tau_plus": 5.0, "tau_minus": 0.95, "min_opacity": 0.005, "percent_dense": 0.01, "extent": 4.4}
        r.update(rules or {})
        r["k_views"] = len(cams)
        n = self.params.n
        dev = self.params.means.device
        s_plus = torch.zeros(n, device=dev)
        r_minus = torch.zeros(n, device=dev)
        scratch = gs_densify_scratch(n, device=dev)
        photo = torch.zeros(1, device=dev)
        for cam, tgt in zip(cams, targets):
            sl = self.forward([cam])
            s = torch.cuda.current_stream().cuda_stream
            L.check(lib.gs_loss(sl.plan.handle, sl.rgb.data_ptr(), tgt.data_ptr(), self.lam, None, None, 0.0,
                                sl.dL_drgb.data_ptr(), None, photo.data_ptr(), sl.scratch.data_ptr(), s), "gs_loss")
            gs_densify_score(sl.plan, sl.rgb, tgt, tau, photo, s_plus, r_minus, scratch)
        action = torch.empty(n, dtype=torch.int32, device=dev)
        offsets = torch.empty(n, dtype=torch.int64, device=dev)
        new_n = gs_densify_plan(self.params, s_plus, r_minus, r, action, offsets, scratch)
        if max_gaussians is not None and new_n > max_gaussians:
            r_capped = dict(r, tau_plus=float("inf"))
            new_n = gs_densify_plan(self.params, s_plus, r_minus, r_capped, action, offsets, scratch)
        counts = torch.bincount(action.long(), minlength=4).tolist()
        if new_n == n and counts[L.GS_DENSIFY_KEEP] == n:
            return {"n_before": n, "n_after": n, "prune": 0, "clone": 0, "split": 0}
        rng = np.random.default_rng(seed)
        normals = torch.from_numpy(rng.standard_normal((n, 2, 3)).astype(np.float32)).to(dev)
        like = lambda: Gaussians(*(torch.empty((new_n,) + tuple(x.shape[1:]), device=dev)
                                   for x in self.params.tensors()), self.params.sh_degree)
        dst, dm, dv = like(), like(), like()
        gs_densify_apply(self.params, self.m, self.v, action, offsets, normals, dst, dm, dv)
        self.params, self.m, self.v = dst, dm, dv
        self.grads = dst.zeros_like()
        self.cap = max(self.cap, 16 * new_n)
        sizes = list(self._slots)
        default = self._default.sizes if self._default is not None else None
        self._slots = {}
        for sz in sizes:
            self._slot(sz)
        if default is not None:
            self._default = self._slots[default]
        self._build_adam()
        return {"n_before": n, "n_after": new_n, "prune": counts[L.GS_DENSIFY_PRUNE],
                "clone": counts[L.GS_DENSIFY_CLONE], "split": counts[L.GS_DENSIFY_SPLIT]}

    # ------------------------------------------------------------ checkpoint
    def _state_tensors(self) -> dict:
        out = {}
        for group, g in (("params", self.params), ("m", self.m), ("v", self.v)):
            for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
                out[f"{group}.{name}"] = getattr(g, name)
        return out

    def state_dict(self) -> dict:
        """Everything a resumed run needs: parameters, Adam moments and step
        count (host copies), learning rates and loss settings."""
        st = {k: v.detach().cpu().clone() for k, v in self._state_tensors().items()}
        st["d_step"] = int(self.d_step.item())
        st["step_count"] = self.step_count
        st["lrs"] = dict(self.lrs)
        st["lam"], st["disp_weight"] = self.lam, self.disp_weight
        if self.pose is not None:
            st["pose"] = self.pose.buf.detach().cpu().clone()
            st["pose_cfg"] = dict(self.pose_cfg)
        return st

    def load_state_dict(self, st: dict) -> None:
        """Copy a state_dict in place: the device buffers keep their
        addresses, so captured graphs stay valid."""
        for k, v in self._state_tensors().items():
            if st[k].shape != v.shape:
                raise ValueError(f"{k}: shape {tuple(st[k].shape)} != {tuple(v.shape)}")
            v.data.copy_(st[k].to(v.device))
        self.d_step.fill_(int(st["d_step"]))
        self.step_count = int(st["step_count"])
        self.lam, self.disp_weight = float(st["lam"]), float(st["disp_weight"])
        self.lrs = dict(st["lrs"])
        if self.pose is not None and "pose" in st:
            self.pose.buf.copy_(st["pose"].to(self.pose.buf.device))
            self.set_pose_lr(st["pose_cfg"]["lr_rot"], st["pose_cfg"]["lr_trans"])
            self.pose_cfg["every"] = int(st["pose_cfg"]["every"])
        self._build_adam()

    def save(self, path: str) -> None:
        torch.save(self.state_dict(), path)

    def load(self, path: str) -> None:
        self.load_state_dict(torch.load(path, map_location="cpu", weights_only=False))

    def capture(self, cams, target: torch.Tensor, target_disp: torch.Tensor | None = None) -> "StepGraph":
        """Capture one training step on `cams` into a CUDA graph.  The graph
        reads the parameters, the optimiser state and `target` (and
        `target_disp`) in place, so refilling those tensors between replays
        is seen; the cameras, learning rates and buffer addresses are fixed
        at capture.  Call ensure_capacity (and one eager step) first."""
        return StepGraph(self, cams, target, target_disp)


class HostFeeder:
    """Per-step inputs that live in pinned host memory, fed to the device
    with the copy of step i+1's input running on a side stream while step i
    computes (two device buffers, events between the streams).

        feeder = HostFeeder(like=device_tensor_of_the_input_shape)
        for i in ...:
            x = feeder.get(host[i], host[i + 1] if more else None)
            trainer.step(cams[i], x)
            feeder.done()
    """

    def __init__(self, like: torch.Tensor):
        self.buf = [torch.empty_like(like), torch.empty_like(like)]
        self.stream = torch.cuda.Stream(like.device)
        self.ready = [torch.cuda.Event(), torch.cuda.Event()]
        self.free = [torch.cuda.Event(), torch.cuda.Event()]
        self.slot = 0
        self.primed = False

    def _copy(self, slot: int, host: torch.Tensor) -> None:
        self.stream.wait_event(self.free[slot])  # the buffer's previous step is done with it
        with torch.cuda.stream(self.stream):
            self.buf[slot].copy_(host, non_blocking=True)
            self.ready[slot].record(self.stream)

    def get(self, host_now: torch.Tensor, host_next: torch.Tensor | None = None) -> torch.Tensor:
        """The device copy of host_now for this step (prefetched by the
        previous call when it was given as host_next); starts copying
        host_next."""
        slot = self.slot
        if not self.primed:
            self._copy(slot, host_now)
        torch.cuda.current_stream().wait_event(self.ready[slot])
        self.primed = host_next is not None
        if self.primed:
            self._copy(1 - slot, host_next)
        self.slot = 1 - slot
        return self.buf[slot]

    def done(self) -> None:
        """Mark the buffer of the last get() free once the work enqueued so
        far on the current stream (the step that read it) has run."""
        self.free[1 - self.slot].record(torch.cuda.current_stream())


class StepGraph:
    """A captured training step; ``replay()`` enqueues the whole step (every
    launch of it) as one graph launch on the current stream."""

    def __init__(self, trainer: Trainer, cams, target, target_disp=None):
        self.trainer = trainer
        self.cams = _as_list(cams)
        trainer.slot_for(self.cams)  # plan and buffers exist before capture
        trainer._cam(self.cams)
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        trainer._capturing = True  # the periodic pose update stays out of the graph
        try:
            with torch.cuda.graph(self.graph, stream=side):
                trainer.step(self.cams, target, target_disp)
        finally:
            trainer._capturing = False
        trainer.step_count -= 1  # capture does not run the step
        torch.cuda.current_stream().wait_stream(side)

    def replay(self) -> None:
        self.graph.replay()
        self.trainer.step_count += 1
        self.trainer._pose_tick(torch.cuda.current_stream().cuda_stream)


def default_ng_lrs() -> dict:
    """Scaffold-GS style rates for the decoder (the paper gives none)."""
    return {"feat": 7.5e-3, "anchor_ls": 7e-3, "mlp": 4e-3}


class NgTrainer(Trainer):
    """Neural-Gaussian training step (Sec. 2.3) on one view: the decoder
    infers the anchors' child Gaussians for the view, the children go
    through the same splatting kernels as explicit 3DGS, and their gradients
    flow back through the decoder into the anchor features, the anchors'
    log-scales and the MLP, which one Adam update then trains.  The anchor
    positions stay fixed.  ng_lrs overrides the rates of default_ng_lrs()
    by name; {"anchor_ls": 0.0} trains only the features and the MLP, as
    Sec. 2.3 states."""

    NG_STAGES = ("decode", "preprocess", "bin_sort", "render_fwd", "loss", "render_bwd_blend", "preprocess_bwd",
                 "decode_bwd", "adam")

    def __init__(self, ng: NgParams, width: int | None = None, height: int | None = None, *,
                 ng_lrs: dict | None = None, fused_decode: bool = False, **kw):
        """fused_decode: decode and preprocess the children in one launch
        (gs_ng_decode_preprocess) in the training step; the results are the
        same bit for bit."""
        self.ng = ng
        self.fused_decode = bool(fused_decode)
        self.ng_grads = ng.zeros_like()
        self.ng_m = ng.zeros_like()
        self.ng_v = ng.zeros_like()
        self.ng_lrs = {**default_ng_lrs(), **(ng_lrs or {})}
        self.ng_ws = gs_ng_workspace(ng.n, device=kw.get("device", "cuda"))
        children = ng_children(ng.n, device=kw.get("device", "cuda"))
        kw.setdefault("inst_capacity", max(1 << 20, 16 * children.n))
        kw["fused_adam"] = False  # the children are decoded, not optimised
        if kw.get("pose") is not None:
            raise ValueError("pose refinement is not wired into the neural-Gaussian decoder's view direction")
        super().__init__(children, width, height, **kw)
        self.STAGES = NgTrainer.NG_STAGES
        self._ngp = ng.struct()
        self._ngg = self.ng_grads.struct()

    @property
    def children(self) -> Gaussians:
        return self.params

    def _state_tensors(self) -> dict:
        out = {}
        for group, g in (("ng", self.ng), ("m", self.ng_m), ("v", self.ng_v)):
            for name in ("anchor_xyz", "feat", "anchor_ls", "w1", "b1", "w2", "b2"):
                out[f"{group}.{name}"] = getattr(g, name)
        return out

    def load_state_dict(self, st: dict) -> None:
        super().load_state_dict(st)
        self._ngp = self.ng.struct()

    def _build_adam(self) -> None:
        groups = []
        for name, lr in (("feat", self.ng_lrs["feat"]), ("anchor_ls", self.ng_lrs["anchor_ls"]),
                         ("w1", self.ng_lrs["mlp"]), ("b1", self.ng_lrs["mlp"]), ("w2", self.ng_lrs["mlp"]),
                         ("b2", self.ng_lrs["mlp"])):
            groups.append({"p": getattr(self.ng, name), "g": getattr(self.ng_grads, name),
                           "m": getattr(self.ng_m, name), "v": getattr(self.ng_v, name), "lr": lr})
        self._adam = adam_groups_array(groups)
        self._pstruct = self.params.struct()
        self._gstruct = self.grads.struct()

    def _decode(self, cam, s) -> None:
        c = self._cam([cam])
        L.check(L.lib().gs_ng_decode_fwd(ctypes.byref(self._ngp), c, ctypes.byref(self._pstruct),
                                         self.ng_ws.data_ptr(), s), "gs_ng_decode_fwd")

    def forward(self, cams, stream=None):
        cam = _as_list(cams)
        if len(cam) != 1:
            raise ValueError("the neural-Gaussian step decodes for one view at a time")
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        self._decode(cam[0], s)
        return super().forward(cams, stream)

    def step(self, cams, target: torch.Tensor, target_disp: torch.Tensor | None = None, stream=None,
             events=None) -> None:
        cam = _as_list(cams)
        if len(cam) != 1:
            raise ValueError("the neural-Gaussian step decodes for one view at a time")
        st = stream if stream is not None else torch.cuda.current_stream()
        s = st.cuda_stream
        ev = (lambda i: events[i].record(st)) if events is not None else (lambda i: None)
        ev(0)
        if self.fused_decode:
            sl = self.slot_for(cam)
            L.check(L.lib().gs_ng_decode_preprocess(ctypes.byref(self._ngp), self._cam(cam), ctypes.byref(self._pstruct),
                                                    self.ng_ws.data_ptr(), sl.plan.handle, sl.plan.ws.data_ptr(), s),
                    "gs_ng_decode_preprocess")
        else:
            self._decode(cam[0], s)
        ev(1)
        self._splat_stages(cam, target, target_disp, s, ev, 2, with_pre=not self.fused_decode)
        c = self._cam(cam)
        L.check(L.lib().gs_ng_decode_bwd(ctypes.byref(self._ngp), c, ctypes.byref(self._gstruct), 1,
                                         ctypes.byref(self._ngg), self.ng_ws.data_ptr(), s), "gs_ng_decode_bwd")
        ev(8)
        self.step_count += 1
        L.check(L.lib().gs_adam_step_multi_dev(self._adam, len(self._adam), self.betas[0], self.betas[1], 1e-15,
                                               self.d_step.data_ptr(), s), "gs_adam_step_multi_dev")
        ev(9)

    def status(self) -> int:
        """Synchronise and return the decoder's device status (0 = ok)."""
        e = ctypes.c_int32(0)
        return int(L.lib().gs_ng_read_status(self.ng_ws.data_ptr(), ctypes.byref(e),
                                             torch.cuda.current_stream().cuda_stream))
