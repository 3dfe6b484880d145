"""One training step of 3DGS through the C ABI: preprocess -> bin/sort ->
forward blend -> loss -> per-Gaussian backward (+ preprocess backward) ->
Adam, all enqueued on one CUDA stream with no host synchronisation.

Learning rates default to the 3DGS values the paper trains with (its Sec. 4
builds on 3DGS and names no optimiser settings); SH DC coefficients and the
higher SH coefficients get different rates inside one Adam group.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .api import Gaussians, Plan, _stream, adam_groups_array, camera_struct


def default_lrs(extent: float = 1.0) -> dict:
    return {"means": 1.6e-4 * extent, "log_scales": 5e-3, "quats": 1e-3, "opacity_logits": 0.05,
            "sh_dc": 2.5e-3, "sh_rest": 2.5e-3 / 20.0}


class Trainer:
    """Explicit-3DGS trainer over views of one resolution (one view per step)."""

    def __init__(self, params: Gaussians, width: int, height: int, lam: float = 0.2,
                 bg=(0.0, 0.0, 0.0), lrs: dict | None = None, inst_capacity: int | None = None,
                 load_balanced: bool = True, device="cuda"):
        self.params = params
        self.grads = params.zeros_like()
        self.m = params.zeros_like()
        self.v = params.zeros_like()
        self.width, self.height = int(width), int(height)
        self.lam = float(lam)
        self.bg = tuple(float(b) for b in bg)
        self.lrs = dict(lrs or default_lrs())
        self.load_balanced = bool(load_balanced)
        self.device = device
        self.step_count = 0
        P = self.width * self.height
        self.rgb = torch.empty(3 * P, device=device)
        self.disp = torch.empty(P, device=device)
        self.T = torch.empty(P, device=device)
        self.dL_drgb = torch.empty(3 * P, device=device)
        self.loss = torch.zeros(1, device=device)
        cap = inst_capacity if inst_capacity is not None else max(1 << 20, 16 * params.n)
        self._make_plan(cap)
        self._bg = (ctypes.c_float * 3)(*self.bg)
        self._build_adam()
        self._cam_cache = {}

    # ------------------------------------------------------------ set-up
    def _make_plan(self, cap: int) -> None:
        self.plan = Plan(self.params.n, self.params.sh_degree, [(self.width, self.height)], cap,
                         device=self.device)
        self.scratch = torch.empty(int(L.lib().gs_loss_scratch_floats(self.plan.handle)),
                                   device=self.device)

    def _build_adam(self) -> None:
        K = (self.params.sh_degree + 1) ** 2
        p, g, m, v = self.params, self.grads, self.m, self.v
        groups = []
        for name in ("means", "log_scales", "quats", "opacity_logits"):
            groups.append({"p": getattr(p, name), "g": getattr(g, name), "m": getattr(m, name),
                           "v": getattr(v, name), "lr": self.lrs[name]})
        groups.append({"p": p.sh, "g": g.sh, "m": m.sh, "v": v.sh, "lr": self.lrs["sh_rest"],
                       "period": 3 * K, "head": 3, "lr_head": self.lrs["sh_dc"]})
        self._adam = adam_groups_array(groups)
        self._pstruct = p.struct()
        self._gstruct = g.struct()

    def _cam(self, cam):
        key = id(cam)
        c = self._cam_cache.get(key)
        if c is None:
            c = (L.GsCamera * 1)(camera_struct(cam))
            self._cam_cache[key] = (c, cam)
            return c
        return c[0]

    def ensure_capacity(self, cams, slack: float = 1.25) -> int:
        """Bin every camera once and grow the instance capacity to fit the
        largest view with `slack` to spare.  Synchronises; call outside timed
        regions.  Returns the largest instance count seen."""
        worst = 0
        for cam in cams:
            self.forward(cam)
            st = self.plan.status()
            if st["error"]:
                raise L.GsError(st["error"], "device status")
            worst = max(worst, st["n_instances"])
        if worst * slack > self.plan.inst_capacity:
            self._make_plan(int(worst * slack) + 1024)
        return worst

    # ------------------------------------------------------------ step
    def forward(self, cam, stream=None) -> None:
        lib = L.lib()
        s = _stream(stream)
        ws = self.plan.ws.data_ptr()
        c = self._cam(cam)
        L.check(lib.gs_preprocess(self.plan.handle, ws, ctypes.byref(self._pstruct), c, s), "gs_preprocess")
        L.check(lib.gs_bin_sort(self.plan.handle, ws, int(self.load_balanced), s), "gs_bin_sort")
        L.check(lib.gs_render_fwd(self.plan.handle, ws, self._bg, self.rgb.data_ptr(), self.disp.data_ptr(),
                                  self.T.data_ptr(), s), "gs_render_fwd")

    STAGES = ("preprocess", "bin_sort", "render_fwd", "loss", "render_bwd_blend", "preprocess_bwd", "adam")

    def step(self, cam, target: torch.Tensor, stream=None, events=None) -> None:
        """One full training step on view `cam` against `target` (flat planar
        3*H*W float32 on the device).  The loss lands in self.loss.

        events: optional list of len(STAGES) + 1 CUDA events recorded on the
        stream around the stages, for per-stage timing."""
        lib = L.lib()
        st = stream if stream is not None else torch.cuda.current_stream()
        s = st.cuda_stream
        h = self.plan.handle
        ws = self.plan.ws.data_ptr()
        c = self._cam(cam)
        ev = (lambda i: events[i].record(st)) if events is not None else (lambda i: None)
        ev(0)
        L.check(lib.gs_preprocess(h, ws, ctypes.byref(self._pstruct), c, s), "gs_preprocess")
        ev(1)
        L.check(lib.gs_bin_sort(h, ws, int(self.load_balanced), s), "gs_bin_sort")
        ev(2)
        L.check(lib.gs_render_fwd(h, ws, self._bg, self.rgb.data_ptr(), self.disp.data_ptr(),
                                  self.T.data_ptr(), s), "gs_render_fwd")
        ev(3)
        L.check(lib.gs_loss(h, self.rgb.data_ptr(), target.data_ptr(), self.lam, None, None, 0.0,
                            self.dL_drgb.data_ptr(), None, self.loss.data_ptr(), self.scratch.data_ptr(), s),
                "gs_loss")
        ev(4)
        L.check(lib.gs_render_bwd_blend(h, ws, self.rgb.data_ptr(), self.disp.data_ptr(),
                                        self.dL_drgb.data_ptr(), None, s), "gs_render_bwd_blend")
        ev(5)
        L.check(lib.gs_preprocess_bwd(h, ws, ctypes.byref(self._pstruct), c, ctypes.byref(self._gstruct), s),
                "gs_preprocess_bwd")
        ev(6)
        self.step_count += 1
        L.check(lib.gs_adam_step_multi(self._adam, len(self._adam), 0.9, 0.999, 1e-15, self.step_count, s),
                "gs_adam_step_multi")
        ev(7)
