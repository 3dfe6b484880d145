"""Torch-facing wrappers of the C ABI (same names as include/gs.h).

PyTorch only provides device memory and streams here: each function checks
tensor placement, passes raw device pointers and the current CUDA stream to
libgs.so and raises GsError on a non-zero status.  No computation of the
training step happens in Python.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib as L


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: torch.Tensor | None, dtype=torch.float32) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def camera_struct(cam) -> L.GsCamera:
    """GsCamera from any object with fx, fy, cx, cy, w2c() (3x4), width,
    height and optional near."""
    c = L.GsCamera()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    w = cam.w2c().reshape(-1)
    for i in range(12):
        c.w2c[i] = float(w[i])
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_z = float(getattr(cam, "near", 0.2))
    return c


def cameras_array(cams) -> ctypes.Array:
    arr = (L.GsCamera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera_struct(c)
    return arr


@dataclass
class Gaussians:
    """Gaussian parameter arrays (float32, contiguous, one device)."""

    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    sh: torch.Tensor
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def tensors(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh)

    def struct(self) -> L.GsParams:
        p = L.GsParams()
        p.n = self.n
        p.sh_degree = self.sh_degree
        p.means, p.log_scales, p.quats, p.opacity_logits, p.sh = (_ptr(t) for t in self.tensors())
        return p

    def zeros_like(self) -> "Gaussians":
        return Gaussians(*(torch.zeros_like(t) for t in self.tensors()), sh_degree=self.sh_degree)

    @staticmethod
    def from_scene(scene, device="cuda") -> "Gaussians":
        t = lambda a: torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)
        return Gaussians(t(scene.means), t(scene.log_scales), t(scene.quats), t(scene.opacity_logits),
                         t(scene.sh), int(scene.sh_degree))


class Plan:
    """A gs_plan plus the device workspace it describes."""

    def __init__(self, n: int, sh_degree: int, sizes, inst_capacity: int, device="cuda",
                 tuning: dict | None = None):
        """tuning: optional {"bucket": 32 | 64, "bwd_warps": 1 | 2 | 4 | 8,
        "bwd_chains": 0 | 1 | 2, "bbox_3sigma": 0 | 1, "bwd_per_pixel": 0 | 1,
        "bin_radix": 0 | 1, "fwd_pixels": 1 | 2} (bbox_3sigma and
        bwd_per_pixel are the Tab. 1 ablation switches; bin_radix takes the
        key-write + radix-sort binning instead of the counting binning, same
        lists; fwd_pixels 2 blends two pixels per thread in packed pairs)."""
        lib = L.lib()
        self.sizes = [(int(w), int(h)) for (w, h) in sizes]
        V = len(self.sizes)
        ws_ = (ctypes.c_int32 * V)(*[w for w, _ in self.sizes])
        hs_ = (ctypes.c_int32 * V)(*[h for _, h in self.sizes])
        self.tuning = {"bucket": 64, "bwd_warps": 1, "bwd_chains": 0, "bbox_3sigma": 0, "bwd_per_pixel": 0,
                       "bin_radix": 0, "fwd_pixels": 2, **(tuning or {})}
        tu = L.GsTuning(*(int(self.tuning[k]) for k in ("bucket", "bwd_warps", "bwd_chains", "bbox_3sigma",
                                                        "bwd_per_pixel", "bin_radix", "fwd_pixels")))
        self.handle = lib.gs_plan_create_tuned(int(n), int(sh_degree), V, ws_, hs_, int(inst_capacity),
                                               ctypes.byref(tu))
        if not self.handle:
            raise L.GsError(L.GS_ERR_ARG, "gs_plan_create")
        self.n, self.sh_degree, self.inst_capacity = int(n), int(sh_degree), int(inst_capacity)
        self.bytes = int(lib.gs_plan_workspace_bytes(self.handle))
        self.pixels = int(lib.gs_plan_pixels(self.handle))
        self.ws = torch.empty(self.bytes, dtype=torch.uint8, device=device)
        self.ws.zero_()
        self.pose = None  # attached pose-refinement state (set_pose)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and L._lib is not None:
            L._lib.gs_plan_destroy(h)
            self.handle = None

    @property
    def n_views(self) -> int:
        return len(self.sizes)

    def image_shape(self):
        """(3 * total pixels,) is the flat colour layout; per view planar CHW."""
        return (3 * self.pixels,)

    def view(self, which: int, dtype=torch.uint8) -> torch.Tensor:
        """A tensor aliasing one workspace buffer (GS_WS_*)."""
        ptr = ctypes.c_void_p()
        nb = ctypes.c_size_t()
        L.check(L.lib().gs_workspace_view(self.handle, self.ws.data_ptr(), which, ctypes.byref(ptr),
                                          ctypes.byref(nb)), "gs_workspace_view")
        off = ptr.value - self.ws.data_ptr()
        return self.ws[off:off + nb.value].view(dtype)

    def set_pose(self, state: "PoseState | None") -> None:
        """Attach a pose-refinement state (gs_plan_set_pose); None detaches."""
        L.check(L.lib().gs_plan_set_pose(self.handle, state.buf.data_ptr() if state is not None else None),
                "gs_plan_set_pose")
        self.pose = state  # keeps the buffer alive while attached

    def status(self, stream=None) -> dict:
        st = L.GsStatus()
        rc = L.lib().gs_read_status(self.handle, self.ws.data_ptr(), ctypes.byref(st), _stream(stream))
        return {"rc": rc, "n_instances": st.n_instances, "n_buckets": st.n_buckets,
                "inst_capacity": st.inst_capacity, "overflow": st.overflow, "error": st.error}


# ---------------------------------------------------------------- the ABI

def gs_preprocess(plan: Plan, params: Gaussians, cams, stream=None) -> None:
    ca = cameras_array(cams)
    p = params.struct()
    L.check(L.lib().gs_preprocess(plan.handle, plan.ws.data_ptr(), ctypes.byref(p), ca, _stream(stream)),
            "gs_preprocess")


def gs_bin_sort(plan: Plan, load_balanced: bool = True, stream=None) -> None:
    L.check(L.lib().gs_bin_sort(plan.handle, plan.ws.data_ptr(), int(bool(load_balanced)), _stream(stream)),
            "gs_bin_sort")


def gs_render_fwd(plan: Plan, bg, out_rgb, out_disp, out_T, stream=None) -> None:
    bgc = (ctypes.c_float * 3)(*[float(b) for b in bg])
    L.check(L.lib().gs_render_fwd(plan.handle, plan.ws.data_ptr(), bgc, _ptr(out_rgb), _ptr(out_disp),
                                  _ptr(out_T), _stream(stream)), "gs_render_fwd")


def gs_render_bwd(plan: Plan, params: Gaussians, cams, bg, rgb, disp, dL_drgb, dL_ddisp,
                  grads: Gaussians, stream=None) -> None:
    ca = cameras_array(cams)
    bgc = (ctypes.c_float * 3)(*[float(b) for b in bg])
    p = params.struct()
    g = grads.struct()
    L.check(L.lib().gs_render_bwd(plan.handle, plan.ws.data_ptr(), ctypes.byref(p), ca, bgc, _ptr(rgb),
                                  _ptr(disp), _ptr(dL_drgb), _ptr(dL_ddisp), ctypes.byref(g),
                                  _stream(stream)), "gs_render_bwd")


def gs_loss_scratch(plan: Plan, device="cuda") -> torch.Tensor:
    return torch.empty(int(L.lib().gs_loss_scratch_floats(plan.handle)), dtype=torch.float32, device=device)


def gs_loss(plan: Plan, rgb, target, lam: float, dL_drgb, loss, scratch, disp=None, target_disp=None,
            disp_weight: float = 0.0, dL_ddisp=None, stream=None) -> None:
    L.check(L.lib().gs_loss(plan.handle, _ptr(rgb), _ptr(target), float(lam), _ptr(disp), _ptr(target_disp),
                            float(disp_weight), _ptr(dL_drgb), _ptr(dL_ddisp), _ptr(loss), _ptr(scratch),
                            _stream(stream)), "gs_loss")


def gs_adam_step(p, g, m, v, lr: float, step: int, b1=0.9, b2=0.999, eps=1e-15, stream=None) -> None:
    L.check(L.lib().gs_adam_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), float(lr), float(b1),
                                 float(b2), float(eps), int(step), _stream(stream)), "gs_adam_step")


def adam_groups_array(groups) -> ctypes.Array:
    """groups: list of dicts p, g, m, v, lr and optional period, head, lr_head."""
    arr = (L.GsAdamGroup * len(groups))()
    for i, gr in enumerate(groups):
        a = arr[i]
        a.p, a.g, a.m, a.v = _ptr(gr["p"]), _ptr(gr["g"]), _ptr(gr["m"]), _ptr(gr["v"])
        a.n = gr["p"].numel()
        a.lr = float(gr["lr"])
        a.period = int(gr.get("period", 0))
        a.head = int(gr.get("head", 0))
        a.lr_head = float(gr.get("lr_head", 0.0))
    return arr


def gs_adam_step_multi(groups, step: int, b1=0.9, b2=0.999, eps=1e-15, stream=None, _arr=None) -> None:
    arr = _arr if _arr is not None else adam_groups_array(groups)
    L.check(L.lib().gs_adam_step_multi(arr, len(arr), float(b1), float(b2), float(eps), int(step),
                                       _stream(stream)), "gs_adam_step_multi")


def gs_adam_step_multi_dev(groups, d_step: torch.Tensor, b1=0.9, b2=0.999, eps=1e-15, stream=None,
                           _arr=None) -> None:
    """Adam over groups with the step count kept on the device (int32
    tensor of one element, incremented by the call)."""
    if d_step.dtype != torch.int32 or not d_step.is_cuda:
        raise TypeError("d_step must be a CUDA int32 tensor")
    arr = _arr if _arr is not None else adam_groups_array(groups)
    L.check(L.lib().gs_adam_step_multi_dev(arr, len(arr), float(b1), float(b2), float(eps), _ptr(d_step, None),
                                           _stream(stream)), "gs_adam_step_multi_dev")


def adam_hparams(lrs: dict, b1=0.9, b2=0.999, eps=1e-15, visible_only: bool = False) -> L.GsAdamHparams:
    """lrs with keys means, log_scales, quats, opacity_logits, sh_dc, sh_rest."""
    return L.GsAdamHparams(float(lrs["means"]), float(lrs["log_scales"]), float(lrs["quats"]),
                           float(lrs["opacity_logits"]), float(lrs["sh_dc"]), float(lrs["sh_rest"]), float(b1),
                           float(b2), float(eps), int(bool(visible_only)))


def gs_preprocess_bwd_adam(plan: Plan, params: Gaussians, cams, m: Gaussians, v: Gaussians, lrs: dict,
                           d_step: torch.Tensor, b1=0.9, b2=0.999, eps=1e-15, visible_only: bool = False,
                           stream=None) -> None:
    """Preprocess backward fused with the Adam update (parameters, m and v
    updated in place; d_step incremented).  visible_only: the sparse Adam
    that leaves Gaussians which touched no tile as they are."""
    if d_step.dtype != torch.int32 or not d_step.is_cuda:
        raise TypeError("d_step must be a CUDA int32 tensor")
    ca = cameras_array(cams)
    p, ms, vs = params.struct(), m.struct(), v.struct()
    hp = adam_hparams(lrs, b1, b2, eps, visible_only)
    L.check(L.lib().gs_preprocess_bwd_adam(plan.handle, plan.ws.data_ptr(), ctypes.byref(p), ca, ctypes.byref(ms),
                                           ctypes.byref(vs), ctypes.byref(hp), _ptr(d_step, None),
                                           _stream(stream)), "gs_preprocess_bwd_adam")


# ------------------------------------------------- densification (Sec. 3.2)

def gs_densify_scratch(n: int, device="cuda") -> torch.Tensor:
    return torch.zeros(int(L.lib().gs_densify_scratch_bytes(int(n))), dtype=torch.uint8, device=device)


def gs_densify_score(plan: Plan, rgb, target, tau: float, photo, s_plus, r_minus, scratch, stream=None) -> None:
    """Add the views' Eq. 4 / Eq. 6 terms to s_plus and r_minus (float32, N);
    photo: float32 device tensor with one photometric loss per view."""
    L.check(L.lib().gs_densify_score(plan.handle, plan.ws.data_ptr(), _ptr(rgb), _ptr(target), float(tau),
                                     _ptr(photo), _ptr(s_plus), _ptr(r_minus), _ptr(scratch, None),
                                     _stream(stream)), "gs_densify_score")


def gs_densify_plan(params: "Gaussians", s_plus, r_minus, rules: dict, action, offsets, scratch,
                    stream=None) -> int:
    """Actions (int32, N) and first output slots (int64, N); returns the new
    Gaussian count (synchronises)."""
    if action.dtype != torch.int32 or offsets.dtype != torch.int64:
        raise TypeError("action must be int32 and offsets int64")
    r = L.GsDensifyRules(float(rules["tau_plus"]), float(rules["tau_minus"]), float(rules["min_opacity"]),
                         float(rules["percent_dense"]), float(rules["extent"]), int(rules["k_views"]))
    p = params.struct()
    out = ctypes.c_int64(0)
    L.check(L.lib().gs_densify_plan(params.n, ctypes.byref(p), _ptr(s_plus), _ptr(r_minus), ctypes.byref(r),
                                    _ptr(action, None), _ptr(offsets, None), _ptr(scratch, None), ctypes.byref(out),
                                    _stream(stream)), "gs_densify_plan")
    return int(out.value)


def gs_densify_apply(src: "Gaussians", src_m: "Gaussians", src_v: "Gaussians", action, offsets, normals,
                     dst: "Gaussians", dst_m: "Gaussians", dst_v: "Gaussians", stream=None) -> None:
    """normals: float32 (N, 2, 3) standard normal samples (used by splits)."""
    a, b, c = src.struct(), src_m.struct(), src_v.struct()
    d, e, f = dst.struct(), dst_m.struct(), dst_v.struct()
    L.check(L.lib().gs_densify_apply(src.n, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), _ptr(action, None),
                                     _ptr(offsets, None), _ptr(normals), ctypes.byref(d), ctypes.byref(e),
                                     ctypes.byref(f), _stream(stream)), "gs_densify_apply")


def gs_sort_pairs_u32(keys_in, vals_in, keys_out, vals_out, begin_bit: int, end_bit: int, scratch=None,
                      stream=None) -> None:
    n = keys_in.numel()
    if scratch is None:
        scratch = torch.empty(int(L.lib().gs_sort_scratch_bytes(n)), dtype=torch.uint8, device=keys_in.device)
    for t in (keys_in, vals_in, keys_out, vals_out):
        if t.dtype not in (torch.int32, torch.uint32):
            raise TypeError("sort buffers are 32-bit integers")
    L.check(L.lib().gs_sort_pairs_u32(_ptr(keys_in, None), _ptr(vals_in, None), _ptr(keys_out, None),
                                      _ptr(vals_out, None), n, int(begin_bit), int(end_bit),
                                      _ptr(scratch, None), _stream(stream)), "gs_sort_pairs_u32")


# ------------------------------------------------------ neural Gaussians

@dataclass
class NgParams:
    """Anchor set and MLP of the neural-Gaussian decoder (float32, device)."""

    anchor_xyz: torch.Tensor
    feat: torch.Tensor
    anchor_ls: torch.Tensor
    w1: torch.Tensor
    b1: torch.Tensor
    w2: torch.Tensor
    b2: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.anchor_xyz.shape[0])

    def tensors(self):
        return (self.anchor_xyz, self.feat, self.anchor_ls, self.w1, self.b1, self.w2, self.b2)

    def struct(self) -> L.GsNgParams:
        p = L.GsNgParams()
        p.n_anchors = self.n
        p.anchor_xyz = None if self.anchor_xyz is None else _ptr(self.anchor_xyz)
        p.feat, p.anchor_ls, p.w1, p.b1, p.w2, p.b2 = (_ptr(t) for t in self.tensors()[1:])
        return p

    def zeros_like(self) -> "NgParams":
        return NgParams(*(torch.zeros_like(t) for t in self.tensors()))

    @staticmethod
    def from_dict(d: dict, device="cuda") -> "NgParams":
        t = lambda a: torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)
        return NgParams(t(d["anchor_xyz"]), t(d["feat"]), t(d["anchor_ls"]), t(d["w1"]), t(d["b1"]), t(d["w2"]),
                        t(d["b2"]))


def gs_ng_workspace(n_anchors: int, device="cuda") -> torch.Tensor:
    ws = torch.zeros(int(L.lib().gs_ng_workspace_bytes(int(n_anchors))), dtype=torch.uint8, device=device)
    return ws


def ng_children(n_anchors: int, device="cuda") -> "Gaussians":
    n = n_anchors * L.GS_NG_CHILDREN
    z = lambda *s: torch.zeros(*s, device=device)
    return Gaussians(z(n, 3), z(n, 3), z(n, 4), z(n), z(n, 1, 3), 0)


def gs_ng_decode_fwd(ng: NgParams, cam, children: "Gaussians", ws: torch.Tensor, stream=None) -> None:
    c = (L.GsCamera * 1)(camera_struct(cam))
    p = ng.struct()
    ch = children.struct()
    L.check(L.lib().gs_ng_decode_fwd(ctypes.byref(p), c, ctypes.byref(ch), ws.data_ptr(), _stream(stream)),
            "gs_ng_decode_fwd")


def gs_ng_decode_preprocess(ng: NgParams, cam, children: "Gaussians", ws: torch.Tensor, plan: Plan,
                            stream=None) -> None:
    """gs_ng_decode_fwd and gs_preprocess of the children on `plan` in one launch."""
    c = (L.GsCamera * 1)(camera_struct(cam))
    p = ng.struct()
    ch = children.struct()
    L.check(L.lib().gs_ng_decode_preprocess(ctypes.byref(p), c, ctypes.byref(ch), ws.data_ptr(), plan.handle,
                                            plan.ws.data_ptr(), _stream(stream)), "gs_ng_decode_preprocess")


def gs_ng_decode_bwd(ng: NgParams, cam, child_grads: "Gaussians", grads: NgParams, ws: torch.Tensor,
                     zero_child_grads: bool = False, stream=None) -> None:
    c = (L.GsCamera * 1)(camera_struct(cam))
    p = ng.struct()
    cg = child_grads.struct()
    g = grads.struct()
    L.check(L.lib().gs_ng_decode_bwd(ctypes.byref(p), c, ctypes.byref(cg), int(bool(zero_child_grads)),
                                     ctypes.byref(g), ws.data_ptr(), _stream(stream)), "gs_ng_decode_bwd")


def gs_ng_status(ws: torch.Tensor, stream=None) -> int:
    e = ctypes.c_int32(0)
    return int(L.lib().gs_ng_read_status(ws.data_ptr(), ctypes.byref(e), _stream(stream)))


# ---------------------------------------------------------------- pose refinement (Sec. 2.5)

class PoseState:
    """The device state of the global pose correction (gs.h's pose-state
    layout): correction (Delta_R, Delta_t), Adam moments and step, and the
    slots the preprocess backward adds dL/d(omega, tau) into."""

    R, T, M, V, STEP, ACC = slice(0, 9), slice(9, 12), slice(12, 18), slice(18, 24), 24, 32

    def __init__(self, device="cuda"):
        self.buf = torch.empty(L.GS_POSE_STATE_DOUBLES, dtype=torch.float64, device=device)
        self.reset()

    def reset(self, stream=None) -> None:
        L.check(L.lib().gs_pose_init(self.buf.data_ptr(), _stream(stream)), "gs_pose_init")

    def correction(self):
        """(Delta_R (3, 3), Delta_t (3,)) as float64 host arrays (synchronises)."""
        h = self.buf[:12].cpu().numpy()
        return h[:9].reshape(3, 3).copy(), h[9:12].copy()

    def set_correction(self, R, t) -> None:
        self.buf[:9].copy_(torch.as_tensor(R, dtype=torch.float64).reshape(9))
        self.buf[9:12].copy_(torch.as_tensor(t, dtype=torch.float64).reshape(3))

    def slots(self) -> torch.Tensor:
        """(GS_POSE_SLOTS, 6) view of the gradient partial sums."""
        return self.buf[self.ACC:].view(L.GS_POSE_SLOTS, 8)[:, :6]

    def grad(self):
        """The accumulated dL/d(omega, tau) (host float64, synchronises)."""
        return self.slots().sum(0).cpu().numpy()


def pose_hparams(lr_rot: float, lr_trans: float, b1=0.9, b2=0.999, eps=1e-15) -> L.GsPoseHparams:
    return L.GsPoseHparams(float(lr_rot), float(lr_trans), float(b1), float(b2), float(eps))


def gs_pose_step(state: PoseState, lr_rot: float, lr_trans: float, b1=0.9, b2=0.999, eps=1e-15,
                 stream=None, _hp=None) -> None:
    hp = _hp if _hp is not None else pose_hparams(lr_rot, lr_trans, b1, b2, eps)
    L.check(L.lib().gs_pose_step(state.buf.data_ptr(), ctypes.byref(hp), _stream(stream)), "gs_pose_step")
