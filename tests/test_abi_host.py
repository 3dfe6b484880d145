"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point include/gs.h declares, and the pure-host
calls (plan creation, sizes, error strings) behave as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^GS_API[^(;]*?\b(gs_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2601_19489_gb300 import _lib

    return _lib.load()


def test_header_declares_the_path(lib):
    names = _declared()
    for required in ("gs_preprocess", "gs_bin_sort", "gs_render_fwd", "gs_render_bwd", "gs_adam_step"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2601_19489_gb300 import _lib

    for name in _declared():
        assert hasattr(lib, name), name
        assert name in _lib.EXPORTS, name
    assert set(_lib.EXPORTS) == _declared()


def test_plan_rejects_bad_arguments(lib):
    w = (ctypes.c_int32 * 2)(64, 32)
    h = (ctypes.c_int32 * 2)(48, 16)
    assert lib.gs_plan_create(0, 0, 1, w, h, 100) is None
    assert lib.gs_plan_create(10, 4, 1, w, h, 100) is None
    assert lib.gs_plan_create(10, 0, 0, w, h, 100) is None
    assert lib.gs_plan_create(10, 0, 17, w, h, 100) is None
    assert lib.gs_plan_create(10, 0, 1, w, h, 0) is None
    assert lib.gs_plan_create(10, 0, 1, w, h, 1 << 31) is None
    bad = (ctypes.c_int32 * 1)(0)
    assert lib.gs_plan_create(10, 0, 1, bad, h, 100) is None


def test_tuned_plan_choices(lib):
    from paper_2601_19489_gb300 import _lib as L

    w = (ctypes.c_int32 * 1)(1920)
    h = (ctypes.c_int32 * 1)(1080)
    for bucket, warps, chains in ((16, 4, 0), (128, 4, 0), (32, 3, 0), (64, 16, 0), (32, 4, 3), (32, 4, -1)):
        tu = L.GsTuning(bucket, warps, chains)
        assert lib.gs_plan_create_tuned(1000, 0, 1, w, h, 1 << 20, ctypes.byref(tu)) is None
    sizes = {}
    for bucket in (0, 32, 64):
        p = lib.gs_plan_create_tuned(1000, 0, 1, w, h, 1 << 22, ctypes.byref(L.GsTuning(bucket, 0)))
        assert p
        sizes[bucket] = lib.gs_plan_workspace_bytes(p)
        lib.gs_plan_destroy(p)
    p = lib.gs_plan_create(1000, 0, 1, w, h, 1 << 22)
    assert lib.gs_plan_workspace_bytes(p) == sizes[0] == sizes[32]
    lib.gs_plan_destroy(p)
    # 64-splat buckets halve the checkpoint store: 20 bytes x 256 pixels per bucket
    assert sizes[32] - sizes[64] >= 20 * 256 * ((1 << 22) // 64) - 4096


def test_plan_sizes(lib):
    w = (ctypes.c_int32 * 2)(1920, 333)
    h = (ctypes.c_int32 * 2)(1080, 187)
    p = lib.gs_plan_create(1 << 20, 3, 2, w, h, 1 << 24)
    assert p
    try:
        assert lib.gs_plan_pixels(p) == 1920 * 1080 + 333 * 187
        nbytes = lib.gs_plan_workspace_bytes(p)
        # at least the per-instance buffers, checkpoints and records
        assert nbytes > 4 * 4 * (1 << 24) + 48 * 2 * (1 << 20)
        ptr = ctypes.c_void_p()
        nb = ctypes.c_size_t()
        base = 1 << 40
        seen = []
        for which in range(10):
            assert lib.gs_workspace_view(p, base, which, ctypes.byref(ptr), ctypes.byref(nb)) == 0
            assert (ptr.value - base) % 256 == 0 and ptr.value - base + nb.value <= nbytes
            seen.append((ptr.value, nb.value))
        assert lib.gs_workspace_view(p, base, 99, ctypes.byref(ptr), ctypes.byref(nb)) == -1
        # distinct buffers do not overlap
        seen.sort()
        for (a, na), (b, _) in zip(seen[:-1], seen[1:]):
            assert a + na <= b
        # per-block partial sums of the fused SSIM pass (32 columns x at
        # least 48 rows per block and channel) and of the L1 passes, and a
        # counter
        blocks = -(-1920 // 32) * -(-1080 // 48) * 3 * 2
        assert lib.gs_loss_scratch_floats(p) >= 2 * blocks + 2
    finally:
        lib.gs_plan_destroy(p)


def test_error_strings(lib):
    for code in (0, -1, -2, -3, -4, -5):
        assert lib.gs_error_string(code)
    assert lib.gs_error_string(-99) == b"unknown error"


def test_argument_errors_are_caught_on_the_host(lib):
    assert lib.gs_preprocess(None, None, None, None, None) == -1
    assert lib.gs_bin_sort(None, None, 1, None) == -1
    assert lib.gs_render_fwd(None, None, None, None, None, None, None) == -1
    assert lib.gs_sort_pairs_u32(None, None, None, None, -1, 0, 8, None, None) == -1
    assert lib.gs_sort_pairs_u32(None, None, None, None, 0, 0, 8, None, None) == 0  # empty: no-op
    from paper_2601_19489_gb300 import _lib

    assert lib.gs_adam_step_multi(None, 0, 0.9, 0.999, 1e-15, 1, None) == -1
    g = (_lib.GsAdamGroup * 1)()
    assert lib.gs_adam_step_multi(g, 1, 0.9, 0.999, 1e-15, 0, None) == -1  # step < 1


def test_pose_entry_points_check_arguments_on_the_host(lib):
    """Argument errors are reported before anything is enqueued (no GPU is
    touched: the pointers below are never dereferenced)."""
    from paper_2601_19489_gb300 import _lib as L

    w = (ctypes.c_int32 * 1)(64)
    h = (ctypes.c_int32 * 1)(48)
    plan = lib.gs_plan_create(10, 0, 1, w, h, 100)
    assert plan
    try:
        assert lib.gs_plan_set_pose(plan, None) == L.GS_OK  # detach
        assert lib.gs_plan_set_pose(plan, ctypes.c_void_p(8)) == L.GS_ERR_ARG  # misaligned
        assert lib.gs_plan_set_pose(None, ctypes.c_void_p(16)) == L.GS_ERR_ARG
    finally:
        lib.gs_plan_destroy(plan)
    ok = L.GsPoseHparams(1e-3, 1e-3, 0.9, 0.999, 1e-15)
    assert lib.gs_pose_step(None, ctypes.byref(ok), None) == L.GS_ERR_ARG
    assert lib.gs_pose_step(ctypes.c_void_p(24), ctypes.byref(ok), None) == L.GS_ERR_ARG
    assert lib.gs_pose_step(ctypes.c_void_p(16), None, None) == L.GS_ERR_ARG
    for bad in (L.GsPoseHparams(1e-3, 1e-3, 1.0, 0.999, 1e-15), L.GsPoseHparams(1e-3, 1e-3, 0.9, 0.2, 1e-15),
                L.GsPoseHparams(-1.0, 1e-3, 0.9, 0.999, 1e-15), L.GsPoseHparams(1e-3, 1e-3, 0.9, 0.999, -1.0)):
        assert lib.gs_pose_step(ctypes.c_void_p(16), ctypes.byref(bad), None) == L.GS_ERR_ARG
    assert lib.gs_pose_init(None, None) == L.GS_ERR_ARG
    assert lib.gs_pose_init(ctypes.c_void_p(40), None) == L.GS_ERR_ARG
    assert L.GS_POSE_STATE_DOUBLES == 32 + 8 * L.GS_POSE_SLOTS
    hdr = open(os.path.join(ROOT, "include", "gs.h")).read()
    assert re.search(r"#define GS_POSE_SLOTS %d\b" % L.GS_POSE_SLOTS, hdr)


def test_trainer_exposes_the_default_views_buffers():
    """The default view's image buffers are reachable from the trainer (the
    smoke check and the tests read them)."""
    from paper_2601_19489_gb300.trainer import Trainer

    for name in ("plan", "rgb", "disp"):
        assert isinstance(getattr(Trainer, name), property), name


def test_misaligned_parameter_rows_are_refused_on_the_host(lib):
    """quats and sh move in float4s: a pointer off a 16-byte boundary is an
    argument error, reported before anything is enqueued."""
    from paper_2601_19489_gb300 import _lib as L

    w = (ctypes.c_int32 * 1)(64)
    h = (ctypes.c_int32 * 1)(48)
    plan = lib.gs_plan_create(10, 1, 1, w, h, 100)
    assert plan
    try:
        cam = L.GsCamera()
        cam.fx = cam.fy = 64.0
        cam.cx, cam.cy, cam.width, cam.height, cam.near_z = 32.0, 24.0, 64, 48, 0.2
        for bad in ("quats", "sh"):
            p = L.GsParams()
            p.n, p.sh_degree = 10, 1
            p.means, p.log_scales, p.quats, p.opacity_logits, p.sh = 256, 512, 768, 1024, 1280
            setattr(p, bad, getattr(p, bad) + 4)
            rc = lib.gs_preprocess(plan, ctypes.c_void_p(4096), ctypes.byref(p), ctypes.byref(cam), None)
            assert rc == L.GS_ERR_ARG, bad
    finally:
        lib.gs_plan_destroy(plan)


def test_more_argument_errors_are_caught_on_the_host(lib):
    """Each call below carries one invalid argument that the host check
    reports before any launch (the device pointers are never touched)."""
    from paper_2601_19489_gb300 import _lib as L

    ARG = L.GS_ERR_ARG
    w = (ctypes.c_int32 * 1)(64)
    h = (ctypes.c_int32 * 1)(48)
    plan = lib.gs_plan_create(10, 1, 1, w, h, 100)
    assert plan
    fake = ctypes.c_void_p(4096)
    try:
        # loss: lambda outside [0, 1]; disparity without its target
        assert lib.gs_loss(plan, fake, fake, ctypes.c_float(1.5), None, None, ctypes.c_float(0.0), fake, None,
                           fake, fake, None) == ARG
        assert lib.gs_loss(plan, fake, fake, ctypes.c_float(0.2), fake, None, ctypes.c_float(0.1), fake, fake,
                           fake, fake, None) == ARG
        # densification: negative mask threshold; K < 1; empty set
        assert lib.gs_densify_score(plan, fake, fake, fake, ctypes.c_float(-0.1), fake, fake, fake, fake,
                                    None) == ARG
        p = L.GsParams()
        p.n, p.sh_degree = 10, 1
        p.means, p.log_scales, p.quats, p.opacity_logits, p.sh = 256, 512, 768, 1024, 1280
        rules = L.GsDensifyRules(5.0, 0.95, 0.005, 0.01, 4.0, 0)
        out_n = ctypes.c_int64(0)
        assert lib.gs_densify_plan(10, ctypes.byref(p), fake, fake, ctypes.byref(rules), fake, fake, fake,
                                   ctypes.byref(out_n), None) == ARG
        assert lib.gs_densify_apply(0, ctypes.byref(p), ctypes.byref(p), ctypes.byref(p), fake, fake, fake,
                                    ctypes.byref(p), ctypes.byref(p), ctypes.byref(p), None) == ARG
        # fused Adam: b1 outside (0, 1)
        cam = L.GsCamera()
        cam.fx = cam.fy = 64.0
        cam.cx, cam.cy, cam.width, cam.height, cam.near_z = 32.0, 24.0, 64, 48, 0.2
        hp = L.GsAdamHparams(1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1.0, 0.999, 1e-15, 0)
        assert lib.gs_preprocess_bwd_adam(plan, fake, ctypes.byref(p), ctypes.byref(cam), ctypes.byref(p),
                                          ctypes.byref(p), ctypes.byref(hp), fake, None) == ARG
    finally:
        lib.gs_plan_destroy(plan)
    # decoder: no anchors; a child set of the wrong size
    ng = L.GsNgParams(0, 256, 512, 768, 1024, 1280, 1536, 1792)
    kids = L.GsParams()
    kids.n, kids.sh_degree = 10, 0
    assert lib.gs_ng_decode_fwd(ctypes.byref(ng), ctypes.byref(L.GsCamera()), ctypes.byref(kids), fake,
                                None) == ARG
    ng.n_anchors = 4
    assert lib.gs_ng_decode_fwd(ctypes.byref(ng), ctypes.byref(L.GsCamera()), ctypes.byref(kids), fake,
                                None) == ARG
    # fused decode + preprocess: no plan; a plan of two views; a plan whose
    # size differs from the children's; an SH-degree-3 plan
    kids.n = 40
    kids.means = kids.log_scales = kids.quats = kids.opacity_logits = kids.sh = 4096
    assert lib.gs_ng_decode_preprocess(ctypes.byref(ng), ctypes.byref(L.GsCamera()), ctypes.byref(kids), fake,
                                       None, fake, None) == ARG
    for n, deg, views in ((40, 0, 2), (41, 0, 1), (40, 3, 1)):
        ws_ = (ctypes.c_int32 * views)(*([64] * views))
        hs_ = (ctypes.c_int32 * views)(*([48] * views))
        pl = lib.gs_plan_create(n, deg, views, ws_, hs_, 1 << 12)
        assert pl
        try:
            assert lib.gs_ng_decode_preprocess(ctypes.byref(ng), ctypes.byref(L.GsCamera()), ctypes.byref(kids),
                                               fake, pl, fake, None) == ARG
        finally:
            lib.gs_plan_destroy(pl)


def test_wait_probe_arguments_are_checked_on_the_host(lib):
    from paper_2601_19489_gb300 import _lib as L

    fake = ctypes.c_void_p(4096)
    assert lib.gs_ng_wait_probe(None, 10, 0, None) == L.GS_ERR_ARG
    assert lib.gs_ng_wait_probe(fake, 0, 0, None) == L.GS_ERR_ARG
    assert lib.gs_ng_wait_probe(fake, (1 << 22) + 1, 0, None) == L.GS_ERR_ARG
    assert lib.gs_ng_wait_probe(fake, 10, 2, None) == L.GS_ERR_ARG
