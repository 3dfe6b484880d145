/*
 * gs.h — C ABI of the GB300 (sm_103a) differentiable 3D Gaussian Splatting
 * training step.
 *
 * Paper: "Fast Converging 3D Gaussian Splatting for 1-Minute Reconstruction"
 * (arXiv 2601.19489).  The step follows Sec. 2.1 (preprocessCUDA: projection,
 * compact SnugBox, per-column tile test, load-balanced tile-key write, depth
 * sort; renderCUDA: front-to-back alpha blending) and Sec. 2.2 (checkpoints
 * every 32 splats, per-Gaussian parallel backward), followed by Adam (also
 * fused into the preprocess backward, dense or visible-only).  Around it:
 * the neural-Gaussian decoder of Sec. 2.3 (gs_ng_*), the global pose
 * refinement of Sec. 2.5 (gs_pose_*, gs_plan_set_pose) and the score-guided
 * densification and pruning of Sec. 3.2 (gs_densify_*).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named d_* are DEVICE pointers; pointers named h_* (and the
 *    camera / parameter structs themselves) are HOST pointers read during the
 *    call only.  The library never allocates device memory: the caller owns
 *    every device buffer, including the workspace `ws`.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Every call only enqueues work on that stream and returns
 *    without synchronising, except gs_read_status which synchronises it.
 *  - Return value: GS_OK (0) or a negative GS_ERR_* code.  Argument errors are
 *    detected on the host before anything is enqueued.  Errors that only the
 *    device can see (instance-capacity overflow, a timed-out wait, an
 *    internal consistency check) are recorded in the workspace status words
 *    and reported by gs_read_status.
 *  - Images are planar float32: colour is [view][3][height][width], single
 *    channel maps are [view][height][width], views concatenated in order.
 *  - Cameras use OpenCV axes (x right, y down, z forward); w2c is the
 *    row-major 3x4 world-to-camera matrix [R | t]; the pixel (i, j) has its
 *    centre at (i + 0.5, j + 0.5) in the same units as (cx, cy).
 *  - Gaussian parameters are float32 arrays of n rows: means n x 3,
 *    log_scales n x 3, quats n x 4 as (w, x, y, z), opacity_logits n,
 *    sh n x K x 3 with K = (sh_degree + 1)^2 (coefficient-major per Gaussian,
 *    real spherical harmonics with the Condon-Shortley phase).  quats and sh
 *    (of parameters and of gradients) must start 16-byte aligned: they are
 *    moved in float4s (GS_ERR_ARG otherwise).
 *  - Gradients are ACCUMULATED (+=) into the caller's gradient arrays, so
 *    several views or calls sum.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Every entry point is exported from the shared library (which otherwise
 * builds with hidden visibility). */
#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

#define GS_MAX_VIEWS 16
#define GS_TILE 16       /* tile edge in pixels (Sec. 2.2: 16x16 tiles) */
#define GS_BUCKET 32     /* default splats per checkpoint bucket (Sec. 2.2) */

enum {
    GS_OK = 0,
    GS_ERR_ARG = -1,      /* bad argument (null pointer, size, degree, alignment) */
    GS_ERR_CAPACITY = -2, /* more tile instances than the workspace holds */
    GS_ERR_CUDA = -3,     /* a CUDA runtime call failed */
    GS_ERR_TIMEOUT = -4,  /* a bounded device-side wait gave up */
    GS_ERR_INTERNAL = -5  /* a device-side consistency check failed */
};

typedef struct {
    float fx, fy, cx, cy;  /* pinhole intrinsics, pixels */
    float w2c[12];         /* row-major [R | t], world -> camera */
    int32_t width, height; /* image size in pixels */
    float near_z;          /* Gaussians with camera z <= near_z are culled (0.2) */
} gs_camera;

typedef struct {
    int64_t n;              /* number of Gaussians */
    int32_t sh_degree;      /* 0..3 */
    float *means;           /* device, n x 3 */
    float *log_scales;      /* device, n x 3 */
    float *quats;           /* device, n x 4 */
    float *opacity_logits;  /* device, n */
    float *sh;              /* device, n x K x 3 */
} gs_params;

typedef struct {
    int64_t n_instances;     /* Gaussian-tile pairs of the last gs_bin_sort */
    int64_t n_buckets;       /* checkpoint buckets of the last gs_bin_sort */
    int64_t inst_capacity;   /* capacity the plan was made with */
    int32_t overflow;        /* 1: n_instances > inst_capacity, result truncated */
    int32_t error;           /* 0 or a GS_ERR_* code seen on the device */
} gs_status;

/* ------------------------------------------------------------------ plan
 * A plan is a small HOST object that fixes the sizes of one training step:
 * the Gaussian count, SH degree, the views (1..GS_MAX_VIEWS, each with its
 * own resolution) and the capacity for tile instances.  It computes the
 * workspace layout; it owns no device memory.
 *
 * gs_plan_create returns NULL on bad arguments (n <= 0, degree outside 0..3,
 * n_views outside 1..GS_MAX_VIEWS, non-positive sizes, capacity <= 0 or
 * >= 2^31).  inst_capacity bounds the number of (Gaussian, tile) pairs; a
 * step that needs more sets the overflow status (see gs_read_status) and
 * renders only the pairs that fit. */
typedef struct gs_plan gs_plan;

GS_API gs_plan *gs_plan_create(int64_t n, int32_t sh_degree, int32_t n_views, const int32_t *h_widths,
                               const int32_t *h_heights, int64_t inst_capacity);

/* Launch-shape choices that change speed but not results (beyond float32
 * summation order), for an autotuner to pick per workload:
 *   bucket     splats per checkpoint bucket of the forward and per unit of
 *              work of the per-Gaussian backward (Sec. 2.2 uses 32): 32 or
 *              64.  At 64 each lane of the backward owns two adjacent splats
 *              and evaluates both in packed float32 pairs, branch-free;
 *              checkpoint memory and traffic halve.
 *   bwd_warps  warps per CTA of the per-Gaussian backward (the warps of a CTA
 *              share one tile's staged pixel data): 1, 2, 4 or 8.
 *   bwd_chains pixel chains a lane of the 32-splat backward pipeline walks:
 *              2 (two interleaved halves of the bucket's live pixels: more
 *              independent work per step), 1 (one chain: fewer idle steps
 *              while the pipeline fills and drains), or 0: two when the
 *              bucket has at least 128 live pixels, else one.  Ignored at 64.
 * A zero field takes the default (32, 4, 0; fwd_pixels 1).  gs_plan_create
 * uses the defaults (the Python layer's default plan takes bucket 64, one
 * backward warp, chains 0 and fwd_pixels 2: the autotuner's pick at 1M
 * Gaussians and 1080p).
 * Returns NULL on the same conditions as gs_plan_create or an unsupported
 * choice. */
typedef struct {
    int32_t bucket;
    int32_t bwd_warps;
    int32_t bwd_chains;
    /* Ablation switches (Sec. 4, Tab. 1), both 0 by default:
     *   bbox_3sigma    bin each Gaussian into the tiles holding the pixel
     *                  centres of the classic square of half-width
     *                  ceil(3 sqrt(largest eigenvalue of Sigma')) instead of
     *                  the SnugBox with its per-column test (Sec. 2.1, "F").
     *                  Not result-exact: a Gaussian with opacity above ~0.35 can
     *                  reach alpha >= 1/255 outside that box.
     *   bwd_per_pixel  the classic per-pixel backward (a thread per pixel walks
     *                  its list back to front; warp sums of each splat's
     *                  gradient, then atomics) instead of the per-Gaussian
     *                  backward of Sec. 2.2 ("B"); no checkpoints are written. */
    int32_t bbox_3sigma;
    int32_t bwd_per_pixel;
    /* bin_radix  1: gs_bin_sort with load_balanced = 1 takes the key-write +
     *            radix-sort path (the only path of load_balanced = 0) instead
     *            of the counting binning; both give the same per-tile lists.
     *            0 by default. */
    int32_t bin_radix;
    /* fwd_pixels pixels per thread of the forward blend: 1 (a CTA of 256
     *            threads per tile), or 2 (128 threads, each blending two
     *            horizontally adjacent pixels in packed float32 pairs,
     *            branch-free; the same float32 operations per pixel, so the
     *            blend decisions are identical).  0 takes 1. */
    int32_t fwd_pixels;
} gs_tuning;
GS_API gs_plan *gs_plan_create_tuned(int64_t n, int32_t sh_degree, int32_t n_views, const int32_t *h_widths,
                                     const int32_t *h_heights, int64_t inst_capacity, const gs_tuning *tuning);
GS_API void gs_plan_destroy(gs_plan *plan);
/* Bytes of device workspace the plan needs (256-byte aligned base required). */
GS_API size_t gs_plan_workspace_bytes(const gs_plan *plan);
/* Pixels summed over views (the length of one image channel). */
GS_API int64_t gs_plan_pixels(const gs_plan *plan);

/* Device address and size of an internal workspace buffer, for inspection
 * by tests and tools.  `which` is one of GS_WS_*.  Returns GS_ERR_ARG for an
 * unknown id. */
enum {
    GS_WS_RECORDS = 0,    /* float4 x 3 per (view, Gaussian): {mx, my, A, B}, {C, log2 o, 1/z,
                             mx_lo}, {r, g, b, my_lo}; (A, B, C) = conic * log2(e) / 2,
                             mean2d = (mx + mx_lo, my + my_lo) */
    GS_WS_TILES_TOUCHED,  /* uint32 per (view, Gaussian) */
    GS_WS_RECTS,          /* uint16 x 4 per (view, Gaussian): candidate tile box */
    GS_WS_DEPTH_ORDER,    /* uint32 per rank: item id v*n + g in ascending depth */
    GS_WS_INST_TILE,      /* uint32 per instance, sorted global tile id (radix
                             binning path only; not written by the counting path) */
    GS_WS_INST_GID,       /* uint32 per instance, item id v*n + g */
    GS_WS_TILE_RANGES,    /* uint32 x 2 per global tile: [start, end) */
    GS_WS_N_CONTRIB,      /* uint32 per pixel: list position of last blended splat + 1 */
    GS_WS_GRAD2D,         /* float x 12 per (view, Gaussian): 2D gradients */
    GS_WS_STATUS,         /* status words */
    GS_WS_BIN,            /* float2 per (view, Gaussian): binning level set, A C - B^2 */
    GS_WS_COUNT
};
GS_API int gs_workspace_view(const gs_plan *plan, void *ws, int which, void **d_ptr, size_t *bytes);

/* Synchronise `stream` and read the status words of `ws` (see gs_status).
 * Returns GS_OK, GS_ERR_CAPACITY when the last bin/sort overflowed, or the
 * device-recorded error. */
GS_API int gs_read_status(const gs_plan *plan, const void *ws, gs_status *out, void *stream);

GS_API const char *gs_error_string(int code);

/* ------------------------------------------------------- a1: preprocess
 * Sec. 2.1 (preprocessCUDA) with Eq. 1-2: per (view, Gaussian) project the
 * mean, build the 2D covariance with the local affine (EWA) approximation,
 * invert it to the conic, evaluate the SH colour along the viewing direction,
 * take the opacity-aware level set t = 2 ln(255 o), bound it by the SnugBox
 * and count the touched tiles exactly with the per-column test.
 * h_cams: n_views cameras (host), sizes must match the plan.
 * Writes the projected records, tile counts and boxes into ws. */
GS_API int gs_preprocess(const gs_plan *plan, void *ws, const gs_params *params, const gs_camera *h_cams,
                         void *stream);

/* ---------------------------------------------- a2-a4: bin, sort, ranges
 * Sec. 2.1: order the visible Gaussians of every view by depth (on-device
 * radix sort), then build every tile's list of the Gaussians that touch it
 * (the SnugBox tile columns with the exact per-column ellipse test), each
 * list in (depth, id) order, and record each tile's [start, end) range in
 * the instance list.
 * load_balanced = 1 (default path, "counting binning"): tiles are grouped
 * in blocks of 8 x 8; one (block, Gaussian) entry per block the Gaussian's
 * SnugBox meets is written in depth order and stably sorted by block
 * (a radix sort over these few entries), so a Gaussian of any size is cut
 * into pieces of at most 8 columns; each block's entries are cut into
 * chunks of 128, which warps claim from a counter.  Per chunk, 32 entries
 * at a time, one per lane: each lane computes its entry's 64-bit mask of
 * the block's tiles it touches (the exact per-column test, the lanes
 * visiting the columns in lockstep), and a 32 x 32 bit transpose across the
 * warp turns the masks into per-tile entry sets whose sizes are the chunk's
 * counts per tile.  After a scan of the counts (tiles of a block, chunks of
 * a tile, blocks), a second pass transposes the masks again and each lane
 * appends the entries that touch its two tiles, in entry order, to those
 * tiles' runs, writing each Gaussian id straight to its final position (in
 * whole 32-byte sectors).  Tile lists lie block by block in the instance
 * list.
 * load_balanced = 0 ("Sq", and load_balanced = 1 with the plan's bin_radix):
 * one (tile, Gaussian) key per touched tile is written in depth order — by
 * one thread walking its Gaussian's columns (Sq), or by the load-balanced
 * column walk — and the keys are stably radix-sorted by tile; tile lists lie
 * in tile order.  Every path gives the same list for every tile. */
GS_API int gs_bin_sort(const gs_plan *plan, void *ws, int load_balanced, void *stream);

/* --------------------------------------------------------- a5: forward
 * Sec. 2.1 (renderCUDA) and Sec. 2.2: per pixel, front-to-back blending of
 * its tile's depth-sorted splats with alpha = min(0.99, o e^power), skipping
 * alpha < 1/255 and stopping before T (1 - alpha) < 1e-4; every 32 (or 64,
 * the plan's bucket) splats the per-pixel T, C and D are checkpointed in ws
 * for the backward (each tile takes its buckets from a counter the call
 * restarts, so the checkpoints belong to the last forward), and each tile's
 * backward work units (chunks of up to 8 buckets) are filed under one of 8
 * work classes by log2 of its last contributor.  With fwd_pixels = 2 (the
 * tuning field) a thread blends two adjacent pixels in packed float32 pairs;
 * the results are identical.
 * h_bg: 3 floats (host) background colour.  Outputs (device, may not alias):
 * d_out_rgb  colour C + T bg, planar per view;  d_out_disp  blended
 * disparity sum(alpha T / z);  d_out_T  final transmittance. */
GS_API int gs_render_fwd(const gs_plan *plan, void *ws, const float *h_bg, float *d_out_rgb,
                         float *d_out_disp, float *d_out_T, void *stream);

/* ------------------------------------------- a7 + a8: backward
 * Sec. 2.2: per-Gaussian parallel backward.  One warp per checkpoint
 * bucket (lane = splat at 32 splats, two splats per lane in packed pairs at
 * 64), iterates the tile's pixels seeded from the forward's checkpoints,
 * accumulates in registers and issues one atomic per splat parameter; the
 * persistent CTAs claim the forward's work units, heaviest class first.
 * Then the per-Gaussian preprocess backward chains the 2D gradients to the
 * parameters.
 * d_rgb, d_disp: the forward's outputs for the same ws (device).
 * d_dL_drgb, d_dL_ddisp: upstream gradients, same layouts (d_dL_ddisp may be
 * NULL: no disparity loss).  h_cams: the cameras given to gs_preprocess.
 * grads: device arrays with the layout of params, ACCUMULATED (+=). */
GS_API int gs_render_bwd(const gs_plan *plan, void *ws, const gs_params *params, const gs_camera *h_cams,
                         const float *h_bg, const float *d_rgb, const float *d_disp, const float *d_dL_drgb,
                         const float *d_dL_ddisp, gs_params *grads, void *stream);

/* The two halves of gs_render_bwd, for callers that time or schedule them
 * separately.  gs_render_bwd_blend (a7) overwrites the per-(view, Gaussian)
 * 2D gradients in ws (GS_WS_GRAD2D: dL/d mean2d, conic a b c, opacity,
 * 1/z, rgb); gs_preprocess_bwd (a8) chains them to the parameters and
 * ACCUMULATES into grads.  Same arguments and rules as gs_render_bwd. */
GS_API int gs_render_bwd_blend(const gs_plan *plan, void *ws, const float *d_rgb, const float *d_disp,
                               const float *d_dL_drgb, const float *d_dL_ddisp, void *stream);
GS_API int gs_preprocess_bwd(const gs_plan *plan, void *ws, const gs_params *params,
                             const gs_camera *h_cams, gs_params *grads, void *stream);

/* a8 + a9 fused, for a step whose gradient is complete after the blend
 * backward (every view of the step is in this plan): the preprocess backward
 * of every Gaussian, summed over the plan's views, followed at once by the
 * Adam update of gs_adam_step_multi_dev on that Gaussian's parameters, in
 * place.  The gradient is never stored, which saves writing it here and
 * reading it back in Adam.  Gaussians that touched no tile are updated with
 * a zero gradient, as an unfused step would.
 * params: parameters (device, read and written).  adam_m, adam_v: first and
 * second moments with the layout of params (device, read and written).
 * d_step: device int32 step count, incremented on the stream first; the
 * incremented value is the t of the bias corrections.  Rates per parameter
 * group; the SH DC coefficients (the first 3 floats of a Gaussian's SH row)
 * take lr_sh_dc, the rest lr_sh_rest.  b1, b2 in (0, 1).  Every array of
 * params, adam_m and adam_v must start 16-byte aligned (GS_ERR_ARG
 * otherwise).
 * visible_only != 0 selects the sparse (visible-only) Adam of the Taming-3DGS
 * line the paper builds on (Sec. 2.2): a Gaussian that touched no tile in any
 * view of the plan keeps its parameters and both moments unchanged (its
 * moments do not decay); the others get the update above with the global
 * step count t. */
typedef struct {
    float lr_means, lr_log_scales, lr_quats, lr_opacity, lr_sh_dc, lr_sh_rest;
    float b1, b2, eps;
    int32_t visible_only;
} gs_adam_hparams;
GS_API int gs_preprocess_bwd_adam(const gs_plan *plan, void *ws, gs_params *params, const gs_camera *h_cams,
                                  const gs_params *adam_m, const gs_params *adam_v, const gs_adam_hparams *hp,
                                  int32_t *d_step, void *stream);

/* ------------------------------------------------------------ a6: loss
 * Eq. 5: loss = (1 - lambda) L1 + lambda (1 - SSIM) over all views' colour
 * pixels, SSIM with an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2,
 * C2 = 0.03^2, zero-padded same-size windows, averaged over channels and
 * pixels; L1 = mean absolute difference.  Sec. 3.1: optional disparity term
 * disp_weight * mean |disp - target_disp| (d_disp may be NULL to skip).
 * Writes dL/d(rgb) to d_dL_drgb and, if d_disp is given, dL/d(disp) to
 * d_dL_ddisp (both overwritten), and the scalar loss to d_loss (device, one
 * float).  d_scratch: device float scratch of gs_loss_scratch_floats(plan)
 * (per-block partial sums and a completion counter; a few KB, independent of
 * the pixel count), 8-byte aligned (GS_ERR_ARG otherwise).  Calls sharing
 * one scratch must not overlap on the GPU.  With lambda > 0 the SSIM
 * statistics, maps and gradient are one launch (the last block to finish
 * reduces the loss value); lambda = 0 gives plain L1. */
GS_API int64_t gs_loss_scratch_floats(const gs_plan *plan);
GS_API int gs_loss(const gs_plan *plan, const float *d_rgb, const float *d_target, float lambda,
                   const float *d_disp, const float *d_target_disp, float disp_weight, float *d_dL_drgb,
                   float *d_dL_ddisp, float *d_loss, float *d_scratch, void *stream);

/* ------------------------------------------------------------ a9: Adam
 * Adam with bias correction (the optimiser of the 3DGS training the paper
 * builds on; the paper names none): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps); then g = 0.
 * All arrays device float32 of n elements; step >= 1.  At most 8 groups per
 * call. */
GS_API int gs_adam_step(float *d_p, float *d_g, float *d_m, float *d_v, int64_t n, float lr, float b1,
                        float b2, float eps, int32_t step, void *stream);

/* The same update over several parameter groups in one launch.  Within a
 * group, when period > 0 the first `head` elements of every `period`
 * consecutive elements use lr_head instead of lr (e.g. the DC coefficients
 * of an n x K x 3 SH array: period = 3K, head = 3). */
typedef struct {
    float *p, *g, *m, *v;  /* device */
    int64_t n;
    float lr;
    int64_t period;
    int64_t head;
    float lr_head;
} gs_adam_group;
GS_API int gs_adam_step_multi(const gs_adam_group *h_groups, int32_t n_groups, float b1, float b2,
                              float eps, int32_t step, void *stream);

/* The same update with the step count in device memory, so that a training
 * step captured once in a CUDA graph can be replayed: d_step (device int32,
 * 0 before the first update) is incremented on the stream first, and the
 * incremented value is the t of the bias corrections, evaluated in float32
 * as 1 - b^t = -expm1(t log1p(b - 1)) (b - 1 is exact for b in [0.5, 1)
 * and rounds once below).  b1 and b2 must lie in (0, 1).
 * Two launches; the groups are captured by value. */
GS_API int gs_adam_step_multi_dev(const gs_adam_group *h_groups, int32_t n_groups, float b1, float b2,
                                  float eps, int32_t *d_step, void *stream);

/* -------------------------------------------------- building blocks
 * Stable LSD radix sort of (uint32 key, uint32 value) pairs on bits
 * [begin_bit, end_bit) of the key; used by gs_bin_sort and exported for
 * testing.  n pairs from d_keys_in/d_vals_in are written sorted to
 * d_keys_out/d_vals_out (may not alias the inputs; the inputs are used as
 * ping-pong buffers and are clobbered).  d_scratch: device bytes of
 * gs_sort_scratch_bytes(n). */
GS_API size_t gs_sort_scratch_bytes(int64_t n);
GS_API int gs_sort_pairs_u32(uint32_t *d_keys_in, uint32_t *d_vals_in, uint32_t *d_keys_out,
                             uint32_t *d_vals_out, int64_t n, int32_t begin_bit, int32_t end_bit,
                             void *d_scratch, void *stream);

/* ------------------------------------------ a10: neural-Gaussian decoder
 * Sec. 2.3: anchors with learnable features and a shallow MLP shared by all
 * anchors infer the attributes of the anchors' child Gaussians; only the
 * features (and the anchors' log-scales) and the MLP are trained.  The paper
 * fixes no architecture; this library's decoder is
 *   x = [feature (32), unit view direction anchor - camera centre (3)]
 *   h = ReLU(W1 x + b1) (32),  y = W2 h + b2 (140 = 10 children x 14)
 *   per child (u = its 14 outputs): mean = anchor + tanh(u0..2) e^{s_off},
 *   opacity = tanh(u3) (children with opacity <= 0 are not rendered),
 *   colour = sigmoid(u4..6), log-scale = s_scale + log sigmoid(u7..9),
 *   rotation = u10..13.
 * The GEMMs run on the tensor cores with bf16 operands (features, view
 * direction, weights, h; in the backward dL/dy and dL/dh) and fp32 sums. */
#define GS_NG_FEAT 32
#define GS_NG_HIDDEN 32
#define GS_NG_CHILDREN 10

typedef struct {
    int64_t n_anchors;
    float *anchor_xyz;  /* device, n x 3 (fixed; no gradient) */
    float *feat;        /* device, n x 32 */
    float *anchor_ls;   /* device, n x 6: offset log-scales (3), child log-scales (3) */
    float *w1, *b1;     /* device, 32 x 35 (row-major, output-major), 32 */
    float *w2, *b2;     /* device, 140 x 32, 140 */
} gs_ng_params;

/* Device workspace the decoder needs for n anchors (bf16 weights, the hidden
 * activations kept from the forward for the backward, per-CTA partial sums
 * of the weight gradients, a status word). */
GS_API size_t gs_ng_workspace_bytes(int64_t n_anchors);
/* Decode the children for one camera into `children` (n = 10 * n_anchors,
 * sh_degree 0; arrays overwritten): child i of anchor a is Gaussian 10 a + i,
 * its opacity as a logit (-30 when opacity <= 0) and its colour as the SH DC
 * coefficient (colour - 0.5) * 2 sqrt(pi). */
GS_API int gs_ng_decode_fwd(const gs_ng_params *ng, const gs_camera *h_cam, gs_params *children, void *d_ws,
                            void *stream);
/* Sec. 2.3 with NEXT-4's fusion: gs_ng_decode_fwd and gs_preprocess of the
 * children in one launch.  The decoder's epilogue computes each child's
 * parameters, writes them to `children` (as gs_ng_decode_fwd; the backward
 * reads them) and preprocesses the child from registers into `plan_ws`,
 * exactly as gs_preprocess(plan, plan_ws, children, h_cam) would (same
 * records, tile counts, rectangles and depth keys, bit for bit).  `plan`:
 * one view of h_cam's size, n = children->n, SH degree 0, no pose state
 * attached (GS_ERR_ARG otherwise).  Follow with gs_bin_sort etc. as after
 * gs_preprocess. */
GS_API int gs_ng_decode_preprocess(const gs_ng_params *ng, const gs_camera *h_cam, gs_params *children, void *d_ws,
                                   const gs_plan *plan, void *plan_ws, void *stream);
/* Backward of gs_ng_decode_fwd for the same camera and workspace: maps the
 * children's parameter gradients to the anchors' feature and log-scale
 * gradients and the MLP gradients, ACCUMULATED (+=) into `grads` (its
 * anchor_xyz may be NULL).  With zero_child_grads != 0 the children's
 * gradient arrays are set to zero as they are read (they are accumulators
 * of the splatting backward, so the next step starts from zero without a
 * separate pass); the arrays are written through the pointers in
 * child_grads even though the struct itself is not modified. */
GS_API int gs_ng_decode_bwd(const gs_ng_params *ng, const gs_camera *h_cam, const gs_params *child_grads,
                            int32_t zero_child_grads, gs_ng_params *grads, void *d_ws, void *stream);
/* Synchronise `stream` and read the decoder's device status (GS_ERR_TIMEOUT
 * if a bounded wait for the tensor cores gave up). */
GS_API int gs_ng_read_status(void *d_ws, int32_t *out_error, void *stream);
/* Failure detection of the decoder's bounded waits, checked without a fault:
 * one thread of a one-block launch initialises an mbarrier for one arrival
 * and waits for its first phase with the same bounded wait the tensor-core
 * kernels use, giving up after `limit` tries (1 .. 2^22).  With arrive = 0
 * nothing arrives (no copy and no MMA is in flight), the wait runs out and
 * GS_ERR_TIMEOUT is written to *d_err (device int32, left alone if already
 * non-zero); with arrive = 1 the thread arrives first and *d_err is not
 * touched.  The paper has no counterpart; the kernels it checks are the
 * decoder's (Sec. 2.3).  Returns GS_ERR_ARG for a NULL d_err, a limit
 * outside the range or arrive not 0 or 1. */
GS_API int gs_ng_wait_probe(int32_t *d_err, int64_t limit, int32_t arrive, void *stream);

/* ------------------------------ densification and pruning (Sec. 3.2)
 * Multi-view score-guided densification and pruning, in three calls:
 *
 * gs_densify_score: after gs_render_fwd on a plan (one or more views), add
 *   each view's terms to the per-Gaussian scores.  Eq. 3: the view's error
 *   E(u,v) = sum_c |rgb_c - target_c| divided by its maximum over the view;
 *   mask M = [E / max E > tau].  Eq. 4: d_s_plus[i] += number of masked
 *   pixels of the view that Gaussian i is blended into (same alpha, cut-off
 *   and stop decisions as the forward).  Eq. 6: d_r_minus[i] += that number
 *   times d_photo[v], the view's photometric loss (device float per view of
 *   the plan, e.g. gs_loss of that view alone).  d_rgb, d_target: planar
 *   colour of the plan's views (device).  Scores accumulate (+=).
 *   d_scratch: device bytes of gs_densify_scratch_bytes(n).
 *
 * gs_densify_plan: from the accumulated scores over K views, every
 *   Gaussian's action (d_action[i], one of GS_DENSIFY_*) and its first
 *   output slot (d_offsets[i], int64): s+ = d_s_plus / K; s- = d_r_minus /
 *   max d_r_minus; prune if s- > tau_minus or sigmoid(opacity logit) <
 *   min_opacity; else clone (largest scale <= percent_dense * extent) or
 *   split (larger) if s+ > tau_plus; else keep.  Writes the new Gaussian
 *   count to *out_new_n (host) and synchronises the stream.
 *
 * gs_densify_apply: write the new Gaussian set (parameters and both Adam
 *   moments) into dst, dst_m, dst_v (device arrays with room for the new
 *   count; same SH degree): kept Gaussians are copied with their moments;
 *   a clone adds a copy with zero moments; a split replaces the Gaussian by
 *   two at mean + R diag(s) z_k (z_k: d_normals[6 i + 3 k .. + 3], standard
 *   normal samples supplied by the caller) with scales s / 1.6, the same
 *   rotation, opacity and SH, and zero moments.  Output order follows the
 *   sources.  The paper gives no thresholds or split rule; these are the 3DGS
 *   rules the method builds on. */
enum { GS_DENSIFY_PRUNE = 0, GS_DENSIFY_KEEP = 1, GS_DENSIFY_CLONE = 2, GS_DENSIFY_SPLIT = 3 };
typedef struct {
    float tau_plus;       /* threshold on s+ (masked pixels per view) */
    float tau_minus;      /* threshold on the normalised s- */
    float min_opacity;    /* opacity below which a Gaussian is pruned */
    float percent_dense;  /* clone/split boundary as a fraction of extent */
    float extent;         /* scene extent */
    int32_t k_views;      /* K, the number of views scored */
} gs_densify_rules;
GS_API size_t gs_densify_scratch_bytes(int64_t n);
GS_API int gs_densify_score(const gs_plan *plan, void *ws, const float *d_rgb, const float *d_target, float tau,
                            const float *d_photo, float *d_s_plus, float *d_r_minus, void *d_scratch, void *stream);
GS_API int gs_densify_plan(int64_t n, const gs_params *params, const float *d_s_plus, const float *d_r_minus,
                           const gs_densify_rules *rules, int32_t *d_action, int64_t *d_offsets, void *d_scratch,
                           int64_t *out_new_n, void *stream);
GS_API int gs_densify_apply(int64_t n, const gs_params *src, const gs_params *src_m, const gs_params *src_v,
                            const int32_t *d_action, const int64_t *d_offsets, const float *d_normals,
                            gs_params *dst, gs_params *dst_m, gs_params *dst_v, void *stream);

/* ------------------------------ global pose refinement (Sec. 2.5)
 * One learnable correction (Delta_R, Delta_t) shared by every camera of every
 * plan it is attached to (training and evaluation views alike), applied on
 * the camera side: a camera with world -> camera transform [W | t] is used as
 * [Delta_R W | Delta_R t + Delta_t].  The loss gradient with respect to a
 * left increment xi = (omega, tau) of the correction (the camera then seeing
 * exp([omega]_x) (Delta_R (W p + t) + Delta_t) + tau: omega an axis-angle
 * rotation about the camera centre, tau a translation, both in the camera
 * frame) accumulates over every step; gs_pose_step turns the accumulated sum
 * into one Adam increment and folds it into the correction (the paper does
 * this every 300 iterations).
 *
 * The whole state is one device buffer of GS_POSE_STATE_DOUBLES doubles,
 * owned by the caller, 16-byte aligned:
 *   [0..8]    Delta_R, row-major          [9..11]   Delta_t
 *   [12..17]  Adam first moments of xi    [18..23]  Adam second moments
 *   [24]      Adam step count             [25..31]  unused
 *   [32 + 8 s + k], s < GS_POSE_SLOTS, k < 6: partial sums of dL/d(omega,
 *             tau); the gradient is their sum over s (spread over slots so
 *             that concurrent atomic adds do not queue on one address).
 *
 * gs_pose_init: the identity correction, zero moments, step and sums.
 * gs_plan_set_pose: attach a state to a plan (NULL detaches).  While
 *   attached, gs_preprocess composes the correction with each camera (in
 *   double precision, the corrected transform rounded once to float32, the
 *   camera centre -R^T t computed from the rounded values) into the
 *   workspace, and the preprocess backward (gs_preprocess_bwd,
 *   gs_preprocess_bwd_adam, gs_render_bwd) uses those cameras and adds its
 *   views' dL/d(omega, tau) into the state's sums.  The backward therefore
 *   uses the correction of the step's gs_preprocess.  The plan keeps the
 *   pointer only; the state must outlive its use.  GS_ERR_ARG for a
 *   misaligned state.
 * gs_pose_step: sum the slots into g, then in double precision: t += 1;
 *   m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
 *   xi = -lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps) with lr = lr_rot
 *   for omega and lr_trans for tau; Delta_R <- exp([omega]_x) Delta_R,
 *   Delta_t <- exp([omega]_x) Delta_t + tau; the sums restart from zero. */
#define GS_POSE_SLOTS 256
#define GS_POSE_STATE_DOUBLES (32 + 8 * GS_POSE_SLOTS)
typedef struct {
    double lr_rot, lr_trans; /* Adam rates of omega (radians) and tau (scene units) */
    double b1, b2, eps;      /* b1, b2 in [0.5, 1), eps >= 0 */
} gs_pose_hparams;
GS_API int gs_pose_init(double *d_state, void *stream);
GS_API int gs_plan_set_pose(gs_plan *plan, double *d_state);
GS_API int gs_pose_step(double *d_state, const gs_pose_hparams *hp, void *stream);

/* The same sort for callers that cannot allocate device memory: plug-ins
 * whose host framework owns every byte of device memory through its own
 * pool, code that runs under a fixed device-memory budget, and loops that
 * cannot take cudaMalloc's implicit device synchronisation.  The paper has
 * no counterpart to this entry point; it is a convenience of this library.
 *
 * The caller passes only the key and value buffers (same rules as
 * gs_sort_pairs_u32).  The scratch lives in a static device array inside the
 * library, 609 KiB per GPU that loads the library, held until the process
 * exits.  n may not exceed GS_SORT_NOALLOC_MAX_N (2^31 - 1, the limit of
 * gs_sort_pairs_u32, which this call wraps); larger n returns GS_ERR_ARG
 * before any work is enqueued.  The call makes no allocation: no cudaMalloc,
 * no cudaFree, no allocating library routine.
 *
 * The first call on each device looks up the array's device address with
 * that device current (cudaGetSymbolAddress) and caches it; make that first
 * call before any stream capture.  The cached address does not survive
 * cudaDeviceReset: a process that resets a device must not call this entry
 * point on it again.  All calls on a device share the one array, which
 * keeps the previous call's contents (every pass rewrites it in full, so
 * nothing needs clearing): calls that may overlap on the GPU — on different
 * streams without ordering between them — race on it and must be
 * serialised by the caller. */
#define GS_SORT_NOALLOC_MAX_N 2147483647LL
GS_API int gs_sort_pairs_u32_noalloc(uint32_t *d_keys_in, uint32_t *d_vals_in, uint32_t *d_keys_out,
                                     uint32_t *d_vals_out, int64_t n, int32_t begin_bit,
                                     int32_t end_bit, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
