// Internal definitions shared by the CUDA translation units of libgs:
// the host plan (workspace layout), the per-view constants passed to kernels
// by value, and the few device functions whose float32 results must be
// bit-identical wherever they are evaluated (the tile-column test used by
// both the tile count and the tile-key write; the alpha evaluation used by
// both the forward blend and the backward).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

constexpr int kTile = GS_TILE;             // 16 x 16 pixel tiles
constexpr int kTilePix = kTile * kTile;    // 256 pixels
constexpr int kBucket = GS_BUCKET;         // default splats per checkpoint
constexpr int kTwoChainAuto = 128;         // automatic chain choice: two chains from 128 live pixels
constexpr int kCkptCh = 5;                 // T, C.r, C.g, C.b, D
constexpr int kTileClasses = 8;            // backward work classes of a tile (by its last contributor)
#ifndef GS_BWD_CHUNK
#define GS_BWD_CHUNK 8
#endif
constexpr int kBwdChunk = GS_BWD_CHUNK;    // buckets per backward work unit (a tile's buckets in chunks)
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTStop = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;
// The stored conic is (a, b, c) * kH so that e^power = 2^(-(A dx^2 + 2 B dx dy + C dy^2)).
constexpr float kH = 0.5f * kLog2e;
constexpr float kInvH = 1.0f / kH;
// Binning uses a level set widened by a relative 2^-10 and an absolute 2^-12
// (in units of t), so every pixel the float32 blend can reach lies in a
// touched tile; the extra tiles only hold pairs with alpha < 1/255.
constexpr float kLevelRel = 1.0f + 1.0f / 1024.0f;
constexpr float kLevelAbs = 1.0f / 4096.0f;
constexpr int kSortBlocks = 608;           // 4 x 152 SMs: fixed grid of the sort/scan passes
constexpr int kBinBlocks = 2432;           // 16 x 152 SMs: fixed grid of the tile-count scan and key write
constexpr int kSortThreads = 256;
constexpr int kBlk = 8;                    // counting binning: blocks of kBlk x kBlk tiles
constexpr int kBlkTiles = kBlk * kBlk;
constexpr int kChunk = 128;                // coarse entries per chunk (one warp)
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

// Per-view constants, copied into kernel parameters by value.
struct ViewDev {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float campos[3];
    float limx, limy, near_z;
    int W, H, tiles_x, tiles_y;
    int tile_off, pix_off;
    int blocks_x, block_off;  // 8 x 8-tile blocks of the counting binning
};

struct ViewsDev {
    int V;
    int total_tiles;
    int total_blocks;
    ViewDev v[GS_MAX_VIEWS];
};

// Device status words at the start of the workspace.
struct StatusDev {
    uint32_t n_inst;      // instances required by the last bin/sort
    uint32_t n_buckets;   // buckets of the last bin/sort
    uint32_t overflow;    // 1 if n_inst > capacity
    int32_t error;        // first device-side error code
    uint32_t done_blocks;  // k_count: blocks finished (cleared with error by gs_bin_sort)
    uint32_t n_coarse;     // (Gaussian, tile block) entries of the counting binning
    uint32_t n_chunks;     // their chunks
    uint32_t done_offsets;  // k_fine_offsets: CTAs finished (cleared by gs_bin_sort)
    uint32_t bwd_next_tile;  // per-Gaussian backward: next unclaimed tile (cleared per launch)
    uint32_t next_mask_chunk;     // k_fine_mask: next unclaimed chunk (cleared by gs_bin_sort)
    uint32_t next_scatter_chunk;  // k_fine_scatter: the same
    uint32_t pad[53];
};

}  // namespace gs

// Workspace layout: byte offsets of every buffer from the workspace base.
struct gs_plan {
    int64_t n;
    int32_t sh_degree, K;
    int32_t V;
    int32_t W[GS_MAX_VIEWS], H[GS_MAX_VIEWS];
    int32_t tiles_x[GS_MAX_VIEWS], tiles_y[GS_MAX_VIEWS];
    int32_t tile_off[GS_MAX_VIEWS + 1];
    int64_t pix_off[GS_MAX_VIEWS + 1];
    int64_t VN;
    int32_t total_tiles;
    int32_t tile_bits;
    int64_t total_pixels;
    int64_t inst_cap;
    int64_t bucket_cap;
    int32_t bucket, bucket_shift;  // splats per checkpoint bucket (32 or 64) and its log2
    int32_t bwd_warps;             // warps per CTA of the per-Gaussian backward
    int32_t two_chain_min;         // live pixels from which a backward bucket walks two chains
    int32_t bbox_3sigma;           // ablation: classic 3-sigma tile box
    int32_t bwd_per_pixel;         // ablation: classic per-pixel backward
    int32_t bin_radix;             // binning by key write + radix sort of the instances
    int32_t fwd_pixels;            // pixels per thread of the forward blend (1, or 2 packed)
    int32_t blocks_x[GS_MAX_VIEWS], block_off[GS_MAX_VIEWS + 1];
    int32_t total_blocks, block_bits;
    int64_t coarse_cap, chunk_cap;
    double *pose;                  // attached pose-refinement state (gs_plan_set_pose) or nullptr
    // offsets
    size_t o_status, o_rec, o_touched, o_rect, o_dkey[2], o_dval[2];
    size_t o_ikey[2], o_ival[2], o_ranges, o_tile_maxc, o_bucket_off, o_ncontrib;
    size_t o_tile_order;  // kTileClasses x unit_cap backward work units (tile, chunk) by class, from the forward
    size_t o_tile_count;  // kTileClasses counts of those lists
    int64_t unit_cap;     // units a class list can hold: tiles + bucket_cap / kBwdChunk
    size_t o_ckpt, o_grad2d, o_sort_scratch, o_block_sums, o_bin;
    size_t o_brange, o_bchunk, o_btile, o_bbase, o_ccnt, o_cval;  // counting binning
    size_t o_final;  // per-pixel final T, then the background (per-pixel backward only)
    size_t o_posed;  // GS_MAX_VIEWS ViewDev: the cameras with the pose correction applied
    size_t sort_scratch_bytes;
    size_t bytes;
    int inst_final;   // which ping-pong buffer holds the sorted instances
    int depth_final;  // which ping-pong buffer holds the depth-sorted ids
};

namespace gs {

template <typename T>
__host__ __device__ inline T *ws_at(void *ws, size_t off) {
    return reinterpret_cast<T *>(reinterpret_cast<char *>(ws) + off);
}

ViewsDev make_views(const gs_plan *plan, const gs_camera *cams);
// GS_OK, or GS_ERR_ARG for a camera that does not match the plan's views.
int check_cams(const gs_plan *plan, const gs_camera *cams);
int check_cuda(cudaError_t e);
int launch_error();

// One-thread launch that increments the device step count of Adam (adam.cu).
int adam_tick(int32_t *d_step, cudaStream_t s);

// Pose refinement (pose.cu): write the plan's cameras with the attached
// correction applied into the workspace (ViewDev array at o_posed).
int pose_compose(const gs_plan *plan, void *ws, const ViewsDev &vd, cudaStream_t s);

// Radix sort internals (radix_sort.cu), usable with a device-resident count.
size_t sort_scratch_bytes();

// Element count of a fixed-grid pass: the host bound, or the device count
// (the tile-instance count is only known on the device) capped by it.
__device__ __forceinline__ int64_t sort_count(int64_t n_host, const uint32_t *n_dev) {
    if (!n_dev) return n_host;
    int64_t n = (int64_t)(*n_dev);
    return n < n_host ? n : n_host;
}
// The lanes of the warp whose digit equals this lane's (digits of nbits
// bits; a lane may pass 1 << nbits as "no digit", which matches only other
// such lanes): one ballot per bit of the digit.
#ifndef GS_RANK_BALLOT
#define GS_RANK_BALLOT 1
#endif
__device__ __forceinline__ uint32_t warp_peers(uint32_t d, int nbits) {
#if GS_RANK_BALLOT
    uint32_t peers = 0xffffffffu;
    for (int b = 0; b <= nbits; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
#else
    (void)nbits;
    return __match_any_sync(0xffffffffu, d);
#endif
}

int sort_pairs(uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b,
               int64_t n_host, const uint32_t *n_dev, int begin_bit, int end_bit, void *scratch,
               cudaStream_t s, int *final_buf);

// ----------------------------------------------------------------------------
// Half extents of the ellipse A dx^2 + 2 B dx dy + C dy^2 <= tb along x and
// y: sqrt(tb C / detc) and sqrt(tb A / detc) (Eq. 2's tangent points, i.e.
// sqrt(t Sxx) and sqrt(t Syy) of the 2D covariance).
__device__ __forceinline__ void ellipse_extent(float A, float C, float detc, float tb, float *rx,
                                               float *ry) {
    *rx = __fsqrt_rn(__fdiv_rn(__fmul_rn(tb, C), detc));
    *ry = __fsqrt_rn(__fdiv_rn(__fmul_rn(tb, A), detc));
}

// Per-Gaussian constants of the tile-column test.
struct BinGeom {
    float mx, my, B, detc, tC, invC, dx_top, rx, ry;
};

__device__ __forceinline__ void bin_geom(float mx, float my, float A, float B, float C, float detc, float tb,
                                         BinGeom &g) {
    ellipse_extent(A, C, detc, tb, &g.rx, &g.ry);
    g.mx = mx;
    g.my = my;
    g.B = B;
    g.detc = detc;
    g.tC = __fmul_rn(tb, C);
    g.invC = __frcp_rn(C);
    g.dx_top = __fdiv_rn(__fmul_rn(-B, g.ry), A);
}

// Tile-column test.  For the tile column [xa, xb] (pixel-centre x range of the
// column, clipped to the image) return the inclusive tile-row range
// [*ty_lo, *ty_hi] whose pixel-centre rectangles meet the ellipse
//   A dx^2 + 2 B dx dy + C dy^2 <= tb,   (dx, dy) = (x - mx, y - my),
// clipped to the rows [ty0, ty1).  With detc = A C - B^2 > 0 the y-range of
// the ellipse over a column is an interval: its top is the concave upper
// branch  (-B dx + sqrt(tb C - detc dx^2)) / C  maximised at the tangent point
// dx = -B ry / A clamped into the column, its bottom the convex lower branch
// minimised at dx = +B ry / A (Eq. 2, with the sign of its radicand
// corrected).  Every operation is an explicitly rounded intrinsic so the tile
// count and the tile-key write compute the same rows.
__device__ __forceinline__ int column_rows(const BinGeom &g, float xa, float xb, float img_h, int ty0, int ty1,
                                           int *ty_lo, int *ty_hi) {
    const float dxa = fmaxf(__fsub_rn(xa, g.mx), -g.rx);
    const float dxb = fminf(__fsub_rn(xb, g.mx), g.rx);
    if (dxa > dxb) return 0;
    float d = fminf(fmaxf(g.dx_top, dxa), dxb);
    float disc = fmaxf(__fsub_rn(g.tC, __fmul_rn(g.detc, __fmul_rn(d, d))), 0.0f);
    float y_hi = __fadd_rn(g.my, __fmul_rn(__fadd_rn(__fmul_rn(-g.B, d), __fsqrt_rn(disc)), g.invC));
    d = fminf(fmaxf(-g.dx_top, dxa), dxb);
    disc = fmaxf(__fsub_rn(g.tC, __fmul_rn(g.detc, __fmul_rn(d, d))), 0.0f);
    float y_lo = __fadd_rn(g.my, __fmul_rn(__fsub_rn(__fmul_rn(-g.B, d), __fsqrt_rn(disc)), g.invC));
    y_lo = fmaxf(y_lo, 0.5f);
    y_hi = fminf(y_hi, __fsub_rn(img_h, 0.5f));
    if (!(y_lo <= y_hi)) return 0;
    int lo = (int)ceilf(__fmul_rn(__fsub_rn(y_lo, 15.5f), 0.0625f));
    int hi = (int)floorf(__fmul_rn(__fsub_rn(y_hi, 0.5f), 0.0625f));
    lo = max(lo, ty0);
    hi = min(hi, ty1 - 1);
    if (lo > hi) return 0;
    *ty_lo = lo;
    *ty_hi = hi;
    return hi - lo + 1;
}

// Tile rectangle [tx0, tx1) x [ty0, ty1) of the SnugBox (pixel-centre bounds
// of the ellipse, clipped to the image).  Returns false when it is empty.
__device__ __forceinline__ bool snug_rect(float mx, float my, float rx, float ry, float img_w,
                                          float img_h, int *tx0, int *ty0, int *tx1, int *ty1) {
    float xl = fmaxf(__fsub_rn(mx, rx), 0.5f), xh = fminf(__fadd_rn(mx, rx), __fsub_rn(img_w, 0.5f));
    float yl = fmaxf(__fsub_rn(my, ry), 0.5f), yh = fminf(__fadd_rn(my, ry), __fsub_rn(img_h, 0.5f));
    if (!(xl <= xh) || !(yl <= yh)) return false;
    *tx0 = (int)ceilf(__fmul_rn(__fsub_rn(xl, 15.5f), 0.0625f));
    *tx1 = (int)floorf(__fmul_rn(__fsub_rn(xh, 0.5f), 0.0625f)) + 1;
    *ty0 = (int)ceilf(__fmul_rn(__fsub_rn(yl, 15.5f), 0.0625f));
    *ty1 = (int)floorf(__fmul_rn(__fsub_rn(yh, 0.5f), 0.0625f)) + 1;
    return *tx0 < *tx1 && *ty0 < *ty1;
}

__device__ __forceinline__ uint2 pack_rect(int tx0, int ty0, int tx1, int ty1) {
    return make_uint2((uint32_t)tx0 | ((uint32_t)ty0 << 16), (uint32_t)tx1 | ((uint32_t)ty1 << 16));
}

__device__ __forceinline__ void unpack_rect(uint2 r, int *tx0, int *ty0, int *tx1, int *ty1) {
    *tx0 = (int)(r.x & 0xffffu);
    *ty0 = (int)(r.x >> 16);
    *tx1 = (int)(r.y & 0xffffu);
    *ty1 = (int)(r.y >> 16);
}

// Pixel-centre x range of tile column tx, clipped to the image width.
__device__ __forceinline__ void column_span(int tx, float img_w, float *xa, float *xb) {
    *xa = (float)(tx * kTile) + 0.5f;
    *xb = fminf((float)(tx * kTile) + 15.5f, __fsub_rn(img_w, 0.5f));
}

// ----------------------------------------------------------------------------
// Alpha of one (splat, pixel) pair, shared by the forward blend and the
// backward so both take identical float32 decisions.
//   r0 = (mx, my, A, B), r1 = (C, log2 o, ...)   (A, B, C = kH * conic)
// with (mx, my) and (px, py) in tile-local pixel coordinates (see
// tile_local_mean), so dx, dy carry no rounding of large image coordinates.
// power2 = -(A dx^2 + 2 B dx dy + C dy^2) is the exponent in base 2; the pair
// is skipped when power2 > 0 (never for a positive-definite conic) and
// alpha = min(0.99, 2^(power2 + log2 o)).
// 2^x with the hardware approximation (PTX ex2.approx.ftz.f32: relative error
// about 2^-22, subnormal results flushed to zero).
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Work class of a tile for the backward, from its largest last-contributor
// position: 0 for >= 4096, one class per halving, 7 below 64.  The backward
// takes the classes in order, heaviest first.
__device__ __forceinline__ int tile_work_class(uint32_t maxc) {
    const int lg = 31 - __clz((int)(maxc | 1u));  // floor(log2(maxc)), 0 for maxc <= 1
    return min(kTileClasses - 1, max(0, 12 - lg));
}

// 1/x with the hardware approximation (PTX rcp.approx.ftz.f32: within one
// ulp of the rounded reciprocal for normal x).
__device__ __forceinline__ float fast_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Tile-local mean: (hi - x0) + lo from the record's compensated mean
// (r0.xy = high parts, r1.w / r2.w = low parts) and the tile origin x0, y0.
__device__ __forceinline__ float2 tile_local_mean(const float4 &r0, float mx_lo, float my_lo, float x0,
                                                  float y0) {
    return make_float2(__fadd_rn(__fsub_rn(r0.x, x0), mx_lo), __fadd_rn(__fsub_rn(r0.y, y0), my_lo));
}

// Packed float32 pairs: two values side by side in one 64-bit register pair,
// so one f32x2 instruction (round to nearest, element by element: the same
// results as the scalar operations) serves both.
typedef unsigned long long f2x;

__device__ __forceinline__ f2x pk2(float a, float b) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f2x r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
    f2x d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
    f2x d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
    f2x d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
    f2x d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
struct PairEval {
    float dx, dy, power2, raw, alpha;
};

// The same evaluation with r0.w already doubled (2B, exact): for records
// staged once and evaluated against many pixels.
__device__ __forceinline__ void eval_pair_b2(const float4 &r0, const float4 &r1, float px, float py,
                                             PairEval &e) {
    e.dx = __fsub_rn(px, r0.x);
    e.dy = __fsub_rn(py, r0.y);
    float u = __fmaf_rn(r0.z, e.dx, __fmul_rn(r0.w, e.dy));  // A dx + 2B dy
    float w = __fmul_rn(__fmul_rn(r1.x, e.dy), e.dy);        // C dy^2
    e.power2 = -__fmaf_rn(u, e.dx, w);
    e.raw = fast_exp2(__fadd_rn(e.power2, r1.y));
    e.alpha = fminf(kAlphaMax, e.raw);
}

__device__ __forceinline__ void eval_pair(const float4 &r0, const float4 &r1, float px, float py,
                                          PairEval &e) {
    float4 q = r0;
    q.w = __fmul_rn(2.0f, r0.w);
    eval_pair_b2(q, r1, px, py, e);
}

}  // namespace gs
