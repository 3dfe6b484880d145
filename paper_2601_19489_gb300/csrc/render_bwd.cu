// a7: per-Gaussian parallel backward of the blend (Sec. 2.2).
//
// A warp takes one checkpoint bucket of the tile's depth-sorted list; each
// lane owns splats of the bucket.  The warp walks the tile's pixels as a
// pipeline: at step s lane l handles the (s - l)th pixel, receiving from lane
// l-1 (shuffle) the state in front of its splats — transmittance T and the
// running sum
//   S = sum_{j<=k} alpha_j T_j (g . rgb_j + g_D / z_j)
// — while lane 0 seeds each pixel from the forward's checkpoint.  With
// S_fin = g . C_out + g_D D_out the pixel's final value, the gradient of the
// pixel loss w.r.t. alpha_k is
//   dL/dalpha_k = T_k (g . rgb_k + g_D / z_k) - (S_fin - S_k) / (1 - alpha_k),
// the front-to-back form of the classic back-to-front recursion.  Gradients
// accumulate in registers over all pixels; each lane then adds its splats'
// 10 values to the per-(view, Gaussian) accumulator with float4 atomics.
// Pixels whose blend ended before the bucket are compacted away first, so the
// pipeline only steps through pixels the bucket can affect.  A CTA of the
// persistent grid claims one work unit at a time from a counter: a tile and a
// chunk of up to 8 of its buckets, in the forward's work classes (heaviest
// tiles first; per-tile work is very uneven).  It stages the tile's
// per-pixel gradients and its warps share the chunk's buckets greedily.
//
// Two kernels:
//   k_render_bwd      32-splat buckets, one splat per lane; each lane walks
//                     the live pixels as one chain or as two interleaved
//                     chains (the list's halves) that hide the shuffle latency.
//   k_render_bwd_pk   64-splat buckets, two adjacent splats per lane, the
//                     pair's arithmetic in packed float32 pairs (f32x2 add,
//                     mul and fma: one issue slot for both splats) and
//                     branch-free: a pair the forward did not blend (beyond
//                     the pixel's last contributor, below 1/255) gets alpha 0
//                     and no gradient, so the lanes never diverge inside a step.
#include "gs_internal.cuh"

namespace gs {

// Per CTA: the current tile's per-pixel data (staged once for all warps) and
// each warp's compacted pixel list for the bucket it is working on.
template <int kWarps>
struct BwdShared {
    float4 g[kTilePix];                       // (g_r, g_g, g_b, g_D), zero outside the image
    float4 fin[kTilePix];                     // (S_fin, n_contrib as bits, tile-local px, py)
    float2 ck[kWarps][kTilePix];              // per warp, compacted: (T, S) in front of its bucket
    uint8_t pix[kWarps][kTilePix];            // per warp, compacted: pixel index in the tile
    uint32_t next;                            // next unclaimed bucket of the tile
    uint2 unit;                               // the work unit this CTA claimed: (tile, chunk)
};

// Stage the tile's per-pixel data: the upstream gradient and
// (S_fin, n_contrib) of every pixel, zero outside the image, with the
// pixel's tile-local centre.
template <int kThreads>
__device__ __forceinline__ void stage_tile_pixels(const ViewDev &cam, int tx, int ty, const float *__restrict__ img_rgb,
                                                  const float *__restrict__ img_disp, const float *__restrict__ dL_drgb,
                                                  const float *__restrict__ dL_ddisp,
                                                  const uint32_t *__restrict__ n_contrib, float4 *sg, float4 *sfin) {
    const size_t npix = (size_t)cam.W * cam.H;
    const size_t base = (size_t)cam.pix_off;
    for (int p = threadIdx.x; p < kTilePix; p += kThreads) {
        const int ix = tx * kTile + (p & (kTile - 1)), iy = ty * kTile + (p >> 4);
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 fin = make_float4(0.f, __uint_as_float(0u), (float)(p & (kTile - 1)) + 0.5f, (float)(p >> 4) + 0.5f);
        if (ix < cam.W && iy < cam.H) {
            const size_t pix = (size_t)iy * cam.W + ix;
            g.x = dL_drgb[3 * base + pix];
            g.y = dL_drgb[3 * base + npix + pix];
            g.z = dL_drgb[3 * base + 2 * npix + pix];
            g.w = dL_ddisp ? dL_ddisp[base + pix] : 0.0f;
            fin.x = g.x * img_rgb[3 * base + pix] + g.y * img_rgb[3 * base + npix + pix] +
                    g.z * img_rgb[3 * base + 2 * npix + pix] + (dL_ddisp ? g.w * img_disp[base + pix] : 0.0f);
            fin.y = __uint_as_float(n_contrib[base + pix]);
        }
        sg[p] = g;
        sfin[p] = fin;
    }
}

// The pixels still running at list position j0 (n_contrib > j0), compacted
// into the warp's list in pixel order, each seeded with the checkpoint of
// its bucket: T in front of j0 and X = S(j0) = g . C + g_D D in front of j0
// for the first bucket, X = S(j0) - S_fin for the others (see bwd_pair).
// Returns their number.
__device__ __forceinline__ int compact_live(const float4 *sg, const float4 *sfin, const float *__restrict__ ckb,
                                           uint32_t j0, float2 *ck, uint8_t *pix) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    int m_total = 0;
    for (int p0 = 0; p0 < kTilePix; p0 += 32) {
        const int p = p0 + lane;
        const bool alive = __float_as_uint(sfin[p].y) > j0;
        const uint32_t bal = __ballot_sync(0xffffffffu, alive);
        if (alive) {
            const int m = m_total + __popc(bal & lt_mask);
            const float4 g = sg[p];
            const float sck = g.x * ckb[kTilePix + p] + g.y * ckb[2 * kTilePix + p] + g.z * ckb[3 * kTilePix + p] +
                              g.w * ckb[4 * kTilePix + p];
            ck[m] = make_float2(ckb[p], j0 == 0 ? sck : sck - sfin[p].x);
            pix[m] = (uint8_t)p;
        }
        m_total += __popc(bal);
    }
    __syncwarp();
    return m_total;
}

// The next work unit of the backward, (tile, chunk of kBwdChunk buckets):
// claim number i from the counter, mapped through the forward's per-class
// lists (class 0 first); x = all ones once every unit is taken.
__device__ __forceinline__ uint2 claim_unit(uint32_t *unit_ctr, const uint2 *__restrict__ units,
                                            const uint32_t *class_count, int64_t unit_cap) {
    const uint32_t i = atomicAdd(unit_ctr, 1u);
    uint32_t base = 0;
    for (int c = 0; c < kTileClasses; ++c) {
        const uint32_t n = class_count[c];
        if (i < base + n) return units[(size_t)c * unit_cap + (i - base)];
        base += n;
    }
    return make_uint2(0xffffffffu, 0u);
}

// Per-splat sums over its pixels; the mean's gradient is linear in
// (dx, dy) with the splat's conic as coefficients, so only sx = sum dpw dx
// and sy = sum dpw dy are accumulated and the conic is applied once.
struct SplatGrad {
    float sx, sy, xx, xy, yy, pw, r, g, b, iz;
};

// One (splat, pixel) pair of the pipeline: T, X enter as the state in front
// of the splat and leave as the state behind it.  X runs as S + const: in
// the first bucket X = S and the value behind the splat is S_fin - X; in
// later buckets X = S - S_fin (seeded from the checkpoint) and the value
// behind is -X.  Both are the same quantity; the second keeps the running
// sum at the size of what is still behind, so its float32 rounding shrinks
// as the pixel saturates instead of growing with everything in front.
__device__ __forceinline__ void bwd_pair(const float4 *__restrict__ sg, const float4 *__restrict__ sfin,
                                         const uint8_t *__restrict__ spix, int m, uint32_t k, const float4 &r0,
                                         const float4 &r1, const float4 &r2, bool first, float &T, float &Sv,
                                         SplatGrad &acc) {
    const int p = spix[m];
    const float2 fin = make_float2(sfin[p].x, sfin[p].y);
    if (k >= __float_as_uint(fin.y)) return;  // beyond this pixel's last blended splat
    PairEval e;
    eval_pair(r0, r1, (float)(p & (kTile - 1)) + 0.5f, (float)(p >> 4) + 0.5f, e);
    if (e.power2 > 0.0f || e.alpha < kAlphaMin) return;
    const float4 g = sg[p];
    const float w = e.alpha * T;
    const float gdot = g.x * r2.x + g.y * r2.y + g.z * r2.z + g.w * r1.z;
    acc.r += w * g.x;
    acc.g += w * g.y;
    acc.b += w * g.z;
    acc.iz += w * g.w;
    const float S_in = Sv;
    Sv = S_in + w * gdot;
    if (e.raw <= kAlphaMax) {  // the clamp passes no gradient
        const float dL_da = T * gdot - __fdividef((first ? fin.x : 0.0f) - Sv, 1.0f - e.alpha);
        const float dpw = dL_da * e.raw;  // dL/dpower (natural log units)
        const float sx = dpw * e.dx, sy = dpw * e.dy;
        acc.pw += dpw;
        acc.sx += sx;
        acc.sy += sy;
        acc.xx += sx * e.dx;
        acc.xy += sx * e.dy;
        acc.yy += sy * e.dy;
    }
    T = T * (1.0f - e.alpha);
}

template <int kWarps>
__global__ void __launch_bounds__(kWarps * 32)
k_render_bwd(ViewsDev views, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ inst_item,
             const float4 *__restrict__ rec, const uint32_t *__restrict__ bucket_off,
             const uint32_t *__restrict__ tile_maxc, const float *__restrict__ ckpt,
             const uint32_t *__restrict__ n_contrib, const float *__restrict__ img_rgb,
             const float *__restrict__ img_disp, const float *__restrict__ dL_drgb,
             const float *__restrict__ dL_ddisp, float4 *__restrict__ grad2d, int two_chain_min,
             uint32_t *__restrict__ tile_ctr, const uint2 *__restrict__ tile_order,
             const uint32_t *__restrict__ class_count, int64_t unit_cap) {
    constexpr int kThreads = kWarps * 32;
    constexpr int kBucketSplats = 32;
    __shared__ BwdShared<kWarps> S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint8_t *spix = S.pix[warp];

    for (;;) {
        // tiles are claimed one at a time from a counter, in the forward's
        // work classes (heaviest first): per-tile work is uneven, so a CTA
        // that finishes a light tile takes the next one, and the longest
        // tiles do not come last
        if (threadIdx.x == 0) S.unit = claim_unit(tile_ctr, tile_order, class_count, unit_cap);
        __syncthreads();
        const uint2 unit = S.unit;
        __syncthreads();  // every thread has read S.unit before the next claim
        if (unit.x >= (uint32_t)views.total_tiles) break;
        const int t = (int)unit.x;
        const uint32_t lb0 = unit.y * kBwdChunk;  // this unit's buckets: lb0 .. lb0 + kBwdChunk - 1
        const uint2 range = ranges[t];
        const uint32_t maxc = min(tile_maxc[t], range.y - range.x);
        const uint32_t nb = (maxc + kBucketSplats - 1) / kBucketSplats;  // buckets that hold blended splats
        const uint32_t lb_end = min(nb, lb0 + kBwdChunk);
        if (lb0 >= lb_end) continue;  // uniform
        int v = 0;
        while (v + 1 < views.V && t >= views.v[v + 1].tile_off) ++v;
        const ViewDev &cam = views.v[v];
        const int lt = t - cam.tile_off;
        const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
        stage_tile_pixels<kThreads>(cam, tx, ty, img_rgb, img_disp, dL_drgb, dL_ddisp, n_contrib, S.g, S.fin);
        if (threadIdx.x == 0) S.next = lb0 + kWarps;  // buckets lb0 .. lb0 + kWarps - 1 are taken
        __syncthreads();

        // ---- the warps take the tile's buckets greedily (the first, fullest
        // buckets first) without synchronising until the tile is done
        for (uint32_t lb = lb0 + warp; lb < lb_end;) {
            const uint32_t j0 = lb * kBucketSplats;
            const float *ckb = ckpt + (size_t)(bucket_off[t] + lb) * (kCkptCh * kTilePix);
            const int m_total = compact_live(S.g, S.fin, ckb, j0, S.ck[warp], S.pix[warp]);
            const int h = (m_total + 1) >> 1;
            const float2 *ck_in = S.ck[warp];
            const int nsplat = min((int)(range.y - range.x) - (int)j0, 32);
            // this lane's splat, in the tile-local frame of the forward
            const bool valid = lane < nsplat;
            float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
            uint32_t item = 0;
            if (valid) {
                item = inst_item[range.x + j0 + lane];
                r0 = rec[3 * (size_t)item];
                r1 = rec[3 * (size_t)item + 1];
                r2 = rec[3 * (size_t)item + 2];
                const float2 mm = tile_local_mean(r0, r1.w, r2.w, (float)(tx * kTile), (float)(ty * kTile));
                r0.x = mm.x;
                r0.y = mm.y;
            }
            const uint32_t k = j0 + (uint32_t)lane;
            SplatGrad acc = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (m_total >= two_chain_min) {
                // two independent pixel chains (first and second half of
                // the compacted list) interleave to hide the shuffle
                // latency; the pipeline fills and drains over 31 steps
                float TA = 0.f, SA = 0.f, TB = 0.f, SB = 0.f;
                for (int s = 0; s < h + 31; ++s) {
                    float tA = __shfl_up_sync(0xffffffffu, TA, 1);
                    float sA = __shfl_up_sync(0xffffffffu, SA, 1);
                    float tB = __shfl_up_sync(0xffffffffu, TB, 1);
                    float sB = __shfl_up_sync(0xffffffffu, SB, 1);
                    const int mA = s - lane, mB = h + s - lane;
                    if (lane == 0) {
                        if (mA < h) {
                            const float2 c = ck_in[mA];
                            tA = c.x;
                            sA = c.y;
                        }
                        if (mB < m_total) {
                            const float2 c = ck_in[mB];
                            tB = c.x;
                            sB = c.y;
                        }
                    }
                    TA = tA;
                    SA = sA;
                    TB = tB;
                    SB = sB;
                    if (valid && mA >= 0) {
                        if (mA < h) bwd_pair(S.g, S.fin, spix, mA, k, r0, r1, r2, j0 == 0, TA, SA, acc);
                        if (mB < m_total) bwd_pair(S.g, S.fin, spix, mB, k, r0, r1, r2, j0 == 0, TB, SB, acc);
                    }
                }
            } else {
                // one chain over the whole list: fewer idle lane-steps
                // while the pipeline fills and drains, which pays when
                // few pixels are still running
                float TA = 0.f, SA = 0.f;
                for (int s = 0; s < m_total + 31; ++s) {
                    float tA = __shfl_up_sync(0xffffffffu, TA, 1);
                    float sA = __shfl_up_sync(0xffffffffu, SA, 1);
                    const int mA = s - lane;
                    if (lane == 0 && mA < m_total) {
                        const float2 c = ck_in[mA];
                        tA = c.x;
                        sA = c.y;
                    }
                    TA = tA;
                    SA = sA;
                    if (valid && mA >= 0 && mA < m_total) bwd_pair(S.g, S.fin, spix, mA, k, r0, r1, r2, j0 == 0, TA, SA, acc);
                }
            }
            if (valid) {
                // power = -(a dx^2 + 2 b dx dy + c dy^2) / 2 and (A, B, C) = kH (a, b, c):
                //   d power / d mx = (A dx + B dy) / kH, d power / d a = -dx^2 / 2, ...
                //   d alpha / d o = alpha_raw / o, so dL/do = sum(dL/dpower) / o
                const float inv_o = fast_exp2(-r1.y);
                float4 *gp = grad2d + 3 * (size_t)item;
                const float gmx = (r0.z * acc.sx + r0.w * acc.sy) * kInvH;
                const float gmy = (r0.w * acc.sx + r1.x * acc.sy) * kInvH;
                atomicAdd(gp, make_float4(gmx, gmy, -0.5f * acc.xx, -acc.xy));
                atomicAdd(gp + 1, make_float4(-0.5f * acc.yy, acc.pw * inv_o, acc.iz, 0.0f));
                atomicAdd(gp + 2, make_float4(acc.r, acc.g, acc.b, 0.0f));
            }
            uint32_t next = 0;
            if (lane == 0) next = atomicAdd(&S.next, 1u);
            lb = __shfl_sync(0xffffffffu, next, 0);
        }
        __syncthreads();  // the next tile overwrites the staging
    }
}

// The pixels still running at list position j0, compacted for the 64-splat
// pipeline in four groups by how far into the bucket they run (n_contrib >
// j0 + 48 first, then > j0 + 32, > j0 + 16, the rest), each group in pixel
// order.  A pixel that stops early in the bucket only needs the first lanes
// (lane l owns positions j0 + 2l, j0 + 2l + 1), so with the short-lived
// pixels last the pipeline drains in fewer steps.  Returns the live count and
// in *steps the number of pipeline steps: max over the list of m + (last
// lane the pixel needs) + 1.
__device__ __forceinline__ int compact_live_grouped(const float4 *sg, const float4 *sfin, const float *__restrict__ ckb,
                                                   uint32_t j0, float2 *ck, uint8_t *pix, int *steps) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    int m_total = 0, need = 0;
#pragma unroll 1
    for (int grp = 3; grp >= 0; --grp) {
        for (int p0 = 0; p0 < kTilePix; p0 += 32) {
            const int p = p0 + lane;
            const uint32_t nc = __float_as_uint(sfin[p].y);
            const bool alive = nc > j0 && min(3u, (nc - j0 - 1u) >> 4) == (uint32_t)grp;
            const uint32_t bal = __ballot_sync(0xffffffffu, alive);
            if (alive) {
                const int m = m_total + __popc(bal & lt_mask);
                const float4 g = sg[p];
                const float sck = g.x * ckb[kTilePix + p] + g.y * ckb[2 * kTilePix + p] +
                                  g.z * ckb[3 * kTilePix + p] + g.w * ckb[4 * kTilePix + p];
                ck[m] = make_float2(ckb[p], j0 == 0 ? sck : sck - sfin[p].x);
                pix[m] = (uint8_t)p;
                need = max(need, m + (int)min(31u, (nc - j0 - 1u) >> 1) + 1);
            }
            m_total += __popc(bal);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) need = max(need, __shfl_xor_sync(0xffffffffu, need, o));
    __syncwarp();
    *steps = need;
    return m_total;
}

// ---------------------------------------------------- packed 64-splat kernel

#ifndef GS_BWD_PK_MINB
#define GS_BWD_PK_MINB 12
#endif
template <int kWarps>
__global__ void __launch_bounds__(kWarps * 32, GS_BWD_PK_MINB * 2 / kWarps > 0 ? GS_BWD_PK_MINB * 2 / kWarps : 1)
k_render_bwd_pk(ViewsDev views, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ inst_item,
                const float4 *__restrict__ rec, const uint32_t *__restrict__ bucket_off,
                const uint32_t *__restrict__ tile_maxc, const float *__restrict__ ckpt,
                const uint32_t *__restrict__ n_contrib, const float *__restrict__ img_rgb,
                const float *__restrict__ img_disp, const float *__restrict__ dL_drgb,
                const float *__restrict__ dL_ddisp, float4 *__restrict__ grad2d, uint32_t *__restrict__ tile_ctr,
                const uint2 *__restrict__ tile_order, const uint32_t *__restrict__ class_count, int64_t unit_cap) {
    constexpr int kThreads = kWarps * 32;
    constexpr int kBucketSplats = 64;
    __shared__ BwdShared<kWarps> S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint8_t *spix = S.pix[warp];
    const f2x kZero2 = pk2(0.f, 0.f);

    for (;;) {
        // tiles are claimed one at a time from a counter, in the forward's
        // work classes (heaviest first): per-tile work is uneven, so a CTA
        // that finishes a light tile takes the next one, and the longest
        // tiles do not come last
        if (threadIdx.x == 0) S.unit = claim_unit(tile_ctr, tile_order, class_count, unit_cap);
        __syncthreads();
        const uint2 unit = S.unit;
        __syncthreads();  // every thread has read S.unit before the next claim
        if (unit.x >= (uint32_t)views.total_tiles) break;
        const int t = (int)unit.x;
        const uint32_t lb0 = unit.y * kBwdChunk;  // this unit's buckets: lb0 .. lb0 + kBwdChunk - 1
        const uint2 range = ranges[t];
        const uint32_t maxc = min(tile_maxc[t], range.y - range.x);
        const uint32_t nb = (maxc + kBucketSplats - 1) / kBucketSplats;
        const uint32_t lb_end = min(nb, lb0 + kBwdChunk);
        if (lb0 >= lb_end) continue;  // uniform
        int v = 0;
        while (v + 1 < views.V && t >= views.v[v + 1].tile_off) ++v;
        const ViewDev &cam = views.v[v];
        const int lt = t - cam.tile_off;
        const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
        stage_tile_pixels<kThreads>(cam, tx, ty, img_rgb, img_disp, dL_drgb, dL_ddisp, n_contrib, S.g, S.fin);
        if (threadIdx.x == 0) S.next = lb0 + kWarps;
        __syncthreads();

        for (uint32_t lb = lb0 + warp; lb < lb_end;) {
            const uint32_t j0 = lb * kBucketSplats;
            const float *ckb = ckpt + (size_t)(bucket_off[t] + lb) * (kCkptCh * kTilePix);
            int n_steps = 0;
            const int m_total = compact_live_grouped(S.g, S.fin, ckb, j0, S.ck[warp], S.pix[warp], &n_steps);
            const float2 *ck_in = S.ck[warp];
            // this lane's splats: list positions kA = j0 + 2 lane and kA + 1.
            // A position beyond the tile's list is beyond every pixel's last
            // contributor, so the n_contrib test masks it; its record is zero.
            const uint32_t kA = j0 + 2u * (uint32_t)lane;
            const uint32_t len = range.y - range.x;
            const bool validA = kA < len, validB = kA + 1 < len;
            float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, b0 = a0, b1 = a0, b2 = a0;
            uint32_t itemA = 0, itemB = 0;
            const float x0 = (float)(tx * kTile), y0 = (float)(ty * kTile);
            if (validA) {
                itemA = inst_item[range.x + kA];
                a0 = rec[3 * (size_t)itemA];
                a1 = rec[3 * (size_t)itemA + 1];
                a2 = rec[3 * (size_t)itemA + 2];
                const float2 mm = tile_local_mean(a0, a1.w, a2.w, x0, y0);
                a0.x = mm.x;
                a0.y = mm.y;
            }
            if (validB) {
                itemB = inst_item[range.x + kA + 1];
                b0 = rec[3 * (size_t)itemB];
                b1 = rec[3 * (size_t)itemB + 1];
                b2 = rec[3 * (size_t)itemB + 2];
                const float2 mm = tile_local_mean(b0, b1.w, b2.w, x0, y0);
                b0.x = mm.x;
                b0.y = mm.y;
            }
            const f2x MX = pk2(a0.x, b0.x), MY = pk2(a0.y, b0.y);
            const f2x CA = pk2(a0.z, b0.z), CB2 = pk2(2.0f * a0.w, 2.0f * b0.w), CC = pk2(a1.x, b1.x);
            const f2x LO = pk2(a1.y, b1.y), IZ = pk2(a1.z, b1.z);
            const f2x CR = pk2(a2.x, b2.x), CG = pk2(a2.y, b2.y), CBL = pk2(a2.z, b2.z);
            f2x acc_r = kZero2, acc_g = kZero2, acc_b = kZero2, acc_iz = kZero2, acc_pw = kZero2;
            f2x acc_sx = kZero2, acc_sy = kZero2, acc_xx = kZero2, acc_xy = kZero2, acc_yy = kZero2;
            float T = 0.f, Sv = 0.f;
            for (int s = 0; s < n_steps; ++s) {
                float t_in = __shfl_up_sync(0xffffffffu, T, 1);
                float s_in = __shfl_up_sync(0xffffffffu, Sv, 1);
                const int m = s - lane;
                if (lane == 0 && m < m_total) {
                    const float2 c = ck_in[m];
                    t_in = c.x;
                    s_in = c.y;
                }
                if (m >= 0 && m < m_total) {  // false only while the pipeline fills and drains
                    const int p = spix[m];
                    const float4 fin = S.fin[p];
                    const float4 g = S.g[p];
                    const uint32_t nc = __float_as_uint(fin.y);
                    const float fsel = j0 == 0 ? fin.x : 0.0f;  // X = S or S - S_fin (bwd_pair)
                    const f2x dx = sub2(pk2(fin.z, fin.z), MX), dy = sub2(pk2(fin.w, fin.w), MY);
                    // q = A dx^2 + 2B dx dy + C dy^2 (base 2), e = log2 o - q
                    const f2x q = fma2(fma2(CA, dx, mul2(CB2, dy)), dx, mul2(mul2(CC, dy), dy));
                    float eA, eB, qA, qB;
                    upk2(sub2(LO, q), eA, eB);
                    upk2(q, qA, qB);
                    const float rawA = fast_exp2(eA), rawB = fast_exp2(eB);
                    // the forward's decisions, bit for bit: its alpha is
                    // min(0.99, 2^(log2 o - q)) from the same float32 operations
                    // (it skips power = -q > 0 and alpha < 1/255)
                    const float cA = fminf(kAlphaMax, rawA), cB = fminf(kAlphaMax, rawB);
                    const bool okA = kA < nc && !(qA < 0.0f) && !(cA < kAlphaMin);
                    const bool okB = kA + 1 < nc && !(qB < 0.0f) && !(cB < kAlphaMin);
                    const float aA = okA ? cA : 0.0f;
                    const float aB = okB ? cB : 0.0f;
                    const f2x gx = pk2(g.x, g.x), gy = pk2(g.y, g.y), gz = pk2(g.z, g.z), gw = pk2(g.w, g.w);
                    float gdA, gdB;
                    upk2(fma2(gx, CR, fma2(gy, CG, fma2(gz, CBL, mul2(gw, IZ)))), gdA, gdB);
                    // the chain through the two splats; T advances as
                    // T (1 - alpha), the forward's own float32 operation, so
                    // the backward walks the forward's transmittances
                    const float omA = 1.0f - aA, omB = 1.0f - aB;
                    const float wA = aA * t_in;
                    const float SA = fmaf(wA, gdA, s_in);
                    const float TA = t_in * omA;
                    const float wB = aB * TA;
                    const float SB = fmaf(wB, gdB, SA);
                    T = TA * omB;
                    Sv = SB;
                    const f2x W = pk2(wA, wB);
                    acc_r = fma2(W, gx, acc_r);
                    acc_g = fma2(W, gy, acc_g);
                    acc_b = fma2(W, gz, acc_b);
                    acc_iz = fma2(W, gw, acc_iz);
                    // dL/dpower = dL/dalpha alpha_raw; zero where the clamp is
                    // active or the pair was not blended
                    const float dA = fmaf(t_in, gdA, (SA - fsel) * fast_rcp(omA));
                    const float dB = fmaf(TA, gdB, (SB - fsel) * fast_rcp(omB));
                    const float pA = (okA && rawA <= kAlphaMax) ? dA * rawA : 0.0f;
                    const float pB = (okB && rawB <= kAlphaMax) ? dB * rawB : 0.0f;
                    const f2x dpw = pk2(pA, pB);
                    const f2x sx = mul2(dpw, dx), sy = mul2(dpw, dy);
                    acc_pw = add2(acc_pw, dpw);
                    acc_sx = fma2(dpw, dx, acc_sx);  // the mean's sums without the rounding of sx, sy
                    acc_sy = fma2(dpw, dy, acc_sy);
                    acc_xx = fma2(sx, dx, acc_xx);
                    acc_xy = fma2(sx, dy, acc_xy);
                    acc_yy = fma2(sy, dy, acc_yy);
                }
            }
            float r[2], gg[2], bb[2], iz[2], pw[2], sx[2], sy[2], xx[2], xy[2], yy[2];
            upk2(acc_r, r[0], r[1]);
            upk2(acc_g, gg[0], gg[1]);
            upk2(acc_b, bb[0], bb[1]);
            upk2(acc_iz, iz[0], iz[1]);
            upk2(acc_pw, pw[0], pw[1]);
            upk2(acc_sx, sx[0], sx[1]);
            upk2(acc_sy, sy[0], sy[1]);
            upk2(acc_xx, xx[0], xx[1]);
            upk2(acc_xy, xy[0], xy[1]);
            upk2(acc_yy, yy[0], yy[1]);
            // the splats' conic and opacity back from the packed pairs
            float cA[2], cB2[2], cC[2], lo[2];
            upk2(CA, cA[0], cA[1]);
            upk2(CB2, cB2[0], cB2[1]);
            upk2(CC, cC[0], cC[1]);
            upk2(LO, lo[0], lo[1]);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (j == 0 ? !validA : !validB) continue;
                const float inv_o = fast_exp2(-lo[j]);
                const float cb = 0.5f * cB2[j];
                float4 *gp = grad2d + 3 * (size_t)(j == 0 ? itemA : itemB);
                const float gmx = (cA[j] * sx[j] + cb * sy[j]) * kInvH;
                const float gmy = (cb * sx[j] + cC[j] * sy[j]) * kInvH;
                atomicAdd(gp, make_float4(gmx, gmy, -0.5f * xx[j], -xy[j]));
                atomicAdd(gp + 1, make_float4(-0.5f * yy[j], pw[j] * inv_o, iz[j], 0.0f));
                atomicAdd(gp + 2, make_float4(r[j], gg[j], bb[j], 0.0f));
            }
            uint32_t next = 0;
            if (lane == 0) next = atomicAdd(&S.next, 1u);
            lb = __shfl_sync(0xffffffffu, next, 0);
        }
        __syncthreads();
    }
}

// ------------------------------------------------ per-pixel backward (ablation)
// The classic formulation the per-Gaussian backward replaces (Sec. 2.2): a CTA
// per tile, a thread per pixel walking its blended list back to front from
// its last contributor.  With T_final and R = T_final (g . bg) (the part of
// the pixel's value behind every splat), each blended splat k gives
//   T_k = T_{k+1} / (1 - alpha_k),  dL/dalpha_k = T_k gdot_k - R / (1 - alpha_k),
// then R += alpha_k T_k gdot_k.  The lanes of a warp visit the same splat at
// the same time, so its 10 sums are reduced over the warp before one lane's
// atomics.
__device__ __forceinline__ float warp_sum10(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kTilePix)
k_render_bwd_pixel(ViewsDev views, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ inst_item,
                   const float4 *__restrict__ rec, const uint32_t *__restrict__ tile_maxc,
                   const uint32_t *__restrict__ n_contrib, const float *__restrict__ final_T,
                   const float *__restrict__ dL_drgb, const float *__restrict__ dL_ddisp,
                   float4 *__restrict__ grad2d) {
    __shared__ float4 s_r0[kTilePix], s_r1[kTilePix], s_r2[kTilePix];
    __shared__ uint32_t s_it[kTilePix];
    const int t = blockIdx.x;
    int v = 0;
    while (v + 1 < views.V && t >= views.v[v + 1].tile_off) ++v;
    const ViewDev &cam = views.v[v];
    const int lt = t - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int ix = tx * kTile + (tid & (kTile - 1)), iy = ty * kTile + (tid >> 4);
    const bool inside = ix < cam.W && iy < cam.H;
    const float px = (float)(tid & (kTile - 1)) + 0.5f, py = (float)(tid >> 4) + 0.5f;
    const float x0 = (float)(tx * kTile), y0 = (float)(ty * kTile);
    const uint2 range = ranges[t];
    const uint32_t maxc = min(tile_maxc[t], range.y - range.x);
    if (maxc == 0) return;  // uniform
    const ViewDev &lv = views.v[views.V - 1];
    const float *bg = final_T + lv.pix_off + (int64_t)lv.W * lv.H;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t last = 0;
    float T = 1.0f, R = 0.0f;
    if (inside) {
        const size_t npix = (size_t)cam.W * cam.H, base = (size_t)cam.pix_off, pix = (size_t)iy * cam.W + ix;
        g = make_float4(dL_drgb[3 * base + pix], dL_drgb[3 * base + npix + pix], dL_drgb[3 * base + 2 * npix + pix],
                        dL_ddisp ? dL_ddisp[base + pix] : 0.0f);
        last = n_contrib[base + pix];
        T = final_T[base + pix];
        R = T * (g.x * bg[0] + g.y * bg[1] + g.z * bg[2]);
    }
    for (int b0 = (int)((maxc - 1) / kTilePix) * kTilePix; b0 >= 0; b0 -= kTilePix) {
        __syncthreads();  // the previous batch is no longer read
        if (b0 + tid < (int)maxc) {
            const uint32_t it = inst_item[range.x + b0 + tid];
            float4 r0 = rec[3 * (size_t)it];
            const float4 r1 = rec[3 * (size_t)it + 1], r2 = rec[3 * (size_t)it + 2];
            const float2 mm = tile_local_mean(r0, r1.w, r2.w, x0, y0);
            r0.x = mm.x;
            r0.y = mm.y;
            s_r0[tid] = r0;
            s_r1[tid] = r1;
            s_r2[tid] = r2;
            s_it[tid] = it;
        }
        __syncthreads();
        for (int j = min(kTilePix, (int)maxc - b0) - 1; j >= 0; --j) {
            const uint32_t k = (uint32_t)(b0 + j);
            SplatGrad acc = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool hit = false;
            const float4 r0 = s_r0[j], r1 = s_r1[j];
            if (k < last) {
                PairEval e;
                eval_pair(r0, r1, px, py, e);
                if (!(e.power2 > 0.0f) && !(e.alpha < kAlphaMin)) {
                    hit = true;
                    const float4 r2 = s_r2[j];
                    T = __fdividef(T, 1.0f - e.alpha);  // transmittance in front of splat k
                    const float w = e.alpha * T;
                    const float gdot = g.x * r2.x + g.y * r2.y + g.z * r2.z + g.w * r1.z;
                    acc.r = w * g.x;
                    acc.g = w * g.y;
                    acc.b = w * g.z;
                    acc.iz = w * g.w;
                    if (e.raw <= kAlphaMax) {
                        const float dL_da = T * gdot - __fdividef(R, 1.0f - e.alpha);
                        const float dpw = dL_da * e.raw;
                        acc.pw = dpw;
                        acc.sx = dpw * e.dx;
                        acc.sy = dpw * e.dy;
                        acc.xx = acc.sx * e.dx;
                        acc.xy = acc.sx * e.dy;
                        acc.yy = acc.sy * e.dy;
                    }
                    R += w * gdot;
                }
            }
            if (__ballot_sync(0xffffffffu, hit) == 0u) continue;  // uniform over the warp
            const float sx = warp_sum10(acc.sx), sy = warp_sum10(acc.sy), xx = warp_sum10(acc.xx);
            const float xy = warp_sum10(acc.xy), yy = warp_sum10(acc.yy), pw = warp_sum10(acc.pw);
            const float cr = warp_sum10(acc.r), cg = warp_sum10(acc.g), cb = warp_sum10(acc.b);
            const float iz = warp_sum10(acc.iz);
            if (lane == 0) {
                const float inv_o = fast_exp2(-r1.y);
                float4 *gp = grad2d + 3 * (size_t)s_it[j];
                const float gmx = (r0.z * sx + r0.w * sy) * kInvH;
                const float gmy = (r0.w * sx + r1.x * sy) * kInvH;
                atomicAdd(gp, make_float4(gmx, gmy, -0.5f * xx, -xy));
                atomicAdd(gp + 1, make_float4(-0.5f * yy, pw * inv_o, iz, 0.0f));
                atomicAdd(gp + 2, make_float4(cr, cg, cb, 0.0f));
            }
        }
    }
}

template <typename Kernel>
static int persistent_grid(Kernel kernel, int threads) {
    // persistent grid: as many CTAs as fit on the device at once
    int dev = 0, sms = 152, per_sm = 8;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return sms * per_sm;
}

template <int kWarps>
static int launch_bwd(const gs_plan *plan, void *ws, const float *d_rgb, const float *d_disp,
                      const float *d_dL_drgb, const float *d_dL_ddisp, float4 *g2d, cudaStream_t s) {
    const ViewsDev vd = make_views(plan, nullptr);
    StatusDev *st = ws_at<StatusDev>(ws, plan->o_status);
    uint32_t *ctr = &st->bwd_next_tile;
    const uint2 *order = ws_at<uint2>(ws, plan->o_tile_order);
    const uint32_t *ccount = ws_at<uint32_t>(ws, plan->o_tile_count);
    int rc = check_cuda(cudaMemsetAsync(ctr, 0, sizeof(uint32_t), s));
    if (rc) return rc;
    if (plan->bucket == 64) {
        k_render_bwd_pk<kWarps><<<persistent_grid(k_render_bwd_pk<kWarps>, kWarps * 32), kWarps * 32, 0, s>>>(
            vd, ws_at<uint2>(ws, plan->o_ranges), ws_at<uint32_t>(ws, plan->o_ival[plan->inst_final]),
            ws_at<float4>(ws, plan->o_rec), ws_at<uint32_t>(ws, plan->o_bucket_off),
            ws_at<uint32_t>(ws, plan->o_tile_maxc), ws_at<float>(ws, plan->o_ckpt),
            ws_at<uint32_t>(ws, plan->o_ncontrib), d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, ctr, order, ccount,
            plan->unit_cap);
        return launch_error();
    }
    k_render_bwd<kWarps><<<persistent_grid(k_render_bwd<kWarps>, kWarps * 32), kWarps * 32, 0, s>>>(
        vd, ws_at<uint2>(ws, plan->o_ranges), ws_at<uint32_t>(ws, plan->o_ival[plan->inst_final]),
        ws_at<float4>(ws, plan->o_rec), ws_at<uint32_t>(ws, plan->o_bucket_off),
        ws_at<uint32_t>(ws, plan->o_tile_maxc), ws_at<float>(ws, plan->o_ckpt),
        ws_at<uint32_t>(ws, plan->o_ncontrib), d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, plan->two_chain_min, ctr,
        order, ccount, plan->unit_cap);
    return launch_error();
}

int preprocess_bwd(const gs_plan *plan, void *ws, const gs_params *params, const gs_camera *cams,
                   gs_params *grads, cudaStream_t s);
int check_params(const gs_plan *plan, const gs_params *p);
int check_cams(const gs_plan *plan, const gs_camera *cams);

}  // namespace gs

using namespace gs;

extern "C" int gs_render_bwd_blend(const gs_plan *plan, void *ws, const float *d_rgb, const float *d_disp,
                                   const float *d_dL_drgb, const float *d_dL_ddisp, void *stream) {
    if (!plan || !ws || !d_rgb || !d_disp || !d_dL_drgb) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float4 *g2d = ws_at<float4>(ws, plan->o_grad2d);
    int rc = check_cuda(cudaMemsetAsync(g2d, 0, (size_t)plan->VN * 3 * sizeof(float4), s));
    if (rc) return rc;
    if (plan->bwd_per_pixel) {
        const ViewsDev vd = make_views(plan, nullptr);
        k_render_bwd_pixel<<<plan->total_tiles, kTilePix, 0, s>>>(
            vd, ws_at<uint2>(ws, plan->o_ranges), ws_at<uint32_t>(ws, plan->o_ival[plan->inst_final]),
            ws_at<float4>(ws, plan->o_rec), ws_at<uint32_t>(ws, plan->o_tile_maxc),
            ws_at<uint32_t>(ws, plan->o_ncontrib), ws_at<float>(ws, plan->o_final), d_dL_drgb, d_dL_ddisp, g2d);
        return launch_error();
    }
    switch (plan->bwd_warps) {
        case 1: return launch_bwd<1>(plan, ws, d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, s);
        case 2: return launch_bwd<2>(plan, ws, d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, s);
        case 8: return launch_bwd<8>(plan, ws, d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, s);
        default: return launch_bwd<4>(plan, ws, d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, s);
    }
}

extern "C" int gs_preprocess_bwd(const gs_plan *plan, void *ws, const gs_params *params,
                                 const gs_camera *cams, gs_params *grads, void *stream) {
    if (!plan || !ws) return GS_ERR_ARG;
    int rc = check_params(plan, params);
    if (rc) return rc;
    rc = check_params(plan, grads);
    if (rc) return rc;
    rc = check_cams(plan, cams);
    if (rc) return rc;
    return preprocess_bwd(plan, ws, params, cams, grads, (cudaStream_t)stream);
}

extern "C" int gs_render_bwd(const gs_plan *plan, void *ws, const gs_params *params,
                             const gs_camera *cams, const float *bg, const float *d_rgb,
                             const float *d_disp, const float *d_dL_drgb, const float *d_dL_ddisp,
                             gs_params *grads, void *stream) {
    if (!plan || !ws || !bg) return GS_ERR_ARG;
    int rc = check_params(plan, params);
    if (rc) return rc;
    rc = check_params(plan, grads);
    if (rc) return rc;
    rc = check_cams(plan, cams);
    if (rc) return rc;
    // bg enters through the forward's output colour (S_fin), not separately
    rc = gs_render_bwd_blend(plan, ws, d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, stream);
    if (rc) return rc;
    return preprocess_bwd(plan, ws, params, cams, grads, (cudaStream_t)stream);
}
