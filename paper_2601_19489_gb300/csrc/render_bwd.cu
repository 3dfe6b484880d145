// a7: per-Gaussian parallel backward of the blend (Sec. 2.2).
//
// One warp per bucket of 32 (or 64: two passes of 32) splats; lane l owns
// splat k = pass start + l of the tile's list.  The warp walks the tile's
// pixels as a pipeline: at step s lane l handles the s-l th pixel, receiving
// from lane l-1 (shuffle) the state in
// front of its splat — transmittance T and the running sum
//   S = sum_{j<=k} alpha_j T_j (g . rgb_j + g_D / z_j)
// — while lane 0 seeds each pixel from the forward's checkpoint.  With
// S_fin = g . C_out + g_D D_out the pixel's final value, the gradient of the
// pixel loss w.r.t. alpha_k is
//   dL/dalpha_k = T_k (g . rgb_k + g_D / z_k) - (S_fin - S_k) / (1 - alpha_k),
// the front-to-back form of the classic back-to-front recursion.  Gradients
// accumulate in registers over all pixels; each lane then adds its splat's
// 10 values to the per-(view, Gaussian) accumulator with three float4 atomics.
// Pixels whose blend ended before the bucket are compacted away first, so the
// pipeline only steps through pixels the bucket can affect, and the list is
// walked as two interleaved chains (its halves) to hide the shuffle latency.
// A CTA takes one tile at a time, stages the tile's per-pixel gradients once
// and its warps share the tile's buckets round robin.
#include "gs_internal.cuh"

namespace gs {

// Per CTA: the current tile's per-pixel data (staged once for all warps) and
// each warp's compacted pixel list for the bucket it is working on.  With
// 64-splat buckets (kSub = 2 passes of 32) the state behind a pass's last
// splat is carried to the next pass through the second `ck` buffer.
template <int kWarps, int kSub>
struct BwdShared {
    float4 g[kTilePix];                       // (g_r, g_g, g_b, g_D), zero outside the image
    float2 fin[kTilePix];                     // (S_fin, n_contrib as bits)
    float2 ck[kWarps][kSub > 1 ? 2 : 1][kTilePix];  // per warp, compacted: (T, S) in front of its pass
    uint8_t pix[kWarps][kTilePix];            // per warp, compacted: pixel index in the tile
    uint32_t next;                            // next unclaimed bucket of the tile
};

// Per-splat sums over its pixels; the mean's gradient is linear in
// (dx, dy) with the splat's conic as coefficients, so only sx = sum dpw dx
// and sy = sum dpw dy are accumulated and the conic is applied once.
struct SplatGrad {
    float sx, sy, xx, xy, yy, pw, r, g, b, iz;
};

// One (splat, pixel) pair of the pipeline: T, S enter as the state in front
// of the splat and leave as the state behind it.
__device__ __forceinline__ void bwd_pair(const float4 *__restrict__ sg, const float2 *__restrict__ sfin,
                                         const uint8_t *__restrict__ spix, int m, uint32_t k, const float4 &r0,
                                         const float4 &r1, const float4 &r2, float &T, float &Sv,
                                         SplatGrad &acc) {
    const int p = spix[m];
    const float2 fin = sfin[p];
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
        const float dL_da = T * gdot - __fdividef(fin.x - Sv, 1.0f - e.alpha);
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

template <int kWarps, int kSub>
__global__ void __launch_bounds__(kWarps * 32)
k_render_bwd(ViewsDev views, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ inst_item,
             const float4 *__restrict__ rec, const uint32_t *__restrict__ bucket_off,
             const uint32_t *__restrict__ tile_maxc, const float *__restrict__ ckpt,
             const uint32_t *__restrict__ n_contrib, const float *__restrict__ img_rgb,
             const float *__restrict__ img_disp, const float *__restrict__ dL_drgb,
             const float *__restrict__ dL_ddisp, float4 *__restrict__ grad2d, int two_chain_min) {
    constexpr int kThreads = kWarps * 32;
    constexpr int kBucketSplats = 32 * kSub;
    __shared__ BwdShared<kWarps, kSub> S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint8_t *spix = S.pix[warp];

    for (int t = blockIdx.x; t < views.total_tiles; t += gridDim.x) {
        const uint2 range = ranges[t];
        const uint32_t maxc = min(tile_maxc[t], range.y - range.x);
        const uint32_t nb = (maxc + kBucketSplats - 1) / kBucketSplats;  // buckets that hold blended splats
        if (nb == 0) continue;  // uniform
        int v = 0;
        while (v + 1 < views.V && t >= views.v[v + 1].tile_off) ++v;
        const ViewDev &cam = views.v[v];
        const int lt = t - cam.tile_off;
        const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
        const size_t npix = (size_t)cam.W * cam.H;
        const size_t base = (size_t)cam.pix_off;

        // ---- the tile's pixels, shared by the CTA's warps
        for (int p = threadIdx.x; p < kTilePix; p += kThreads) {
            const int ix = tx * kTile + (p & (kTile - 1)), iy = ty * kTile + (p >> 4);
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 fin = make_float2(0.f, __uint_as_float(0u));
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
            S.g[p] = g;
            S.fin[p] = fin;
        }
        if (threadIdx.x == 0) S.next = kWarps;  // buckets 0..kWarps-1 are taken
        __syncthreads();

        // ---- the warps take the tile's buckets greedily (the first, fullest
        // buckets first) without synchronising until the tile is done
        for (uint32_t lb = warp; lb < nb;) {
            const uint32_t j0 = lb * kBucketSplats;
            // pixels still running at j0, compacted, seeded from the checkpoint
            const float *ckb = ckpt + (size_t)(bucket_off[t] + lb) * (kCkptCh * kTilePix);
            int m_total = 0;
            for (int p0 = 0; p0 < kTilePix; p0 += 32) {
                const int p = p0 + lane;
                const bool alive = __float_as_uint(S.fin[p].y) > j0;
                const uint32_t bal = __ballot_sync(0xffffffffu, alive);
                if (alive) {
                    const int m = m_total + __popc(bal & lt_mask);
                    const float4 g = S.g[p];
                    const float sck = g.x * ckb[kTilePix + p] + g.y * ckb[2 * kTilePix + p] +
                                      g.z * ckb[3 * kTilePix + p] + g.w * ckb[4 * kTilePix + p];
                    S.ck[warp][0][m] = make_float2(ckb[p], sck);
                    S.pix[warp][m] = (uint8_t)p;
                }
                m_total += __popc(bal);
            }
            __syncwarp();
            const int h = (m_total + 1) >> 1;

#pragma unroll 1
            for (int sub = 0; sub < kSub; ++sub) {
                const uint32_t js = j0 + 32u * (uint32_t)sub;
                const int nsplat = min((int)(range.y - range.x) - (int)js, 32);
                if (nsplat <= 0) break;  // uniform
                const float2 *ck_in = S.ck[warp][sub & 1];
                float2 *ck_out = S.ck[warp][(sub + 1) & 1];
                const bool carry = sub + 1 < kSub && lane == 31;
                // this lane's splat, in the tile-local frame of the forward
                const bool valid = lane < nsplat;
                float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
                uint32_t item = 0;
                if (valid) {
                    item = inst_item[range.x + js + lane];
                    r0 = rec[3 * (size_t)item];
                    r1 = rec[3 * (size_t)item + 1];
                    r2 = rec[3 * (size_t)item + 2];
                    const float2 mm = tile_local_mean(r0, r1.w, r2.w, (float)(tx * kTile), (float)(ty * kTile));
                    r0.x = mm.x;
                    r0.y = mm.y;
                }
                const uint32_t k = js + (uint32_t)lane;
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
                            if (mA < h) bwd_pair(S.g, S.fin, spix, mA, k, r0, r1, r2, TA, SA, acc);
                            if (mB < m_total) bwd_pair(S.g, S.fin, spix, mB, k, r0, r1, r2, TB, SB, acc);
                        }
                        // the state behind the pass's last splat seeds the next pass
                        if (carry && mA >= 0) {
                            if (mA < h) ck_out[mA] = make_float2(TA, SA);
                            if (mB < m_total) ck_out[mB] = make_float2(TB, SB);
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
                        const bool live = mA >= 0 && mA < m_total;
                        if (valid && live) bwd_pair(S.g, S.fin, spix, mA, k, r0, r1, r2, TA, SA, acc);
                        if (carry && live) ck_out[mA] = make_float2(TA, SA);
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
                __syncwarp();  // the carried states are visible to lane 0 of the next pass
            }
            uint32_t next = 0;
            if (lane == 0) next = atomicAdd(&S.next, 1u);
            lb = __shfl_sync(0xffffffffu, next, 0);
        }
        __syncthreads();  // the next tile overwrites the staging
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

template <int kWarps, int kSub>
static int launch_bwd(const gs_plan *plan, void *ws, const float *d_rgb, const float *d_disp,
                      const float *d_dL_drgb, const float *d_dL_ddisp, float4 *g2d, cudaStream_t s) {
    const ViewsDev vd = make_views(plan, nullptr);
    // persistent grid: as many CTAs as fit on the device at once
    int dev = 0, sms = 152, per_sm = 8;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_bwd<kWarps, kSub>, kWarps * 32, 0) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    k_render_bwd<kWarps, kSub><<<sms * per_sm, kWarps * 32, 0, s>>>(
        vd, ws_at<uint2>(ws, plan->o_ranges), ws_at<uint32_t>(ws, plan->o_ival[plan->inst_final]),
        ws_at<float4>(ws, plan->o_rec), ws_at<uint32_t>(ws, plan->o_bucket_off),
        ws_at<uint32_t>(ws, plan->o_tile_maxc), ws_at<float>(ws, plan->o_ckpt),
        ws_at<uint32_t>(ws, plan->o_ncontrib), d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, plan->two_chain_min);
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
    const bool two = plan->bucket == 64;
    switch (plan->bwd_warps) {
        case 2: return two ? launch_bwd<2, 2>(plan, ws, d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, s)
                           : launch_bwd<2, 1>(plan, ws, d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, s);
        case 8: return two ? launch_bwd<8, 2>(plan, ws, d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, s)
                           : launch_bwd<8, 1>(plan, ws, d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, s);
        default: return two ? launch_bwd<4, 2>(plan, ws, d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, s)
                            : launch_bwd<4, 1>(plan, ws, d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, g2d, s);
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
