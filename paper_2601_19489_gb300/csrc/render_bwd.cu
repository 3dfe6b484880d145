// a7: per-Gaussian parallel backward of the blend (Sec. 2.2).
//
// One warp per 32-splat bucket; lane l owns splat k = bucket start + l of the
// tile's list.  The warp walks the tile's pixels as a pipeline: at step s lane
// l handles the s-l th pixel, receiving from lane l-1 (shuffle) the state in
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
// pipeline only steps through pixels the bucket can affect.
#include "gs_internal.cuh"

namespace gs {

constexpr int kBwdWarps = 4;
constexpr int kBwdThreads = kBwdWarps * 32;

struct PixStage {
    float4 g[kTilePix];      // (g_r, g_g, g_b, g_D)
    float2 fin[kTilePix];    // (S_fin, n_contrib as float bits)
    float2 ck[kTilePix];     // checkpoint (T, S) in front of the bucket
    uint8_t pix[kTilePix];   // pixel index within the tile
};

__device__ __forceinline__ int find_tile(const uint32_t *bucket_off, int total_tiles, uint32_t b) {
    int lo = 0, hi = total_tiles;  // bucket_off[lo] <= b < bucket_off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(bucket_off + mid) <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kBwdThreads)
k_render_bwd(ViewsDev views, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ inst_item,
             const float4 *__restrict__ rec, const uint32_t *__restrict__ bucket_off,
             const uint32_t *__restrict__ tile_maxc, const float *__restrict__ ckpt,
             const uint32_t *__restrict__ n_contrib, const float *__restrict__ img_rgb,
             const float *__restrict__ img_disp, const float *__restrict__ dL_drgb,
             const float *__restrict__ dL_ddisp, StatusDev *st, float4 *__restrict__ grad2d) {
    __shared__ PixStage stage[kBwdWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    PixStage &S = stage[warp];
    const uint32_t n_buckets = st->n_buckets;
    const uint32_t lt_mask = (1u << lane) - 1u;

    const uint32_t n_warps = gridDim.x * kBwdWarps;
    for (uint32_t b = blockIdx.x * kBwdWarps + warp; b < n_buckets; b += n_warps) {
        const int t = find_tile(bucket_off, views.total_tiles, b);
        const uint32_t j0 = (b - bucket_off[t]) * kBucket;
        if (j0 >= tile_maxc[t]) continue;  // no pixel blended anything at or after j0
        const uint2 range = ranges[t];
        const int nsplat = min((int)(range.y - range.x) - (int)j0, kBucket);
        const bool valid = lane < nsplat;
        int v = 0;
        while (v + 1 < views.V && t >= views.v[v + 1].tile_off) ++v;
        const ViewDev &cam = views.v[v];
        const int lt = t - cam.tile_off;
        const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
        const size_t npix = (size_t)cam.W * cam.H;
        const size_t base = (size_t)cam.pix_off;
        const float *ckb = ckpt + (size_t)b * (kCkptCh * kTilePix);

        // ---- stage the pixels still running at j0, compacted in pixel order
        int m_total = 0;
        for (int p0 = 0; p0 < kTilePix; p0 += 32) {
            const int p = p0 + lane;
            const int ix = tx * kTile + (p & (kTile - 1)), iy = ty * kTile + (p >> 4);
            bool alive = false;
            uint32_t nc = 0;
            size_t pix = 0;
            if (ix < cam.W && iy < cam.H) {
                pix = (size_t)iy * cam.W + ix;
                nc = n_contrib[base + pix];
                alive = nc > j0;
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, alive);
            if (alive) {
                const int m = m_total + __popc(bal & lt_mask);
                const float gr = dL_drgb[3 * base + pix];
                const float gg = dL_drgb[3 * base + npix + pix];
                const float gb = dL_drgb[3 * base + 2 * npix + pix];
                const float gd = dL_ddisp ? dL_ddisp[base + pix] : 0.0f;
                const float sfin = gr * img_rgb[3 * base + pix] + gg * img_rgb[3 * base + npix + pix] +
                                   gb * img_rgb[3 * base + 2 * npix + pix] +
                                   (dL_ddisp ? gd * img_disp[base + pix] : 0.0f);
                const float sck = gr * ckb[kTilePix + p] + gg * ckb[2 * kTilePix + p] +
                                  gb * ckb[3 * kTilePix + p] + gd * ckb[4 * kTilePix + p];
                S.g[m] = make_float4(gr, gg, gb, gd);
                S.fin[m] = make_float2(sfin, __uint_as_float(nc));
                S.ck[m] = make_float2(ckb[p], sck);
                S.pix[m] = (uint8_t)p;
            }
            m_total += __popc(bal);
        }
        __syncwarp();

        // ---- this lane's splat
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
        uint32_t item = 0;
        if (valid) {
            item = inst_item[range.x + j0 + lane];
            r0 = rec[3 * (size_t)item];
            r1 = rec[3 * (size_t)item + 1];
            r2 = rec[3 * (size_t)item + 2];
            // the same tile-local mean the forward staged
            const float2 m = tile_local_mean(r0, r1.w, r2.w, (float)(tx * kTile), (float)(ty * kTile));
            r0.x = m.x;
            r0.y = m.y;
        }
        const uint32_t k = j0 + (uint32_t)lane;
        float g_mx = 0.f, g_my = 0.f, g_xx = 0.f, g_xy = 0.f, g_yy = 0.f, g_pw = 0.f;
        float g_r = 0.f, g_g = 0.f, g_b = 0.f, g_iz = 0.f;
        float T_out = 0.f, S_out = 0.f;

        for (int s = 0; s < m_total + 31; ++s) {
            float T_in = __shfl_up_sync(0xffffffffu, T_out, 1);
            float S_in = __shfl_up_sync(0xffffffffu, S_out, 1);
            const int m = s - lane;
            if (lane == 0 && m < m_total) {
                const float2 c = S.ck[m];
                T_in = c.x;
                S_in = c.y;
            }
            T_out = T_in;
            S_out = S_in;
            if (valid && m >= 0 && m < m_total) {
                const float2 fin = S.fin[m];
                if (k < __float_as_uint(fin.y)) {
                    const int p = S.pix[m];
                    const float px = (float)(p & (kTile - 1)) + 0.5f, py = (float)(p >> 4) + 0.5f;
                    PairEval e;
                    eval_pair(r0, r1, px, py, e);
                    if (e.power2 <= 0.0f && e.alpha >= kAlphaMin) {
                        const float4 g = S.g[m];
                        const float w = e.alpha * T_in;
                        const float gdot = g.x * r2.x + g.y * r2.y + g.z * r2.z + g.w * r1.z;
                        g_r += w * g.x;
                        g_g += w * g.y;
                        g_b += w * g.z;
                        g_iz += w * g.w;
                        S_out = S_in + w * gdot;
                        T_out = T_in * (1.0f - e.alpha);
                        if (e.raw <= kAlphaMax) {  // the clamp passes no gradient
                            const float dL_da = T_in * gdot - (fin.x - S_out) / (1.0f - e.alpha);
                            const float dpw = dL_da * e.raw;  // dL/dpower (natural log units)
                            g_pw += dpw;
                            g_mx += dpw * (r0.z * e.dx + r0.w * e.dy);
                            g_my += dpw * (r0.w * e.dx + r1.x * e.dy);
                            g_xx += dpw * e.dx * e.dx;
                            g_xy += dpw * e.dx * e.dy;
                            g_yy += dpw * e.dy * e.dy;
                        }
                    }
                }
            }
        }
        if (valid) {
            // power = -(a dx^2 + 2 b dx dy + c dy^2) / 2 and (A, B, C) = kH (a, b, c):
            //   d power / d mx = (A dx + B dy) / kH, d power / d a = -dx^2 / 2, ...
            //   d alpha / d o = alpha_raw / o = dpower-weight / o
            const float inv_o = fast_exp2(-r1.y);
            float4 *gp = grad2d + 3 * (size_t)item;
            atomicAdd(gp, make_float4(g_mx * kInvH, g_my * kInvH, -0.5f * g_xx, -g_xy));
            atomicAdd(gp + 1, make_float4(-0.5f * g_yy, g_pw * inv_o, g_iz, 0.0f));
            atomicAdd(gp + 2, make_float4(g_r, g_g, g_b, 0.0f));
        }
        __syncwarp();
    }
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
    StatusDev *st = ws_at<StatusDev>(ws, plan->o_status);
    float4 *g2d = ws_at<float4>(ws, plan->o_grad2d);
    int rc = check_cuda(cudaMemsetAsync(g2d, 0, (size_t)plan->VN * 3 * sizeof(float4), s));
    if (rc) return rc;
    const ViewsDev vd = make_views(plan, nullptr);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_render_bwd<<<sms * 8, kBwdThreads, 0, s>>>(
        vd, ws_at<uint2>(ws, plan->o_ranges), ws_at<uint32_t>(ws, plan->o_ival[plan->inst_final]),
        ws_at<float4>(ws, plan->o_rec), ws_at<uint32_t>(ws, plan->o_bucket_off),
        ws_at<uint32_t>(ws, plan->o_tile_maxc), ws_at<float>(ws, plan->o_ckpt),
        ws_at<uint32_t>(ws, plan->o_ncontrib), d_rgb, d_disp, d_dL_drgb, d_dL_ddisp, st, g2d);
    return launch_error();
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
