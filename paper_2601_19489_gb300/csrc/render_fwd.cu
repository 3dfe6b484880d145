// a5: forward blend (Sec. 2.1 renderCUDA) with the 32-splat checkpoints of
// Sec. 2.2.
//
// One CTA of 256 threads per 16x16 tile, one pixel per thread.  The tile's
// depth-sorted instance list is staged in shared memory in batches of 256
// records (each thread gathers one record, 48 bytes, from the per-Gaussian
// record buffer, which stays L2-resident), with the projected mean moved to
// tile-local coordinates once per splat so the per-pair offsets are exact
// to float32 at any image size.  Each pixel blends front to back
// until its transmittance would fall below 1e-4; a warp whose pixels are all
// done skips the rest of the batch and the CTA leaves when all 256 are done.
// Before list positions 0, B, 2B, ... (B = 32 or 64 splats per bucket) every
// pixel still running stores its (T, C, D) in bucket-major, channel-planar
// layout [bucket][5][256] so the backward's warps read them coalesced; a
// tile's ceil(n / B) buckets are taken from a shared counter by its CTA.
#include "gs_internal.cuh"

namespace gs {

__device__ __forceinline__ int view_of_tile(const ViewsDev &vd, int t) {
    int v = 0;
    while (v + 1 < vd.V && t >= vd.v[v + 1].tile_off) ++v;
    return v;
}

__global__ void __launch_bounds__(kTilePix)
k_render_fwd(ViewsDev views, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ inst_item,
             const float4 *__restrict__ rec, int bucket_shift, float bg_r,
             float bg_g, float bg_b, float *__restrict__ out_rgb, float *__restrict__ out_disp,
             float *__restrict__ out_T, uint32_t *__restrict__ n_contrib, uint32_t *__restrict__ tile_maxc,
             float *__restrict__ ckpt, float *__restrict__ final_T, uint32_t *__restrict__ bucket_off,
             StatusDev *st) {
    __shared__ float4 s_r0[kTilePix];
    __shared__ float4 s_r1[kTilePix];
    __shared__ float4 s_r2[kTilePix];
    __shared__ uint32_t s_maxc, s_boff;

    const int t = blockIdx.x;
    const int v = view_of_tile(views, t);
    const ViewDev &cam = views.v[v];
    const int lt = t - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int tid = threadIdx.x;
    const int ix = tx * kTile + (tid & (kTile - 1)), iy = ty * kTile + (tid >> 4);
    const bool inside = ix < cam.W && iy < cam.H;
    // tile-local pixel centre; the staged means are tile-local too
    const float px = (float)(tid & (kTile - 1)) + 0.5f, py = (float)(tid >> 4) + 0.5f;
    const float x0 = (float)(tx * kTile), y0 = (float)(ty * kTile);
    const uint2 range = ranges[t];
    const int n = (int)(range.y - range.x);
    if (final_T && t == 0 && tid < 3) {  // the background, after the last pixel
        const ViewDev &lv = views.v[views.V - 1];
        final_T[lv.pix_off + (int64_t)lv.W * lv.H + tid] = tid == 0 ? bg_r : (tid == 1 ? bg_g : bg_b);
    }
    if (tid == 0) {
        s_maxc = 0;
        // this tile's checkpoint buckets: ceil(n / bucket) consecutive ones,
        // taken from the shared counter (the order of the tiles' ranges does
        // not matter; the backward reads bucket_off)
        if (ckpt) {
            const uint32_t nb = ((uint32_t)n + (1u << bucket_shift) - 1u) >> bucket_shift;
            s_boff = nb ? atomicAdd(&st->n_buckets, nb) : 0u;
            bucket_off[t] = s_boff;
        }
    }
    __syncthreads();
    float *ck = ckpt ? ckpt + (size_t)s_boff * (kCkptCh * kTilePix) + tid : nullptr;

    float T = 1.0f, Cr = 0.f, Cg = 0.f, Cb = 0.f, D = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    for (int b0 = 0; b0 < n; b0 += kTilePix) {
        if (__syncthreads_count(!done) == 0) break;  // also fences the previous batch
        if (b0 + tid < n) {
            const size_t it = inst_item[range.x + b0 + tid];
            float4 r0 = rec[3 * it];
            const float4 r1 = rec[3 * it + 1], r2 = rec[3 * it + 2];
            const float2 m = tile_local_mean(r0, r1.w, r2.w, x0, y0);
            r0.x = m.x;
            r0.y = m.y;
            r0.w = __fmul_rn(2.0f, r0.w);  // staged as 2B (exact)
            s_r0[tid] = r0;
            s_r1[tid] = r1;
            s_r2[tid] = r2;
        }
        __syncthreads();
        const int cnt = min(kTilePix, n - b0);
        const int bucket = 1 << bucket_shift;
        for (int j0 = 0; j0 < cnt; j0 += bucket) {
            if (__all_sync(0xffffffffu, done)) break;
            if (ckpt && !done) {  // checkpoint before list position b0 + j0
                float *c = ck + (size_t)((b0 + j0) >> bucket_shift) * (kCkptCh * kTilePix);
                c[0] = T;
                c[kTilePix] = Cr;
                c[2 * kTilePix] = Cg;
                c[3 * kTilePix] = Cb;
                c[4 * kTilePix] = D;
            }
            const int j1 = min(j0 + bucket, cnt);
            for (int j = j0; j < j1 && !done; ++j) {
                const float4 r0 = s_r0[j], r1 = s_r1[j];
                PairEval e;
                eval_pair_b2(r0, r1, px, py, e);
                if (e.power2 > 0.0f || e.alpha < kAlphaMin) continue;
                const float test_T = T * (1.0f - e.alpha);
                if (test_T < kTStop) {
                    done = true;
                    break;
                }
                const float4 r2 = s_r2[j];
                const float w = e.alpha * T;
                Cr += r2.x * w;
                Cg += r2.y * w;
                Cb += r2.z * w;
                D += r1.z * w;
                T = test_T;
                last = (uint32_t)(b0 + j + 1);
            }
        }
    }
    if (inside) {
        const size_t npix = (size_t)cam.W * cam.H;
        const size_t pix = (size_t)iy * cam.W + ix;
        const size_t base = (size_t)cam.pix_off;
        out_rgb[3 * base + pix] = Cr + T * bg_r;
        out_rgb[3 * base + npix + pix] = Cg + T * bg_g;
        out_rgb[3 * base + 2 * npix + pix] = Cb + T * bg_b;
        out_disp[base + pix] = D;
        out_T[base + pix] = T;
        n_contrib[base + pix] = last;
        if (final_T) final_T[base + pix] = T;
    }
    // tile maximum of n_contrib: buckets at or beyond it have no work
    uint32_t m = last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if ((tid & 31) == 0) atomicMax(&s_maxc, m);
    __syncthreads();
    if (tid == 0) tile_maxc[t] = s_maxc;
}

}  // namespace gs

using namespace gs;

extern "C" int gs_render_fwd(const gs_plan *plan, void *ws, const float *bg, float *out_rgb,
                             float *out_disp, float *out_T, void *stream) {
    if (!plan || !ws || !bg || !out_rgb || !out_disp || !out_T) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const ViewsDev vd = make_views(plan, nullptr);
    StatusDev *st = ws_at<StatusDev>(ws, plan->o_status);
    // the bucket counter restarts with every forward
    int rc = check_cuda(cudaMemsetAsync(&st->n_buckets, 0, sizeof(uint32_t), s));
    if (rc) return rc;
    k_render_fwd<<<plan->total_tiles, kTilePix, 0, s>>>(
        vd, ws_at<uint2>(ws, plan->o_ranges), ws_at<uint32_t>(ws, plan->o_ival[plan->inst_final]),
        ws_at<float4>(ws, plan->o_rec), plan->bucket_shift, bg[0], bg[1], bg[2], out_rgb, out_disp, out_T,
        ws_at<uint32_t>(ws, plan->o_ncontrib), ws_at<uint32_t>(ws, plan->o_tile_maxc),
        plan->bwd_per_pixel ? nullptr : ws_at<float>(ws, plan->o_ckpt),
        plan->bwd_per_pixel ? ws_at<float>(ws, plan->o_final) : nullptr, ws_at<uint32_t>(ws, plan->o_bucket_off),
        st);
    return launch_error();
}
