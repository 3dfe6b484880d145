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
             uint2 *__restrict__ tile_order, uint32_t *__restrict__ tile_count, int64_t unit_cap, StatusDev *st) {
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
    if (tid == 0) {
        tile_maxc[t] = s_maxc;
        if (ckpt) {
            // the per-Gaussian backward's work units: the buckets it walks
            // (up to the last contributor) in chunks of kBwdChunk, filed by
            // the tile's work class, heaviest class first
            const uint32_t nbw = (min(s_maxc, (uint32_t)n) + (1u << bucket_shift) - 1u) >> bucket_shift;
            const uint32_t chunks = (nbw + kBwdChunk - 1) / kBwdChunk;
            if (chunks) {
                const int c = tile_work_class(s_maxc);
                uint2 *dst = tile_order + (size_t)c * unit_cap + atomicAdd(&tile_count[c], chunks);
                for (uint32_t k = 0; k < chunks; ++k) dst[k] = make_uint2((uint32_t)t, k);
            }
        }
    }
}


// Two horizontally adjacent pixels per thread (128 threads per tile), their
// pair arithmetic in packed float32 pairs.  Every splat is staged with each
// value duplicated into a pair, so one 16-byte shared load yields two packed
// operands: (mx, mx, my, my) tile-local, (A, A, 2B, 2B), (C, C, log2 o,
// log2 o), (r, r, g, g), (b, b, 1/z, 1/z).  The quadratic form, the exponent,
// the transmittance update and the colour sums of both pixels take one f32x2
// instruction each; every element rounds like the scalar operation, so the
// alpha, cut-off and stop decisions are those of the backward bit for bit.
// The step is branch-free: a pixel whose pair is skipped, or which has
// stopped, gets weight 0 and keeps its transmittance.  A warp (a 16 x 4
// pixel block) leaves a batch when all of its 64 pixels have stopped.
constexpr int kFwdPkThreads = kTilePix / 2;
constexpr int kFwdPkBatch = 2 * kFwdPkThreads;  // records staged per round

__global__ void __launch_bounds__(kFwdPkThreads)
k_render_fwd_pk(ViewsDev views, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ inst_item,
                const float4 *__restrict__ rec, int bucket_shift, float bg_r, float bg_g, float bg_b,
                float *__restrict__ out_rgb, float *__restrict__ out_disp, float *__restrict__ out_T,
                uint32_t *__restrict__ n_contrib, uint32_t *__restrict__ tile_maxc, float *__restrict__ ckpt,
                float *__restrict__ final_T, uint32_t *__restrict__ bucket_off, uint2 *__restrict__ tile_order,
                uint32_t *__restrict__ tile_count, int64_t unit_cap, StatusDev *st) {
    __shared__ ulonglong2 s_q0[kFwdPkBatch], s_q1[kFwdPkBatch], s_q2[kFwdPkBatch];
    __shared__ ulonglong2 s_c0[kFwdPkBatch], s_c1[kFwdPkBatch];
    __shared__ uint32_t s_maxc, s_boff;

    const int t = blockIdx.x;
    const int v = view_of_tile(views, t);
    const ViewDev &cam = views.v[v];
    const int lt = t - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int tid = threadIdx.x;
    const int col = 2 * (tid & 7), row = tid >> 3;  // this thread's pixels: (col, row), (col + 1, row)
    const int ix = tx * kTile + col, iy = ty * kTile + row;
    const bool in0 = ix < cam.W && iy < cam.H, in1 = ix + 1 < cam.W && iy < cam.H;
    const f2x PX = pk2((float)col + 0.5f, (float)col + 1.5f), PY = pk2((float)row + 0.5f, (float)row + 0.5f);
    const f2x kOne2 = pk2(1.0f, 1.0f);
    const float x0 = (float)(tx * kTile), y0 = (float)(ty * kTile);
    const uint2 range = ranges[t];
    const int n = (int)(range.y - range.x);
    if (final_T && t == 0 && tid < 3) {  // the background, after the last pixel
        const ViewDev &lv = views.v[views.V - 1];
        final_T[lv.pix_off + (int64_t)lv.W * lv.H + tid] = tid == 0 ? bg_r : (tid == 1 ? bg_g : bg_b);
    }
    if (tid == 0) {
        s_maxc = 0;
        if (ckpt) {
            const uint32_t nb = ((uint32_t)n + (1u << bucket_shift) - 1u) >> bucket_shift;
            s_boff = nb ? atomicAdd(&st->n_buckets, nb) : 0u;
            bucket_off[t] = s_boff;
        }
    }
    __syncthreads();
    float *ck = ckpt ? ckpt + (size_t)s_boff * (kCkptCh * kTilePix) + 2 * tid : nullptr;

    f2x T2 = kOne2, CR = pk2(0.f, 0.f), CG = CR, CB = CR, DD = CR;
    uint32_t last0 = 0, last1 = 0;
    bool run0 = in0, run1 = in1;
    for (int b0 = 0; b0 < n; b0 += kFwdPkBatch) {
        if (__syncthreads_count(run0 || run1) == 0) break;  // also fences the previous batch
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = tid + h * kFwdPkThreads;
            if (b0 + k < n) {
                const size_t it = inst_item[range.x + b0 + k];
                const float4 r0 = rec[3 * it], r1 = rec[3 * it + 1], r2 = rec[3 * it + 2];
                const float2 m = tile_local_mean(r0, r1.w, r2.w, x0, y0);
                const float b2 = __fmul_rn(2.0f, r0.w);  // 2B (exact)
                s_q0[k] = make_ulonglong2(pk2(m.x, m.x), pk2(m.y, m.y));
                s_q1[k] = make_ulonglong2(pk2(r0.z, r0.z), pk2(b2, b2));
                s_q2[k] = make_ulonglong2(pk2(r1.x, r1.x), pk2(r1.y, r1.y));
                s_c0[k] = make_ulonglong2(pk2(r2.x, r2.x), pk2(r2.y, r2.y));
                s_c1[k] = make_ulonglong2(pk2(r2.z, r2.z), pk2(r1.z, r1.z));
            }
        }
        __syncthreads();
        const int cnt = min(kFwdPkBatch, n - b0);
        const int bucket = 1 << bucket_shift;
        for (int j0 = 0; j0 < cnt; j0 += bucket) {
            if (__all_sync(0xffffffffu, !(run0 || run1))) break;
            if (ckpt && (run0 || run1)) {  // checkpoint before list position b0 + j0
                float T0, T1, r0, r1, g0, g1, bb0, bb1, d0, d1;
                upk2(T2, T0, T1);
                upk2(CR, r0, r1);
                upk2(CG, g0, g1);
                upk2(CB, bb0, bb1);
                upk2(DD, d0, d1);
                float2 *c = reinterpret_cast<float2 *>(ck + (size_t)((b0 + j0) >> bucket_shift) * (kCkptCh * kTilePix));
                c[0] = make_float2(T0, T1);
                c[kTilePix / 2] = make_float2(r0, r1);
                c[kTilePix] = make_float2(g0, g1);
                c[3 * kTilePix / 2] = make_float2(bb0, bb1);
                c[2 * kTilePix] = make_float2(d0, d1);
            }
            const int j1 = min(j0 + bucket, cnt);
            for (int jc = j0; jc < j1; jc += 8) {
                if (__all_sync(0xffffffffu, !(run0 || run1))) break;
                const int je = min(jc + 8, j1);
#pragma unroll 4
                for (int j = jc; j < je; ++j) {
                    const ulonglong2 q0 = s_q0[j], q1 = s_q1[j], q2 = s_q2[j];
                    const f2x dx = sub2(PX, q0.x), dy = sub2(PY, q0.y);
                    // q = A dx^2 + 2B dx dy + C dy^2 (base 2); exponent log2 o - q
                    const f2x q = fma2(fma2(q1.x, dx, mul2(q1.y, dy)), dx, mul2(mul2(q2.x, dy), dy));
                    float e0, e1, qa, qb;
                    upk2(sub2(q2.y, q), e0, e1);
                    upk2(q, qa, qb);
                    const float a0 = fminf(kAlphaMax, fast_exp2(e0)), a1 = fminf(kAlphaMax, fast_exp2(e1));
                    const bool ok0 = run0 && !(qa < 0.0f) && !(a0 < kAlphaMin);
                    const bool ok1 = run1 && !(qb < 0.0f) && !(a1 < kAlphaMin);
                    const f2x A2 = pk2(a0, a1);
                    float tt0, tt1, w0, w1, T0, T1;
                    upk2(mul2(T2, sub2(kOne2, A2)), tt0, tt1);  // test T = T (1 - alpha)
                    upk2(mul2(A2, T2), w0, w1);                 // alpha T
                    upk2(T2, T0, T1);
                    const bool st0 = ok0 && tt0 < kTStop, st1 = ok1 && tt1 < kTStop;
                    const bool bl0 = ok0 && !st0, bl1 = ok1 && !st1;
                    run0 = run0 && !st0;
                    run1 = run1 && !st1;
                    T2 = pk2(bl0 ? tt0 : T0, bl1 ? tt1 : T1);
                    last0 = bl0 ? (uint32_t)(b0 + j + 1) : last0;
                    last1 = bl1 ? (uint32_t)(b0 + j + 1) : last1;
                    const f2x W = pk2(bl0 ? w0 : 0.0f, bl1 ? w1 : 0.0f);
                    const ulonglong2 c0 = s_c0[j], c1 = s_c1[j];
                    CR = fma2(c0.x, W, CR);
                    CG = fma2(c0.y, W, CG);
                    CB = fma2(c1.x, W, CB);
                    DD = fma2(c1.y, W, DD);
                }
            }
        }
    }
    float T0, T1, r0, r1, g0, g1, bb0, bb1, d0, d1;
    upk2(T2, T0, T1);
    upk2(CR, r0, r1);
    upk2(CG, g0, g1);
    upk2(CB, bb0, bb1);
    upk2(DD, d0, d1);
    const size_t npix = (size_t)cam.W * cam.H;
    const size_t base = (size_t)cam.pix_off;
    if (in0) {
        const size_t pix = (size_t)iy * cam.W + ix;
        out_rgb[3 * base + pix] = r0 + T0 * bg_r;
        out_rgb[3 * base + npix + pix] = g0 + T0 * bg_g;
        out_rgb[3 * base + 2 * npix + pix] = bb0 + T0 * bg_b;
        out_disp[base + pix] = d0;
        out_T[base + pix] = T0;
        n_contrib[base + pix] = last0;
        if (final_T) final_T[base + pix] = T0;
    }
    if (in1) {
        const size_t pix = (size_t)iy * cam.W + ix + 1;
        out_rgb[3 * base + pix] = r1 + T1 * bg_r;
        out_rgb[3 * base + npix + pix] = g1 + T1 * bg_g;
        out_rgb[3 * base + 2 * npix + pix] = bb1 + T1 * bg_b;
        out_disp[base + pix] = d1;
        out_T[base + pix] = T1;
        n_contrib[base + pix] = last1;
        if (final_T) final_T[base + pix] = T1;
    }
    uint32_t m = max(last0, last1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if ((tid & 31) == 0) atomicMax(&s_maxc, m);
    __syncthreads();
    if (tid == 0) {
        tile_maxc[t] = s_maxc;
        if (ckpt) {
            // the per-Gaussian backward's work units: the buckets it walks
            // (up to the last contributor) in chunks of kBwdChunk, filed by
            // the tile's work class, heaviest class first
            const uint32_t nbw = (min(s_maxc, (uint32_t)n) + (1u << bucket_shift) - 1u) >> bucket_shift;
            const uint32_t chunks = (nbw + kBwdChunk - 1) / kBwdChunk;
            if (chunks) {
                const int c = tile_work_class(s_maxc);
                uint2 *dst = tile_order + (size_t)c * unit_cap + atomicAdd(&tile_count[c], chunks);
                for (uint32_t k = 0; k < chunks; ++k) dst[k] = make_uint2((uint32_t)t, k);
            }
        }
    }
}

}  // namespace gs

using namespace gs;

extern "C" int gs_render_fwd(const gs_plan *plan, void *ws, const float *bg, float *out_rgb,
                             float *out_disp, float *out_T, void *stream) {
    if (!plan || !ws || !bg || !out_rgb || !out_disp || !out_T) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const ViewsDev vd = make_views(plan, nullptr);
    StatusDev *st = ws_at<StatusDev>(ws, plan->o_status);
    // the bucket counter and the tile classes restart with every forward
    int rc = check_cuda(cudaMemsetAsync(&st->n_buckets, 0, sizeof(uint32_t), s));
    if (rc) return rc;
    rc = check_cuda(cudaMemsetAsync(ws_at<uint32_t>(ws, plan->o_tile_count), 0,
                                    kTileClasses * sizeof(uint32_t), s));
    if (rc) return rc;
    uint32_t *ncontrib = ws_at<uint32_t>(ws, plan->o_ncontrib), *tmaxc = ws_at<uint32_t>(ws, plan->o_tile_maxc);
    float *ck = plan->bwd_per_pixel ? nullptr : ws_at<float>(ws, plan->o_ckpt);
    float *fin = plan->bwd_per_pixel ? ws_at<float>(ws, plan->o_final) : nullptr;
    const uint2 *rg = ws_at<uint2>(ws, plan->o_ranges);
    const uint32_t *items = ws_at<uint32_t>(ws, plan->o_ival[plan->inst_final]);
    const float4 *recs = ws_at<float4>(ws, plan->o_rec);
    uint32_t *boff = ws_at<uint32_t>(ws, plan->o_bucket_off);
    uint2 *order = ws_at<uint2>(ws, plan->o_tile_order);
    uint32_t *tcount = ws_at<uint32_t>(ws, plan->o_tile_count);
    if (plan->fwd_pixels == 2)
        k_render_fwd_pk<<<plan->total_tiles, kFwdPkThreads, 0, s>>>(vd, rg, items, recs, plan->bucket_shift, bg[0],
                                                                     bg[1], bg[2], out_rgb, out_disp, out_T, ncontrib,
                                                                     tmaxc, ck, fin, boff, order, tcount, plan->unit_cap, st);
    else
        k_render_fwd<<<plan->total_tiles, kTilePix, 0, s>>>(vd, rg, items, recs, plan->bucket_shift, bg[0], bg[1],
                                                            bg[2], out_rgb, out_disp, out_T, ncontrib, tmaxc, ck, fin,
                                                            boff, order, tcount, plan->unit_cap, st);
    return launch_error();
}
