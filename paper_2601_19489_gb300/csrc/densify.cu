// Multi-view score-guided densification and pruning (Sec. 3.2, Eq. 3-6).
//
// Scores (per view, after that view's forward): the view's error image
// E(u, v) = sum_c |R_c - G_c| is normalised by its maximum (one atomic max
// per view) and thresholded into the mask M; then the tile's sorted list is
// blended again exactly as the forward does (same alpha, cut-off and stop
// decisions), and for every splat the warp counts, by ballot, its pixels
// that are masked and that the splat is blended into: one atomic add per
// (warp, splat) gives s+ += count and r- += count * E_photo of the view.
//
// Plan: r- is normalised by its maximum, every Gaussian gets its action
// (prune, keep, clone, split) and its number of results (0, 1, 2, 2), and a
// two-level scan gives each source its first output slot.
//
// Apply: every source writes its results at its slot (kept: copy with its
// Adam moments; clone: the copy plus a duplicate with zero moments; split:
// two Gaussians at mean + R diag(s) z with scales s / 1.6 and zero moments).
#include "gs_internal.cuh"

namespace gs {

constexpr int kScanBlock = 1024;  // Gaussians per block of the result-count scan
constexpr float kLogSplitScale = 0.47000362924573558f;  // ln 1.6: a split child's scale is s / 1.6

// --------------------------------------------------------------- scores
__global__ void __launch_bounds__(256)
k_err_max(ViewsDev views, const float *__restrict__ rgb, const float *__restrict__ target,
          float *__restrict__ emax) {
    const ViewDev &last = views.v[views.V - 1];
    const int64_t total = last.pix_off + (int64_t)last.W * last.H;
    for (int64_t q = (int64_t)blockIdx.x * 256 + threadIdx.x; q < total; q += (int64_t)gridDim.x * 256) {
        int v = 0;
        while (v + 1 < views.V && q >= views.v[v + 1].pix_off) ++v;
        const int64_t npix = (int64_t)views.v[v].W * views.v[v].H, base = views.v[v].pix_off;
        const int64_t p = q - base;
        const float e = fabsf(rgb[3 * base + p] - target[3 * base + p]) +
                        fabsf(rgb[3 * base + npix + p] - target[3 * base + npix + p]) +
                        fabsf(rgb[3 * base + 2 * npix + p] - target[3 * base + 2 * npix + p]);
        // non-negative floats order like their bit patterns
        atomicMax(reinterpret_cast<unsigned int *>(emax) + v, __float_as_uint(e));
    }
}

__global__ void __launch_bounds__(kTilePix)
k_densify_score(ViewsDev views, int64_t n, const uint2 *__restrict__ ranges,
                const uint32_t *__restrict__ inst_item, const float4 *__restrict__ rec, const float *__restrict__ rgb, const float *__restrict__ target,
                const float *__restrict__ emax, float tau, const float *__restrict__ photo,
                float *__restrict__ s_plus, float *__restrict__ r_minus) {
    __shared__ float4 s_r0[kTilePix];
    __shared__ float4 s_r1[kTilePix];
    __shared__ uint32_t s_g[kTilePix];
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
    bool masked = false;
    if (inside) {
        const int64_t npix = (int64_t)cam.W * cam.H, base = cam.pix_off, p = (int64_t)iy * cam.W + ix;
        const float e = fabsf(rgb[3 * base + p] - target[3 * base + p]) +
                        fabsf(rgb[3 * base + npix + p] - target[3 * base + npix + p]) +
                        fabsf(rgb[3 * base + 2 * npix + p] - target[3 * base + 2 * npix + p]);
        const float m = emax[v];
        masked = m > 0.0f && e / m > tau;
    }
    const float w_minus = photo[v];
    const uint2 range = ranges[t];
    const int n_list = (int)(range.y - range.x);
    float T = 1.0f;
    bool done = !inside || !masked;  // unmasked pixels add nothing
    for (int b0 = 0; b0 < n_list; b0 += kTilePix) {
        if (__syncthreads_count(!done) == 0) break;
        if (b0 + tid < n_list) {
            const uint32_t it = inst_item[range.x + b0 + tid];
            float4 r0 = rec[3 * (size_t)it];
            const float4 r1 = rec[3 * (size_t)it + 1], r2 = rec[3 * (size_t)it + 2];
            const float2 mm = tile_local_mean(r0, r1.w, r2.w, x0, y0);
            r0.x = mm.x;
            r0.y = mm.y;
            r0.w = __fmul_rn(2.0f, r0.w);  // staged as 2B (exact)
            s_r0[tid] = r0;
            s_r1[tid] = r1;
            s_g[tid] = (uint32_t)(it % (uint32_t)n);
        }
        __syncthreads();
        const int cnt = min(kTilePix, n_list - b0);
        for (int j = 0; j < cnt; ++j) {
            if (__all_sync(0xffffffffu, done)) break;
            bool hit = false;
            if (!done) {
                PairEval e;
                eval_pair_b2(s_r0[j], s_r1[j], px, py, e);
                if (!(e.power2 > 0.0f) && !(e.alpha < kAlphaMin)) {
                    const float test_T = T * (1.0f - e.alpha);
                    if (test_T < kTStop) {
                        done = true;
                    } else {
                        hit = true;
                        T = test_T;
                    }
                }
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, hit);
            if (bal && lane == __ffs(bal) - 1) {
                const float c = (float)__popc(bal);
                atomicAdd(s_plus + s_g[j], c);
                atomicAdd(r_minus + s_g[j], c * w_minus);
            }
        }
    }
}

// ----------------------------------------------------------------- plan
__global__ void __launch_bounds__(256)
k_max_f32(const float *__restrict__ x, int64_t n, float *__restrict__ out) {
    float m = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256)
        m = fmaxf(m, x[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned int *>(out), __float_as_uint(m));
}

__global__ void __launch_bounds__(256)
k_densify_actions(int64_t n, const float *__restrict__ log_scales, const float *__restrict__ logits,
                  const float *__restrict__ s_plus, const float *__restrict__ r_minus,
                  const float *__restrict__ r_max, gs_densify_rules R, int32_t *__restrict__ action) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const float top = *r_max;
    const float sm = top > 0.0f ? r_minus[i] / top : 0.0f;
    const float sp = s_plus[i] / (float)R.k_views;
    const float o = 1.0f / (1.0f + expf(-logits[i]));
    const float smax =
        fmaxf(fmaxf(expf(log_scales[3 * i]), expf(log_scales[3 * i + 1])), expf(log_scales[3 * i + 2]));
    int32_t a = GS_DENSIFY_KEEP;
    if (sp > R.tau_plus) a = smax > R.percent_dense * R.extent ? GS_DENSIFY_SPLIT : GS_DENSIFY_CLONE;
    if (sm > R.tau_minus || o < R.min_opacity) a = GS_DENSIFY_PRUNE;
    action[i] = a;
}

__device__ __forceinline__ uint32_t results_of(int32_t a) {
    return a == GS_DENSIFY_PRUNE ? 0u : (a == GS_DENSIFY_KEEP ? 1u : 2u);
}

// block b: the number of results of Gaussians [b * kScanBlock, ...)
__global__ void __launch_bounds__(256)
k_result_sums(const int32_t *__restrict__ action, int64_t n, uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t red[8];
    uint32_t s = 0;
    const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
    for (int k = threadIdx.x; k < kScanBlock; k += 256)
        if (b0 + k < n) s += results_of(action[b0 + k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0;
        for (int w = 0; w < 8; ++w) a += red[w];
        block_sums[blockIdx.x] = a;
    }
}

// one thread: exclusive scan of the block sums (few thousand at most) and
// the total
__global__ void k_result_top(uint32_t *__restrict__ block_sums, int nb, int64_t *__restrict__ total) {
    int64_t run = 0;
    for (int b = 0; b < nb; ++b) {
        const uint32_t s = block_sums[b];
        block_sums[b] = (uint32_t)run;
        run += s;
    }
    *total = run;
}

// offsets[i] = first output slot of Gaussian i
__global__ void __launch_bounds__(kScanBlock)
k_result_offsets(const int32_t *__restrict__ action, int64_t n, const uint32_t *__restrict__ block_base,
                 int64_t *__restrict__ offsets) {
    __shared__ uint32_t wsum[kScanBlock / 32];
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t x = i < n ? results_of(action[i]) : 0u;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    if (i < n) offsets[i] = (int64_t)block_base[blockIdx.x] + before + inc - x;
}

// ---------------------------------------------------------------- apply
struct ApplyArrays {
    const float *src[3][5];  // [params, m, v][means, log_scales, quats, logits, sh]
    float *dst[3][5];
};

__global__ void __launch_bounds__(256)
k_densify_apply(int64_t n, int K3, ApplyArrays A, const int32_t *__restrict__ action,
                const int64_t *__restrict__ offsets, const float *__restrict__ normals) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const int32_t a = action[i];
    if (a == GS_DENSIFY_PRUNE) return;
    const int width[5] = {3, 3, 4, 1, K3};
    const int64_t o = offsets[i];
    const int copies = a == GS_DENSIFY_KEEP ? 1 : 2;
    for (int c = 0; c < copies; ++c) {
        const int64_t d = o + c;
        const bool fresh = a == GS_DENSIFY_SPLIT || c == 1;  // new Gaussians start with zero moments
        for (int k = 0; k < 5; ++k) {
            const int w = width[k];
            for (int j = 0; j < w; ++j) {
                A.dst[0][k][d * w + j] = A.src[0][k][i * w + j];
                A.dst[1][k][d * w + j] = fresh ? 0.0f : A.src[1][k][i * w + j];
                A.dst[2][k][d * w + j] = fresh ? 0.0f : A.src[2][k][i * w + j];
            }
        }
        if (a == GS_DENSIFY_SPLIT) {
            const float *q = A.src[0][2] + 4 * i;
            const float ql = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
            const float w = q[0] / ql, x = q[1] / ql, y = q[2] / ql, z = q[3] / ql;
            const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                                2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                                2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
            const float *ls = A.src[0][1] + 3 * i;
            const float *zc = normals + 6 * i + 3 * c;
            float sz[3];
            for (int j = 0; j < 3; ++j) sz[j] = expf(ls[j]) * zc[j];
            for (int r = 0; r < 3; ++r) {
                A.dst[0][0][d * 3 + r] = A.src[0][0][i * 3 + r] + R[3 * r] * sz[0] + R[3 * r + 1] * sz[1] +
                                         R[3 * r + 2] * sz[2];
                A.dst[0][1][d * 3 + r] = ls[r] - kLogSplitScale;
            }
        }
    }
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_densify_scratch_bytes(int64_t n) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    return (size_t)(64 + GS_MAX_VIEWS) * 4 + (size_t)nb * 4 + 256;
}

extern "C" int gs_densify_score(const gs_plan *plan, void *ws, const float *d_rgb, const float *d_target,
                                float tau, const float *d_photo, float *d_s_plus, float *d_r_minus,
                                void *d_scratch, void *stream) {
    if (!plan || !ws || !d_rgb || !d_target || !d_photo || !d_s_plus || !d_r_minus || !d_scratch ||
        !(tau >= 0.0f))
        return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float *emax = reinterpret_cast<float *>(d_scratch);
    int rc = check_cuda(cudaMemsetAsync(emax, 0, GS_MAX_VIEWS * sizeof(float), s));
    if (rc) return rc;
    const ViewsDev vd = make_views(plan, nullptr);
    k_err_max<<<152 * 8, 256, 0, s>>>(vd, d_rgb, d_target, emax);
    k_densify_score<<<plan->total_tiles, kTilePix, 0, s>>>(
        vd, plan->n, ws_at<uint2>(ws, plan->o_ranges), ws_at<uint32_t>(ws, plan->o_ival[plan->inst_final]),
        ws_at<float4>(ws, plan->o_rec), d_rgb, d_target, emax, tau, d_photo, d_s_plus, d_r_minus);
    return launch_error();
}

extern "C" int gs_densify_plan(int64_t n, const gs_params *params, const float *d_s_plus, const float *d_r_minus,
                               const gs_densify_rules *rules, int32_t *d_action, int64_t *d_offsets,
                               void *d_scratch, int64_t *out_new_n, void *stream) {
    if (n <= 0 || !params || params->n != n || !params->log_scales || !params->opacity_logits || !d_s_plus ||
        !d_r_minus || !rules || rules->k_views < 1 || !d_action || !d_offsets || !d_scratch || !out_new_n)
        return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char *sc = reinterpret_cast<char *>(d_scratch);
    float *r_max = reinterpret_cast<float *>(sc + GS_MAX_VIEWS * 4);
    int64_t *total = reinterpret_cast<int64_t *>(sc + 128);
    uint32_t *block_sums = reinterpret_cast<uint32_t *>(sc + 256);
    const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
    int rc = check_cuda(cudaMemsetAsync(r_max, 0, sizeof(float), s));
    if (rc) return rc;
    k_max_f32<<<152 * 4, 256, 0, s>>>(d_r_minus, n, r_max);
    k_densify_actions<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, params->log_scales, params->opacity_logits,
                                                                 d_s_plus, d_r_minus, r_max, *rules, d_action);
    k_result_sums<<<nb, 256, 0, s>>>(d_action, n, block_sums);
    k_result_top<<<1, 1, 0, s>>>(block_sums, nb, total);
    k_result_offsets<<<nb, kScanBlock, 0, s>>>(d_action, n, block_sums, d_offsets);
    rc = launch_error();
    if (rc) return rc;
    rc = check_cuda(cudaMemcpyAsync(out_new_n, total, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (rc) return rc;
    return check_cuda(cudaStreamSynchronize(s));
}

extern "C" int gs_densify_apply(int64_t n, const gs_params *src, const gs_params *src_m, const gs_params *src_v,
                                const int32_t *d_action, const int64_t *d_offsets, const float *d_normals,
                                gs_params *dst, gs_params *dst_m, gs_params *dst_v, void *stream) {
    const gs_params *in[3] = {src, src_m, src_v};
    gs_params *out[3] = {dst, dst_m, dst_v};
    if (n <= 0 || !d_action || !d_offsets || !d_normals) return GS_ERR_ARG;
    ApplyArrays A;
    for (int k = 0; k < 3; ++k) {
        if (!in[k] || !out[k] || in[k]->n != n || in[k]->sh_degree != src->sh_degree ||
            out[k]->sh_degree != src->sh_degree)
            return GS_ERR_ARG;
        const float *si[5] = {in[k]->means, in[k]->log_scales, in[k]->quats, in[k]->opacity_logits, in[k]->sh};
        float *so[5] = {out[k]->means, out[k]->log_scales, out[k]->quats, out[k]->opacity_logits, out[k]->sh};
        for (int j = 0; j < 5; ++j) {
            if (!si[j] || !so[j]) return GS_ERR_ARG;
            A.src[k][j] = si[j];
            A.dst[k][j] = so[j];
        }
    }
    const int K3 = 3 * (src->sh_degree + 1) * (src->sh_degree + 1);
    k_densify_apply<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, K3, A, d_action, d_offsets,
                                                                                  d_normals);
    return launch_error();
}
