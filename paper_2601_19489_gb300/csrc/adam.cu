// a9: Adam with bias correction, fused with zeroing the gradient.
//   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
//   p -= (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps);  g = 0
// A pure stream: per element it reads and writes p, g, m and v (32 bytes),
// with float4 accesses where the arrays are 16-byte aligned.
// Several parameter groups (different learning rates) go into one launch.
// The step count t either comes from the host (bias corrections computed in
// double there) or lives in device memory, for a step captured once in a
// CUDA graph and replayed: a one-thread launch increments it, and every
// thread of the update derives 1 - b^t = -expm1(t log1p(b - 1)) in float32
// (b - 1 is exact for b in [0.5, 1) and rounds once below; the two library
// calls keep the relative error near 1e-7 even at t = 1, where 1 - b^t
// cancels).
#include <math.h>

#include "gs_internal.cuh"

namespace gs {

constexpr int kMaxGroups = 8;
constexpr int kAdamThreads = 256;

struct AdamGroups {
    int n_groups;
    float b1, b2, eps;
    float step_size[kMaxGroups];   // lr / (1 - b1^t)
    float step_head[kMaxGroups];   // lr_head / (1 - b1^t)
    int64_t period[kMaxGroups], head[kMaxGroups];
    float inv_bc2_sqrt;            // 1 / sqrt(1 - b2^t)
    float *p[kMaxGroups], *g[kMaxGroups], *m[kMaxGroups], *v[kMaxGroups];
    int64_t n[kMaxGroups];
    int64_t slot_off[kMaxGroups + 1];  // prefix of ceil(n / 4) per group
    int vec_ok[kMaxGroups];
    float lr[kMaxGroups], lr_head[kMaxGroups];
    const int32_t *d_step;         // device step count (already incremented), or null
};

__device__ __forceinline__ void adam1(float &p, float &g, float &m, float &v, float b1, float b2,
                                      float eps, float step, float ibc2) {
    m = b1 * m + (1.0f - b1) * g;
    v = b2 * v + (1.0f - b2) * g * g;
    p -= __fdividef(step * m, sqrtf(v) * ibc2 + eps);  // divisor >= eps > 0: fast division, ~2 ulp
    g = 0.0f;
}

__global__ void k_adam_tick(int32_t *d_step) { *d_step += 1; }

template <bool kDevStep>
__global__ void __launch_bounds__(kAdamThreads) k_adam(AdamGroups G) {
    const int64_t total = G.slot_off[G.n_groups];
    float ibc1 = 1.0f, ibc2 = G.inv_bc2_sqrt;
    if (kDevStep) {
        const float t = (float)*G.d_step;
        ibc1 = -1.0f / expm1f(t * log1pf(G.b1 - 1.0f));
        ibc2 = 1.0f / sqrtf(-expm1f(t * log1pf(G.b2 - 1.0f)));
    }
    for (int64_t slot = (int64_t)blockIdx.x * kAdamThreads + threadIdx.x; slot < total;
         slot += (int64_t)gridDim.x * kAdamThreads) {
        int gi = 0;
        while (slot >= G.slot_off[gi + 1]) ++gi;
        const int64_t i = (slot - G.slot_off[gi]) * 4;
        const int64_t n = G.n[gi];
        const float step = kDevStep ? G.lr[gi] * ibc1 : G.step_size[gi];
        const float step_head = kDevStep ? G.lr_head[gi] * ibc1 : G.step_head[gi];
        if (G.vec_ok[gi] && i + 3 < n) {
            float st[4] = {step, step, step, step};
            if (G.period[gi] > 0) {  // per-element rate by position in the period
                const int64_t per = G.period[gi];
                int64_t r = i < 0xffffffffll && per < 0xffffffffll ? (int64_t)((uint32_t)i % (uint32_t)per)
                                                                    : i % per;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    st[c] = r < G.head[gi] ? step_head : step;
                    if (++r == per) r = 0;
                }
            }
            float4 p = *reinterpret_cast<float4 *>(G.p[gi] + i);
            float4 g = *reinterpret_cast<float4 *>(G.g[gi] + i);
            float4 m = *reinterpret_cast<float4 *>(G.m[gi] + i);
            float4 v = *reinterpret_cast<float4 *>(G.v[gi] + i);
            adam1(p.x, g.x, m.x, v.x, G.b1, G.b2, G.eps, st[0], ibc2);
            adam1(p.y, g.y, m.y, v.y, G.b1, G.b2, G.eps, st[1], ibc2);
            adam1(p.z, g.z, m.z, v.z, G.b1, G.b2, G.eps, st[2], ibc2);
            adam1(p.w, g.w, m.w, v.w, G.b1, G.b2, G.eps, st[3], ibc2);
            *reinterpret_cast<float4 *>(G.p[gi] + i) = p;
            *reinterpret_cast<float4 *>(G.g[gi] + i) = g;
            *reinterpret_cast<float4 *>(G.m[gi] + i) = m;
            *reinterpret_cast<float4 *>(G.v[gi] + i) = v;
        } else {
            for (int64_t j = i; j < i + 4 && j < n; ++j) {
                const float st = G.period[gi] > 0 && (j % G.period[gi]) < G.head[gi] ? step_head : step;
                adam1(G.p[gi][j], G.g[gi][j], G.m[gi][j], G.v[gi][j], G.b1, G.b2, G.eps, st, ibc2);
            }
        }
    }
}

int adam_tick(int32_t *d_step, cudaStream_t s) {
    k_adam_tick<<<1, 1, 0, s>>>(d_step);
    return launch_error();
}

static int adam_launch(const gs_adam_group *groups, int n_groups, float b1, float b2, float eps,
                       int step, int32_t *d_step, cudaStream_t s) {
    if (!groups || n_groups < 1 || n_groups > kMaxGroups || (!d_step && step < 1) ||
        !(b1 > 0.f && b1 < 1.f) || !(b2 > 0.f && b2 < 1.f) ||
        !(eps >= 0.f))
        return GS_ERR_ARG;
    AdamGroups G;
    G.n_groups = n_groups;
    G.b1 = b1;
    G.b2 = b2;
    G.eps = eps;
    G.d_step = d_step;
    const double bc1 = d_step ? 1.0 : 1.0 - pow((double)b1, (double)step);
    const double bc2 = d_step ? 1.0 : 1.0 - pow((double)b2, (double)step);
    G.inv_bc2_sqrt = (float)(1.0 / sqrt(bc2));
    G.slot_off[0] = 0;
    for (int i = 0; i < n_groups; ++i) {
        const gs_adam_group &gr = groups[i];
        if (gr.n < 0 || (gr.n > 0 && (!gr.p || !gr.g || !gr.m || !gr.v))) return GS_ERR_ARG;
        G.p[i] = gr.p;
        G.g[i] = gr.g;
        G.m[i] = gr.m;
        G.v[i] = gr.v;
        G.n[i] = gr.n;
        G.step_size[i] = (float)((double)gr.lr / bc1);
        G.step_head[i] = (float)((double)gr.lr_head / bc1);
        G.lr[i] = gr.lr;
        G.lr_head[i] = gr.lr_head;
        if (gr.period < 0 || gr.head < 0 || (gr.period > 0 && gr.head > gr.period)) return GS_ERR_ARG;
        G.period[i] = gr.period;
        G.head[i] = gr.head;
        const uintptr_t mis = ((uintptr_t)gr.p | (uintptr_t)gr.g | (uintptr_t)gr.m | (uintptr_t)gr.v) & 15;
        G.vec_ok[i] = mis == 0;
        G.slot_off[i + 1] = G.slot_off[i] + (gr.n + 3) / 4;
    }
    if (d_step) {
        const int rc = adam_tick(d_step, s);
        if (rc) return rc;
    }
    const int64_t total = G.slot_off[n_groups];
    if (total == 0) return GS_OK;
    int64_t blocks = (total + kAdamThreads - 1) / kAdamThreads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (d_step)
        k_adam<true><<<(unsigned)blocks, kAdamThreads, 0, s>>>(G);
    else
        k_adam<false><<<(unsigned)blocks, kAdamThreads, 0, s>>>(G);
    return launch_error();
}

}  // namespace gs

using namespace gs;

extern "C" int gs_adam_step(float *p, float *g, float *m, float *v, int64_t n, float lr, float b1,
                            float b2, float eps, int32_t step, void *stream) {
    gs_adam_group gr = {p, g, m, v, n, lr, 0, 0, 0.0f};
    return adam_launch(&gr, 1, b1, b2, eps, step, nullptr, (cudaStream_t)stream);
}

extern "C" int gs_adam_step_multi(const gs_adam_group *groups, int32_t n_groups, float b1, float b2,
                                  float eps, int32_t step, void *stream) {
    return adam_launch(groups, n_groups, b1, b2, eps, step, nullptr, (cudaStream_t)stream);
}

extern "C" int gs_adam_step_multi_dev(const gs_adam_group *groups, int32_t n_groups, float b1, float b2,
                                      float eps, int32_t *d_step, void *stream) {
    if (!d_step) return GS_ERR_ARG;
    return adam_launch(groups, n_groups, b1, b2, eps, 0, d_step, (cudaStream_t)stream);
}
