// a1: per-(view, Gaussian) preprocess (Sec. 2.1, Eq. 1-2) and
// a8: its backward (the per-Gaussian parallel chain rule of Sec. 2.2).
//
// Forward, per (view v, Gaussian g):
//   camera-space mean pc = W p + t; culled when pc.z <= near
//   Sigma = R(q/|q|) diag(e^{2s}) R^T  written as M M^T with M = R diag(e^s)
//   J = [[fx/z, 0, -fx x'/z], [0, fy/z, -fy y'/z]] with x' = clamp(x/z, +-1.3 tan(fov_x/2))
//   Sigma' = (J W M)(J W M)^T + 0.3 I = U U^T + 0.3 I; its determinant is
//   |U0 x U1|^2 + 0.3 (|U0|^2 + |U1|^2) + 0.09, a sum of non-negative terms,
//   so the conic Sigma'^{-1} is formed without cancellation
//   mean2d = (fx x/z + cx, fy y/z + cy);  o = sigmoid(logit);  t = 2 ln(255 o)
//   colour = max(0, sum_k sh_k Y_k(d) + 0.5), d = (p - camera centre)/|.|
//   SnugBox of the widened level set and the exact per-column tile count.
// The record written for the blend is r0 = (mx, my, A, B), r1 = (C, log2 o,
// 1/z, mx_lo), r2 = (r, g, b, my_lo) with (A, B, C) = kH * conic and the
// projected mean as the float-float (mx + mx_lo, my + my_lo); binning also
// reads (tb, detc) with tb = kH * t_bin and detc = A C - B^2 = kH^2 / det(Sigma').
#include <string.h>

#include "gs_internal.cuh"
#include "preprocess_item.cuh"

namespace gs {

// kPose: the cameras come from `posed` (the pose-corrected copies written by
// pose_compose) instead of the kernel parameter.
// A warp whose 32 items are 32 consecutive Gaussians of one view (the rule
// for one view; every warp when the Gaussian count is a multiple of 32)
// first moves their SH rows into shared memory with coalesced float4 loads
// (a row per lane would be 3K strided loads per thread, each touching 32
// different rows); the others read their rows directly.
constexpr int kPreThreads = 128;
template <int D, bool kPose>
__global__ void __launch_bounds__(kPreThreads)
k_preprocess(ViewsDev views, const ViewDev *__restrict__ posed, int64_t n, const float *__restrict__ means,
             const float *__restrict__ log_scales, const float4 *__restrict__ quats,
             const float *__restrict__ logits, const float *__restrict__ sh, float4 *__restrict__ rec,
             float2 *__restrict__ bin, uint32_t *__restrict__ touched, uint2 *__restrict__ rects,
             uint32_t *__restrict__ dkey, uint32_t *__restrict__ dval, int box3) {
    constexpr int K = (D + 1) * (D + 1);
    constexpr int K3 = 3 * K;
    constexpr int kRow = K3 + 1;  // odd row stride: the lanes' rows fall in different banks
    constexpr bool kStage = D >= 1;
    __shared__ float s_sh[kStage ? kPreThreads / 32 : 1][kStage ? 32 * kRow : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)views.V * n;
    const float *shrow = nullptr;  // this item's SH row (shared or global memory)
    if (kStage) {
        const int64_t item0 = item - lane;
        const int64_t g0 = item0 % n;
        // uniform over the warp: whole warp in range, one view, 16-byte aligned block
        const bool coop = item0 + 31 < total && g0 + 31 < n && ((g0 * K3) & 3) == 0;
        if (coop) {
            const float4 *src = reinterpret_cast<const float4 *>(sh + g0 * K3);
            constexpr int kQ = (32 * K3 / 4 + 31) / 32;  // float4s per lane
            float4 q[kQ];
#pragma unroll
            for (int u = 0; u < kQ; ++u) {
                const int j = lane + 32 * u;
                if (j < 8 * K3) q[u] = __ldg(src + j);
            }
#pragma unroll
            for (int u = 0; u < kQ; ++u) {
                const int j = lane + 32 * u;
                if (j < 8 * K3) {
                    const float e[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int i = 4 * j + k, r = i / K3, c = i - r * K3;
                        s_sh[warp][r * kRow + c] = e[k];
                    }
                }
            }
            __syncwarp();
            shrow = &s_sh[warp][lane * kRow];
        }
    }
    if (item >= total) return;
    const int v = (int)(item / n);
    const int64_t g = item - (int64_t)v * n;
    if (!shrow) shrow = sh + g * K3;
    const ViewDev &cam = kPose ? posed[v] : views.v[v];
    preprocess_item<D>(cam, item, make_float3(means[3 * g], means[3 * g + 1], means[3 * g + 2]), quats[g],
                       make_float3(log_scales[3 * g], log_scales[3 * g + 1], log_scales[3 * g + 2]), logits[g], shrow,
                       rec, bin, touched, rects, dkey, dval, box3);
}

// a8: one thread per Gaussian, summing over the views where it touched tiles.
// grad2d per (view, Gaussian): {d mx, d my, d a, d b}, {d c, d o, d(1/z), -},
// {d r, d g, d b, -} with (a, b, c) the conic of q = a dx^2 + 2 b dx dy + c dy^2.
// A warp owns 32 consecutive Gaussians: their SH rows (3K floats each) are
// moved between global and shared memory with coalesced warp-wide accesses
// (a row per lane would be 3K strided accesses per thread), and each lane
// reads and accumulates its own row in shared memory (odd row stride: no
// bank conflicts).
// With kAdam the gradient is not stored: the thread that completes it (all
// views of the plan are summed inside the kernel) applies the Adam update to
// the parameter in place, so the gradient never travels through memory.
// Every Gaussian is updated, a Gaussian that touched no tile with a zero
// gradient (its moments still decay and it keeps moving), unless the update
// is visible-only: then such a Gaussian's parameters and moments are left as
// they are, and a warp of 32 of them reads and writes nothing.
constexpr int kPbWarps = 2;
constexpr int kSmallRow = 11;  // a lane's gradients: mean 3, log-scale 3, quaternion 4, logit 1

struct PbArgs {
    int64_t n;
    float *means, *log_scales, *quats, *logits, *sh;  // parameters (written only with Adam)
    const uint32_t *touched;
    const float4 *grad2d;
    float *g_means, *g_log_scales, *g_quats, *g_logits, *g_sh;  // gradient accumulators
    float *m[5], *v[5];          // Adam moments: means, log_scales, quats, logits, sh
    float lr[6];                 // means, log_scales, quats, opacity, SH DC, SH rest
    float b1, b2, eps;
    const int32_t *d_step;       // step count, already incremented for this update
    int visible_only;            // Adam: leave Gaussians that touched no tile untouched
    const ViewDev *posed;        // pose-corrected cameras (kPose)
    double *pose_acc;            // pose-gradient slots: GS_POSE_SLOTS x 8 doubles (kPose)
};

// The same update as k_adam's (same operations, same order): the quotient
// with the fast division (about 2 ulp; the divisor is at least eps > 0).
__device__ __forceinline__ void adam_el(float &p, float g, float &m, float &v, float b1, float b2, float eps,
                                        float step, float ibc2) {
    m = b1 * m + (1.0f - b1) * g;
    v = b2 * v + (1.0f - b2) * g * g;
    p -= __fdividef(step * m, sqrtf(v) * ibc2 + eps);
}

// (row, column) of element i of a warp's block of rows of kW floats; a quad
// starting at a multiple of 4 stays in one row when kW is a multiple of 4.
template <int kW>
__device__ __forceinline__ void quad_rc(int j, int e, int &r, int &c) {
    if constexpr (kW % 4 == 0) {
        r = (4 * j) / kW;
        c = 4 * j - r * kW + e;
    } else {
        const int i = 4 * j + e;
        r = i / kW;
        c = i - r * kW;
    }
}

// Adam over a warp's SH block: parameters from shared memory (row stride
// kRowS), gradients from the shared accumulators, moments streamed in
// float4s, half of a lane's quads in flight per batch.  kFull: all 32 rows
// present (no bounds checks).
// upd: bit r set = row r is updated (a row left out keeps its values).
template <int K3, int kRowS, bool kFull>
__device__ __forceinline__ void adam_sh_block(const float *s_p, const float *s_g, float *sh, float *m, float *v,
                                              int rows, int lane, float s_dc, float s_rest, float b1, float b2,
                                              float eps, float ibc2, uint32_t upd) {
    const int F = kFull ? 32 * K3 : rows * K3, FQ = F >> 2;
    float4 *p4 = reinterpret_cast<float4 *>(sh), *m4 = reinterpret_cast<float4 *>(m);
    float4 *v4 = reinterpret_cast<float4 *>(v);
    constexpr int kQL = (32 * K3 / 4 + 31) / 32;  // quads per lane, full block
    constexpr int kU = (kQL + 1) / 2;
    // a quad of a row left out is neither read nor written (rows of 3K
    // floats hold whole quads when 3K is a multiple of 4)
    auto quad_live = [&](int j) { return K3 % 4 != 0 || ((upd >> ((4 * j) / K3)) & 1u); };
#pragma unroll
    for (int b = 0; b < kQL; b += kU) {
        float4 mq[kU], vq[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int j = lane + 32 * (b + u);
            if (b + u < kQL && (kFull ? j < 8 * K3 : j < FQ) && quad_live(j)) {
                mq[u] = m4[j];
                vq[u] = v4[j];
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int j = lane + 32 * (b + u);
            if (b + u < kQL && (kFull ? j < 8 * K3 : j < FQ) && quad_live(j)) {
                float pv[4], mv[4] = {mq[u].x, mq[u].y, mq[u].z, mq[u].w},
                             vv[4] = {vq[u].x, vq[u].y, vq[u].z, vq[u].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    int r, c;
                    quad_rc<K3>(j, e, r, c);
                    pv[e] = s_p[r * kRowS + c];
                    if ((upd >> r) & 1u)
                        adam_el(pv[e], s_g[r * kRowS + c], mv[e], vv[e], b1, b2, eps, c < 3 ? s_dc : s_rest, ibc2);
                }
                p4[j] = make_float4(pv[0], pv[1], pv[2], pv[3]);
                m4[j] = make_float4(mv[0], mv[1], mv[2], mv[3]);
                v4[j] = make_float4(vv[0], vv[1], vv[2], vv[3]);
            }
        }
    }
    if (!kFull)
        for (int i = 4 * FQ + lane; i < F; i += 32) {  // ragged end of the last warp
            const int r = i / K3, c = i - r * K3;
            if (!((upd >> r) & 1u)) continue;
            float pv = s_p[r * kRowS + c];
            adam_el(pv, s_g[r * kRowS + c], m[i], v[i], b1, b2, eps, c < 3 ? s_dc : s_rest, ibc2);
            sh[i] = pv;
        }
}

template <int D, bool kAdam, bool kPose, bool kVisible>
__global__ void __launch_bounds__(kPbWarps * 32, 8)  // <= 128 registers: 8 CTAs (16 warps) per SM
k_preprocess_bwd(ViewsDev views, PbArgs A) {
    const int64_t n = A.n;
    const float *__restrict__ means = A.means;
    const float *__restrict__ log_scales = A.log_scales;
    const float4 *__restrict__ quats = reinterpret_cast<const float4 *>(A.quats);
    const float *__restrict__ logits = A.logits;
    const float *__restrict__ sh = A.sh;
    const uint32_t *__restrict__ touched = A.touched;
    const float4 *__restrict__ grad2d = A.grad2d;
    constexpr int K = (D + 1) * (D + 1);
    constexpr int K3 = 3 * K;
    constexpr int kRow = K3 + 1;
    __shared__ float s_sh[kPbWarps][32 * kRow];
    __shared__ float s_dsh[kPbWarps][32 * kRow];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t g0 = (int64_t)blockIdx.x * (kPbWarps * 32) + warp * 32;
    const int64_t g = g0 + lane;
    const bool valid = g < n;
    const int rows = (int)(n - g0 < 32 ? (n - g0 > 0 ? n - g0 : 0) : 32);
    uint32_t vmask = 0;  // views in which this Gaussian touched tiles
    if (valid)
        for (int v = 0; v < views.V; ++v)
            if (touched[(int64_t)v * n + g] != 0) vmask |= 1u << v;
    const uint32_t busy = __ballot_sync(0xffffffffu, vmask != 0);
    if ((!kAdam || kVisible) && busy == 0) return;  // uniform over the warp
    // rows the Adam phase updates: all, or (visible-only Adam) the Gaussians
    // that touched a tile in some view of the step
    const uint32_t upd = kVisible ? busy : 0xffffffffu;
    if (kAdam && rows > 0 && (!kVisible || busy == 0xffffffffu)) {
        // ask L2 for the warp's blocks of every array the Adam phase streams
        // (visible-only: when the whole warp is updated)
        // (bulk prefetches, one range per lane, rounded down to whole 16-byte
        // units inside the arrays), so that they arrive while the gradient
        // is being computed
        const int widths[5] = {3, 3, 4, 1, K3};
        const int a = lane % 5, kind = lane / 5;  // lanes 0..14: (array, p / m / v)
        if (lane < 15) {
            const float *base = kind == 0 ? (a == 0 ? A.means : a == 1 ? A.log_scales : a == 2 ? A.quats
                                                     : a == 3 ? A.logits : A.sh)
                                          : (kind == 1 ? A.m[a] : A.v[a]);
            const uint32_t bytes = (uint32_t)(rows * widths[a] * 4) & ~15u;
            if (bytes > 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(base + g0 * widths[a]), "r"(bytes)
                             : "memory");
        }
    }
    float *row = &s_sh[warp][lane * kRow];
    float *drow = &s_dsh[warp][lane * kRow];
    {
        // the warp's SH block (16-byte aligned: 32 rows of 3K floats) moves
        // in float4s, all of a lane's loads issued before any is used
        const int F = rows * K3, FQ = F >> 2;
        const float4 *src = reinterpret_cast<const float4 *>(sh + g0 * K3);
        constexpr int kQ = (32 * K3 / 4 + 31) / 32;  // float4s per lane for a full warp
        float4 q[kQ];
#pragma unroll
        for (int u = 0; u < kQ; ++u) {
            const int j = lane + 32 * u;
            if (j < FQ) q[u] = __ldg(src + j);
        }
#pragma unroll
        for (int u = 0; u < kQ; ++u) {
            const int j = lane + 32 * u;
            if (j < FQ) {
                const float e[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = 4 * j + k, r = i / K3, c = i - r * K3;
                    s_sh[warp][r * kRow + c] = e[k];
                }
            }
        }
        for (int i = 4 * FQ + lane; i < F; i += 32) {  // ragged end of the last warp
            const int r = i / K3, c = i - r * K3;
            s_sh[warp][r * kRow + c] = __ldg(sh + g0 * K3 + i);
        }
    }
#pragma unroll
    for (int c = 0; c < K3; ++c) drow[c] = 0.0f;
    __syncwarp();

    float3 dp = make_float3(0.f, 0.f, 0.f);
    float g_ls[3] = {0.f, 0.f, 0.f}, g_q[4] = {0.f, 0.f, 0.f, 0.f};
    float dlogit = 0.f;
    // kPose: this Gaussian's share of dL/d(omega, tau), the camera-frame
    // increment of the global pose correction (Sec. 2.5), summed over views
    float3 pw = make_float3(0.f, 0.f, 0.f), pt = make_float3(0.f, 0.f, 0.f);
    if (vmask) {
        const float3 p = make_float3(means[3 * g], means[3 * g + 1], means[3 * g + 2]);
        const float4 q = quats[g];
        const float3 ls = make_float3(log_scales[3 * g], log_scales[3 * g + 1], log_scales[3 * g + 2]);
        const float o = 1.0f / (1.0f + expf(-logits[g]));
        float dRg[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float ds[3] = {0.f, 0.f, 0.f};
        Proj P;
        for (int v = 0; v < views.V; ++v) {
            if (!((vmask >> v) & 1u)) continue;
            const int64_t item = (int64_t)v * n + g;
            const ViewDev &cam = kPose ? A.posed[v] : views.v[v];
            project_cov(cam, p, q, ls, P);
            const float4 ga = grad2d[3 * item + 0];
            const float4 gb = grad2d[3 * item + 1];
            const float4 gc = grad2d[3 * item + 2];
            // ---- opacity
            dlogit += gb.y * o * (1.0f - o);
            // ---- colour: SH coefficients and the viewing direction
            {
                float3 dv = sub3(p, make_float3(cam.campos[0], cam.campos[1], cam.campos[2]));
                const float inv_len = rsqrtf(dot3(dv, dv));
                const float3 dir = mul3(dv, inv_len);
                float Y[K];
                sh_eval<D>(dir.x, dir.y, dir.z, Y);
                float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
                for (int k = 0; k < K; ++k)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) raw[ch] += Y[k] * row[3 * k + ch];
                const float gr[3] = {raw[0] > 0.f ? gc.x : 0.f, raw[1] > 0.f ? gc.y : 0.f,
                                     raw[2] > 0.f ? gc.z : 0.f};
                float wk[K];  // dL/dY_k
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    wk[k] = 0.f;
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        drow[3 * k + ch] += gr[ch] * Y[k];
                        wk[k] += gr[ch] * row[3 * k + ch];
                    }
                }
                const float3 ddir = sh_grad_dot<D>(dir.x, dir.y, dir.z, wk);
                // d = dv / |dv|:  d(dv) = (ddir - d (d . ddir)) / |dv|
                const float3 gdv = mul3(sub3(ddir, mul3(dir, dot3(dir, ddir))), inv_len);
                dp = add3(dp, gdv);
                // the camera centre moves by -W^T tau under tau and stays put
                // under omega: dL/dtau = W dL/d(dv)
                if (kPose) pt = add3(pt, make_float3(dot3(P.W0, gdv), dot3(P.W1, gdv), dot3(P.W2, gdv)));
            }
            // ---- conic Q = Sigma'^-1 with Sigma' = U U^T + 0.3 I:
            //   dL/dSigma' = -Q G Q  (G: gradient w.r.t. the symmetric conic matrix,
            //   off-diagonal gb / 2), so dL/dU = 2 dL/dSigma' U = -2 Q G (Q U).
            // Forming W = Q U first keeps a long axis's column small instead of
            // cancelling large entries of dL/dSigma' against it (needle-like
            // Gaussians would otherwise lose most float32 digits).
            const float inv_det = 1.0f / P.det;
            const float qa = P.Syy * inv_det, qb = -P.Sxy * inv_det, qc = P.Sxx * inv_det;
            const float3 W0 = add3(mul3(P.U0, qa), mul3(P.U1, qb));
            const float3 W1 = add3(mul3(P.U0, qb), mul3(P.U1, qc));
            const float hb = 0.5f * ga.w;
            const float3 GW0 = add3(mul3(W0, ga.z), mul3(W1, hb));
            const float3 GW1 = add3(mul3(W0, hb), mul3(W1, gb.x));
            const float3 dU0 = mul3(add3(mul3(GW0, qa), mul3(GW1, qb)), -2.f);
            const float3 dU1 = mul3(add3(mul3(GW0, qb), mul3(GW1, qc)), -2.f);
            // ---- U = T M, M = Rg diag(s):  dT_k = sum_j dU_j Rg[k][j] s_j;  dM[k][j] = T_k dU_j
            const float du0[3] = {dU0.x, dU0.y, dU0.z}, du1[3] = {dU1.x, dU1.y, dU1.z};
            const float t0[3] = {P.T0.x, P.T0.y, P.T0.z}, t1[3] = {P.T1.x, P.T1.y, P.T1.z};
            float dT0[3], dT1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float a0 = 0.f, a1 = 0.f;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float m = P.Rg[3 * k + j] * P.s[j];
                    a0 += du0[j] * m;
                    a1 += du1[j] * m;
                    const float dM = t0[k] * du0[j] + t1[k] * du1[j];
                    dRg[3 * k + j] += dM * P.s[j];
                    ds[j] += dM * P.Rg[3 * k + j];
                }
                dT0[k] = a0;
                dT1[k] = a1;
            }
            // ---- T0 = fx iz (W0 - xz W2), T1 = fy iz (W1 - yz W2)
            const float3 vdT0 = make_float3(dT0[0], dT0[1], dT0[2]);
            const float3 vdT1 = make_float3(dT1[0], dT1[1], dT1[2]);
            float d_iz = cam.fx * dot3(vdT0, sub3(P.W0, mul3(P.W2, P.xz))) +
                         cam.fy * dot3(vdT1, sub3(P.W1, mul3(P.W2, P.yz)));
            const float d_xz = -cam.fx * P.iz * dot3(vdT0, P.W2);
            const float d_yz = -cam.fy * P.iz * dot3(vdT1, P.W2);
            float dx = 0.f, dy = 0.f;
            if (!P.clx) {  // xz = x * iz
                dx += d_xz * P.iz;
                d_iz += d_xz * P.pc.x;
            }
            if (!P.cly) {
                dy += d_yz * P.iz;
                d_iz += d_yz * P.pc.y;
            }
            // ---- mean2d = (fx x iz + cx, fy y iz + cy), disparity 1/z
            dx += ga.x * cam.fx * P.iz;
            dy += ga.y * cam.fy * P.iz;
            d_iz += ga.x * cam.fx * P.pc.x + ga.y * cam.fy * P.pc.y + gb.z;
            const float dz = -d_iz * P.iz * P.iz;
            // ---- pc = W p + t
            dp = add3(dp, add3(add3(mul3(P.W0, dx), mul3(P.W1, dy)), mul3(P.W2, dz)));
            if (kPose) {
                // pc -> exp([omega]_x) pc + tau: dL/dtau = dL/dpc, and
                // dL/domega = pc x dL/dpc plus, through T = J W with W ->
                // exp([omega]_x) W at fixed J, sum_a (W dT_a) x J_a over the rows
                // J_0 = fx iz (1, 0, -xz), J_1 = fy iz (0, 1, -yz)
                const float3 gpc = make_float3(dx, dy, dz);
                pt = add3(pt, gpc);
                const float3 wt0 = make_float3(dot3(P.W0, vdT0), dot3(P.W1, vdT0), dot3(P.W2, vdT0));
                const float3 wt1 = make_float3(dot3(P.W0, vdT1), dot3(P.W1, vdT1), dot3(P.W2, vdT1));
                const float3 j0 = make_float3(cam.fx * P.iz, 0.f, -cam.fx * P.iz * P.xz);
                const float3 j1 = make_float3(0.f, cam.fy * P.iz, -cam.fy * P.iz * P.yz);
                pw = add3(pw, add3(cross3(P.pc, gpc), add3(cross3(wt0, j0), cross3(wt1, j1))));
            }
        }
        // ---- scales: s = exp(log_scale)
        g_ls[0] = ds[0] * P.s[0];
        g_ls[1] = ds[1] * P.s[1];
        g_ls[2] = ds[2] * P.s[2];
        // ---- rotation of the unit quaternion, then its normalisation
        const float w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
        const float *R = dRg;
        float dqn[4];
        dqn[0] = 2.f * (-z * R[1] + y * R[2] + z * R[3] - x * R[5] - y * R[6] + x * R[7]);
        dqn[1] = 2.f * (y * R[1] + z * R[2] + y * R[3] - 2.f * x * R[4] - w * R[5] + z * R[6] + w * R[7] -
                        2.f * x * R[8]);
        dqn[2] = 2.f * (-2.f * y * R[0] + x * R[1] + w * R[2] + x * R[3] + z * R[5] - w * R[6] + z * R[7] -
                        2.f * y * R[8]);
        dqn[3] = 2.f * (-2.f * z * R[0] - w * R[1] + x * R[2] + w * R[3] - 2.f * z * R[4] + y * R[5] +
                        x * R[6] + y * R[7]);
        const float proj = dqn[0] * w + dqn[1] * x + dqn[2] * y + dqn[3] * z;
        const float il = 1.0f / P.qlen;
        g_q[0] = (dqn[0] - w * proj) * il;
        g_q[1] = (dqn[1] - x * proj) * il;
        g_q[2] = (dqn[2] - y * proj) * il;
        g_q[3] = (dqn[3] - z * proj) * il;
    }
    if (kPose) {
        // warp sum, then one lane adds it into the warp's slot (the slots
        // spread the atomic adds over GS_POSE_SLOTS addresses)
        float acc[6] = {pw.x, pw.y, pw.z, pt.x, pt.y, pt.z};
#pragma unroll
        for (int k = 0; k < 6; ++k)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
        if (lane == 0) {
            double *slot = A.pose_acc + 8 * (int)((g0 >> 5) % GS_POSE_SLOTS);
#pragma unroll
            for (int k = 0; k < 6; ++k) atomicAdd(slot + k, (double)acc[k]);
        }
    }
    if (!kAdam) {
        if (vmask) {
            A.g_log_scales[3 * g + 0] += g_ls[0];
            A.g_log_scales[3 * g + 1] += g_ls[1];
            A.g_log_scales[3 * g + 2] += g_ls[2];
            float4 *gq = reinterpret_cast<float4 *>(A.g_quats) + g;  // quaternion rows are 16-byte aligned
            float4 dq = *gq;
            dq.x += g_q[0];
            dq.y += g_q[1];
            dq.z += g_q[2];
            dq.w += g_q[3];
            *gq = dq;
            A.g_means[3 * g + 0] += dp.x;
            A.g_means[3 * g + 1] += dp.y;
            A.g_means[3 * g + 2] += dp.z;
            A.g_logits[g] += dlogit;
        }
        __syncwarp();
        // the warp's SH gradient rows, accumulated with coalesced float4
        // accesses, all loads of a lane in flight together (rows of Gaussians
        // that touched no tile get + 0)
        const int F = rows * K3, FQ = F >> 2;
        float4 *dst = reinterpret_cast<float4 *>(A.g_sh + g0 * K3);
        constexpr int kQ = (32 * K3 / 4 + 31) / 32;
        float4 q[kQ];
#pragma unroll
        for (int u = 0; u < kQ; ++u) {
            const int j = lane + 32 * u;
            if (j < FQ) q[u] = dst[j];
        }
#pragma unroll
        for (int u = 0; u < kQ; ++u) {
            const int j = lane + 32 * u;
            if (j < FQ) {
                float e[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = 4 * j + k, r = i / K3, c = i - r * K3;
                    e[k] += s_dsh[warp][r * kRow + c];
                }
                dst[j] = make_float4(e[0], e[1], e[2], e[3]);
            }
        }
        for (int i = 4 * FQ + lane; i < F; i += 32) {  // ragged end of the last warp
            const int r = i / K3, c = i - r * K3;
            A.g_sh[g0 * K3 + i] += s_dsh[warp][r * kRow + c];
        }
        return;
    }
    // ---- Adam (bias corrections from the device step count, as in k_adam).
    // Each lane parks its small-attribute gradients in shared memory; then the
    // warp updates every attribute array of its 32 Gaussians with coalesced
    // accesses (consecutive lanes, consecutive floats).
    const float tstep = (float)*A.d_step;
    const float ibc1 = -1.0f / expm1f(tstep * log1pf(A.b1 - 1.0f));
    const float ibc2 = 1.0f / sqrtf(-expm1f(tstep * log1pf(A.b2 - 1.0f)));
    __shared__ float s_g[kPbWarps][32 * kSmallRow];
    {
        float *gr = &s_g[warp][lane * kSmallRow];
        gr[0] = dp.x;
        gr[1] = dp.y;
        gr[2] = dp.z;
        gr[3] = g_ls[0];
        gr[4] = g_ls[1];
        gr[5] = g_ls[2];
        gr[6] = g_q[0];
        gr[7] = g_q[1];
        gr[8] = g_q[2];
        gr[9] = g_q[3];
        gr[10] = dlogit;
    }
    __syncwarp();
    // The moments stream with float4 accesses, several per lane in flight
    // (a warp's block of an attribute array starts 16-byte aligned: 32
    // Gaussians of 4 or 12 bytes, or SH rows).
    // (attribute array, floats per Gaussian, offset of its gradient in a lane's row)
    float *const pa[4] = {A.means, A.log_scales, A.quats, A.logits};
    const int width[4] = {3, 3, 4, 1}, goff[4] = {0, 3, 6, 10};
    float4 sp[4], sm[4], sv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int nq = (rows * width[a]) >> 2;
        if (lane < nq) {
            sp[a] = reinterpret_cast<const float4 *>(pa[a] + g0 * width[a])[lane];
            sm[a] = reinterpret_cast<const float4 *>(A.m[a] + g0 * width[a])[lane];
            sv[a] = reinterpret_cast<const float4 *>(A.v[a] + g0 * width[a])[lane];
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int w = width[a];
        const int nq = (rows * w) >> 2;
        const float st = A.lr[a] * ibc1;
        if (lane < nq) {
            float pv[4] = {sp[a].x, sp[a].y, sp[a].z, sp[a].w}, mv[4] = {sm[a].x, sm[a].y, sm[a].z, sm[a].w},
                  vv[4] = {sv[a].x, sv[a].y, sv[a].z, sv[a].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = 4 * lane + e, r = i / w, c = i - r * w;
                if ((upd >> r) & 1u)
                    adam_el(pv[e], s_g[warp][r * kSmallRow + goff[a] + c], mv[e], vv[e], A.b1, A.b2, A.eps, st,
                            ibc2);
            }
            reinterpret_cast<float4 *>(pa[a] + g0 * w)[lane] = make_float4(pv[0], pv[1], pv[2], pv[3]);
            reinterpret_cast<float4 *>(A.m[a] + g0 * w)[lane] = make_float4(mv[0], mv[1], mv[2], mv[3]);
            reinterpret_cast<float4 *>(A.v[a] + g0 * w)[lane] = make_float4(vv[0], vv[1], vv[2], vv[3]);
        }
        for (int i = 4 * nq + lane; i < rows * w; i += 32) {  // ragged end of the last warp
            const int r = i / w, c = i - r * w;
            if (!((upd >> r) & 1u)) continue;
            float *pp = pa[a] + g0 * w, *mm = A.m[a] + g0 * w, *vvp = A.v[a] + g0 * w;
            float pv = pp[i], mv = mm[i], v2 = vvp[i];
            adam_el(pv, s_g[warp][r * kSmallRow + goff[a] + c], mv, v2, A.b1, A.b2, A.eps, st, ibc2);
            pp[i] = pv;
            mm[i] = mv;
            vvp[i] = v2;
        }
    }
    // SH rows
    const float s_dc = A.lr[4] * ibc1, s_rest = A.lr[5] * ibc1;
    if (rows == 32)
        adam_sh_block<K3, kRow, true>(s_sh[warp], s_dsh[warp], A.sh + g0 * K3, A.m[4] + g0 * K3,
                                      A.v[4] + g0 * K3, rows, lane, s_dc, s_rest, A.b1, A.b2, A.eps, ibc2, upd);
    else
        adam_sh_block<K3, kRow, false>(s_sh[warp], s_dsh[warp], A.sh + g0 * K3, A.m[4] + g0 * K3,
                                       A.v[4] + g0 * K3, rows, lane, s_dc, s_rest, A.b1, A.b2, A.eps, ibc2, upd);
}

template <int D, bool kPose>
static void launch_preprocess(const gs_plan *plan, void *ws, const gs_params *pr, const ViewsDev &vd,
                              cudaStream_t s) {
    const int64_t total = plan->VN;
    const unsigned blocks = (unsigned)((total + kPreThreads - 1) / kPreThreads);
    k_preprocess<D, kPose><<<blocks, kPreThreads, 0, s>>>(
        vd, ws_at<ViewDev>(ws, plan->o_posed), plan->n, pr->means, pr->log_scales, (const float4 *)pr->quats, pr->opacity_logits, pr->sh,
        ws_at<float4>(ws, plan->o_rec), ws_at<float2>(ws, plan->o_bin), ws_at<uint32_t>(ws, plan->o_touched),
        ws_at<uint2>(ws, plan->o_rect), ws_at<uint32_t>(ws, plan->o_dkey[0]), ws_at<uint32_t>(ws, plan->o_dval[0]),
        plan->bbox_3sigma);
}

template <int D, bool kAdam>
static void launch_preprocess_bwd(const ViewsDev &vd, const PbArgs &A, cudaStream_t s) {
    const unsigned blocks = (unsigned)((A.n + kPbWarps * 32 - 1) / (kPbWarps * 32));
    const bool vis = kAdam && A.visible_only;
    if (A.pose_acc) {
        if (vis)
            k_preprocess_bwd<D, kAdam, true, kAdam><<<blocks, kPbWarps * 32, 0, s>>>(vd, A);
        else
            k_preprocess_bwd<D, kAdam, true, false><<<blocks, kPbWarps * 32, 0, s>>>(vd, A);
    } else {
        if (vis)
            k_preprocess_bwd<D, kAdam, false, kAdam><<<blocks, kPbWarps * 32, 0, s>>>(vd, A);
        else
            k_preprocess_bwd<D, kAdam, false, false><<<blocks, kPbWarps * 32, 0, s>>>(vd, A);
    }
}

static PbArgs pb_args(const gs_plan *plan, void *ws, const gs_params *pr) {
    PbArgs A;
    memset(&A, 0, sizeof(A));
    A.n = plan->n;
    A.means = pr->means;
    A.log_scales = pr->log_scales;
    A.quats = pr->quats;
    A.logits = pr->opacity_logits;
    A.sh = pr->sh;
    A.touched = ws_at<uint32_t>(ws, plan->o_touched);
    A.grad2d = ws_at<float4>(ws, plan->o_grad2d);
    if (plan->pose) {
        A.posed = ws_at<ViewDev>(ws, plan->o_posed);
        A.pose_acc = plan->pose + 32;
    }
    return A;
}

template <bool kAdam>
static void dispatch_preprocess_bwd(int sh_degree, const ViewsDev &vd, const PbArgs &A, cudaStream_t s) {
    switch (sh_degree) {
        case 0: launch_preprocess_bwd<0, kAdam>(vd, A, s); break;
        case 1: launch_preprocess_bwd<1, kAdam>(vd, A, s); break;
        case 2: launch_preprocess_bwd<2, kAdam>(vd, A, s); break;
        default: launch_preprocess_bwd<3, kAdam>(vd, A, s); break;
    }
}

int check_params(const gs_plan *plan, const gs_params *p) {
    if (!p || p->n != plan->n || p->sh_degree != plan->sh_degree || !p->means || !p->log_scales ||
        !p->quats || !p->opacity_logits || !p->sh)
        return GS_ERR_ARG;
    if ((((uintptr_t)p->quats) | ((uintptr_t)p->sh)) & 15) return GS_ERR_ARG;  // read as float4 rows / blocks
    return GS_OK;
}

int check_cams(const gs_plan *plan, const gs_camera *cams) {
    if (!cams) return GS_ERR_ARG;
    for (int v = 0; v < plan->V; ++v)
        if (cams[v].width != plan->W[v] || cams[v].height != plan->H[v] || !(cams[v].fx > 0.f) ||
            !(cams[v].fy > 0.f))
            return GS_ERR_ARG;
    return GS_OK;
}

int preprocess_bwd(const gs_plan *plan, void *ws, const gs_params *params, const gs_camera *cams,
                   gs_params *grads, cudaStream_t s) {
    const ViewsDev vd = make_views(plan, cams);
    PbArgs A = pb_args(plan, ws, params);
    A.g_means = grads->means;
    A.g_log_scales = grads->log_scales;
    A.g_quats = grads->quats;
    A.g_logits = grads->opacity_logits;
    A.g_sh = grads->sh;
    dispatch_preprocess_bwd<false>(plan->sh_degree, vd, A, s);
    return launch_error();
}

int preprocess_bwd_adam(const gs_plan *plan, void *ws, gs_params *params, const gs_camera *cams,
                        const gs_params *m, const gs_params *v, const gs_adam_hparams *hp, int32_t *d_step,
                        cudaStream_t s) {
    const ViewsDev vd = make_views(plan, cams);
    PbArgs A = pb_args(plan, ws, params);
    const gs_params *mv[2] = {m, v};
    for (int k = 0; k < 2; ++k) {
        float **dst = k == 0 ? A.m : A.v;
        dst[0] = mv[k]->means;
        dst[1] = mv[k]->log_scales;
        dst[2] = mv[k]->quats;
        dst[3] = mv[k]->opacity_logits;
        dst[4] = mv[k]->sh;
    }
    const float lr[6] = {hp->lr_means, hp->lr_log_scales, hp->lr_quats, hp->lr_opacity, hp->lr_sh_dc,
                         hp->lr_sh_rest};
    for (int k = 0; k < 6; ++k) A.lr[k] = lr[k];
    A.b1 = hp->b1;
    A.b2 = hp->b2;
    A.eps = hp->eps;
    A.d_step = d_step;
    A.visible_only = hp->visible_only != 0;
    int rc = adam_tick(d_step, s);
    if (rc) return rc;
    dispatch_preprocess_bwd<true>(plan->sh_degree, vd, A, s);
    return launch_error();
}

}  // namespace gs

using namespace gs;

extern "C" int gs_preprocess(const gs_plan *plan, void *ws, const gs_params *params,
                             const gs_camera *cams, void *stream) {
    if (!plan || !ws) return GS_ERR_ARG;
    int rc = check_params(plan, params);
    if (rc) return rc;
    rc = check_cams(plan, cams);
    if (rc) return rc;
    const ViewsDev vd = make_views(plan, cams);
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->pose) {
        rc = pose_compose(plan, ws, vd, s);
        if (rc) return rc;
        switch (plan->sh_degree) {
            case 0: launch_preprocess<0, true>(plan, ws, params, vd, s); break;
            case 1: launch_preprocess<1, true>(plan, ws, params, vd, s); break;
            case 2: launch_preprocess<2, true>(plan, ws, params, vd, s); break;
            default: launch_preprocess<3, true>(plan, ws, params, vd, s); break;
        }
        return launch_error();
    }
    switch (plan->sh_degree) {
        case 0: launch_preprocess<0, false>(plan, ws, params, vd, s); break;
        case 1: launch_preprocess<1, false>(plan, ws, params, vd, s); break;
        case 2: launch_preprocess<2, false>(plan, ws, params, vd, s); break;
        default: launch_preprocess<3, false>(plan, ws, params, vd, s); break;
    }
    return launch_error();
}

extern "C" int gs_preprocess_bwd_adam(const gs_plan *plan, void *ws, gs_params *params, const gs_camera *cams,
                                      const gs_params *adam_m, const gs_params *adam_v,
                                      const gs_adam_hparams *hp, int32_t *d_step, void *stream) {
    if (!plan || !ws || !hp || !d_step) return GS_ERR_ARG;
    int rc = check_params(plan, params);
    if (!rc) rc = check_params(plan, adam_m);
    if (!rc) rc = check_params(plan, adam_v);
    if (!rc) rc = check_cams(plan, cams);
    if (rc) return rc;
    if (!(hp->b1 > 0.0f && hp->b1 < 1.0f) || !(hp->b2 > 0.0f && hp->b2 < 1.0f) || !(hp->eps >= 0.0f))
        return GS_ERR_ARG;
    // every attribute array is streamed with float4 accesses
    const gs_params *all[3] = {params, adam_m, adam_v};
    for (const gs_params *q : all)
        if ((((uintptr_t)q->means) | ((uintptr_t)q->log_scales) | ((uintptr_t)q->quats) |
             ((uintptr_t)q->opacity_logits) | ((uintptr_t)q->sh)) & 15)
            return GS_ERR_ARG;
    return preprocess_bwd_adam(plan, ws, params, cams, adam_m, adam_v, hp, d_step, (cudaStream_t)stream);
}
