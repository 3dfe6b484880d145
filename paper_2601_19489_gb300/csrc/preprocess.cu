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

namespace gs {

// Real spherical harmonics (Condon-Shortley phase) up to degree 3.
constexpr float kSH0 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kSH1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
constexpr float kSH2a = 1.0925484305920792f;   // sqrt(15 / pi) / 2
constexpr float kSH2b = 0.31539156525252005f;  // sqrt(5 / pi) / 4
constexpr float kSH2c = 0.54627421529603959f;  // sqrt(15 / pi) / 4
constexpr float kSH3a = 0.59004358992664352f;  // sqrt(35 / (2 pi)) / 4
constexpr float kSH3b = 2.8906114426405538f;   // sqrt(105 / pi) / 2
constexpr float kSH3c = 0.45704579946446572f;  // sqrt(21 / (2 pi)) / 4
constexpr float kSH3d = 0.37317633259011540f;  // sqrt(7 / pi) / 4
constexpr float kSH3e = 1.4453057213202769f;   // sqrt(105 / pi) / 4

template <int D>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float *Y) {
    Y[0] = kSH0;
    if (D >= 1) {
        Y[1] = -kSH1 * y;
        Y[2] = kSH1 * z;
        Y[3] = -kSH1 * x;
    }
    if (D >= 2) {
        Y[4] = kSH2a * x * y;
        Y[5] = -kSH2a * y * z;
        Y[6] = kSH2b * (3.0f * z * z - 1.0f);
        Y[7] = -kSH2a * x * z;
        Y[8] = kSH2c * (x * x - y * y);
    }
    if (D >= 3) {
        Y[9] = -kSH3a * y * (3.0f * x * x - y * y);
        Y[10] = kSH3b * x * y * z;
        Y[11] = -kSH3c * y * (5.0f * z * z - 1.0f);
        Y[12] = kSH3d * z * (5.0f * z * z - 3.0f);
        Y[13] = -kSH3c * x * (5.0f * z * z - 1.0f);
        Y[14] = kSH3e * z * (x * x - y * y);
        Y[15] = -kSH3a * x * (x * x - 3.0f * y * y);
    }
}

// sum_k w[k] * grad Y_k(x, y, z): the gradient of the basis polynomials
// w.r.t. (x, y, z) contracted with w (the radial part is removed afterwards
// by the normalisation's Jacobian).
template <int D>
__device__ __forceinline__ float3 sh_grad_dot(float x, float y, float z, const float *w) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (D >= 1) {
        gy -= kSH1 * w[1];
        gz += kSH1 * w[2];
        gx -= kSH1 * w[3];
    }
    if (D >= 2) {
        gx += kSH2a * y * w[4];
        gy += kSH2a * x * w[4];
        gy -= kSH2a * z * w[5];
        gz -= kSH2a * y * w[5];
        gz += 6.0f * kSH2b * z * w[6];
        gx -= kSH2a * z * w[7];
        gz -= kSH2a * x * w[7];
        gx += 2.0f * kSH2c * x * w[8];
        gy -= 2.0f * kSH2c * y * w[8];
    }
    if (D >= 3) {
        const float xx = x * x, yy = y * y, zz5 = 5.0f * z * z - 1.0f;
        gx -= 6.0f * kSH3a * x * y * w[9];
        gy -= 3.0f * kSH3a * (xx - yy) * w[9];
        gx += kSH3b * y * z * w[10];
        gy += kSH3b * x * z * w[10];
        gz += kSH3b * x * y * w[10];
        gy -= kSH3c * zz5 * w[11];
        gz -= 10.0f * kSH3c * y * z * w[11];
        gz += kSH3d * (15.0f * z * z - 3.0f) * w[12];
        gx -= kSH3c * zz5 * w[13];
        gz -= 10.0f * kSH3c * x * z * w[13];
        gx += 2.0f * kSH3e * x * z * w[14];
        gy -= 2.0f * kSH3e * y * z * w[14];
        gz += kSH3e * (xx - yy) * w[14];
        gx -= 3.0f * kSH3a * (xx - yy) * w[15];
        gy += 6.0f * kSH3a * x * y * w[15];
    }
    return make_float3(gx, gy, gz);
}

// Float-float ("double-float") helpers for the few per-Gaussian quantities
// whose rounding decides pixel-level branches: the camera depth that orders
// the blend and the projected mean.  Error-free transforms (Knuth's TwoSum,
// the FMA TwoProduct) and a compensated dot product (Ogita, Rump, Oishi,
// "Accurate sum and dot product", 2005) give results within about half an
// ulp of the exact value of the float32 inputs.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ FF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// r . p + t, compensated
__device__ __forceinline__ FF dot3_plus(const float *r, float3 p, float t) {
    FF acc = two_prod(r[0], p.x);
    FF q = two_prod(r[1], p.y);
    FF s = two_sum(acc.hi, q.hi);
    float lo = __fadd_rn(__fadd_rn(acc.lo, q.lo), s.lo);
    q = two_prod(r[2], p.z);
    FF s2 = two_sum(s.hi, q.hi);
    lo = __fadd_rn(__fadd_rn(lo, q.lo), s2.lo);
    FF s3 = two_sum(s2.hi, t);
    lo = __fadd_rn(lo, s3.lo);
    return two_sum(s3.hi, lo);
}

// (x.hi + x.lo) / (z.hi + z.lo)
__device__ __forceinline__ FF div_ff(FF x, FF z) {
    const float q = __fdiv_rn(x.hi, z.hi);
    float r = __fmaf_rn(-q, z.hi, x.hi);
    r = __fadd_rn(r, __fsub_rn(x.lo, __fmul_rn(q, z.lo)));
    return two_sum(q, __fdiv_rn(r, z.hi));
}

// f * u + c as a normalised float-float
__device__ __forceinline__ FF affine_ff(float f, FF u, float c) {
    const FF p = two_prod(f, u.hi);
    const FF s = two_sum(p.hi, c);
    return two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, p.lo), __fmul_rn(f, u.lo)));
}

__device__ __forceinline__ float3 f3(const float *p) { return make_float3(p[0], p[1], p[2]); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 mul3(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Forward quantities shared by the preprocess and its backward.
struct Proj {
    float3 pc;          // camera-space mean
    float iz;           // 1 / z
    float xz, yz;       // clamped x/z, y/z used in J
    bool clx, cly;      // clamp active
    float3 W0, W1, W2;  // rows of the camera rotation
    float qn[4];        // normalised quaternion (w, x, y, z)
    float qlen;
    float Rg[9];        // rotation of the Gaussian, row-major
    float s[3];         // scales
    float3 T0, T1;      // rows of J W
    float3 U0, U1;      // rows of J W R diag(s)
    float Sxx, Sxy, Syy, det;
};

__device__ __forceinline__ void project_cov(const ViewDev &cam, float3 p, float4 q, float3 ls, Proj &P) {
    P.W0 = f3(cam.R);
    P.W1 = f3(cam.R + 3);
    P.W2 = f3(cam.R + 6);
    P.pc = make_float3(dot3(P.W0, p) + cam.t[0], dot3(P.W1, p) + cam.t[1], dot3(P.W2, p) + cam.t[2]);
    P.iz = 1.0f / P.pc.z;
    const float ux = P.pc.x * P.iz, uy = P.pc.y * P.iz;
    P.xz = fminf(fmaxf(ux, -cam.limx), cam.limx);
    P.yz = fminf(fmaxf(uy, -cam.limy), cam.limy);
    P.clx = !(ux >= -cam.limx && ux <= cam.limx);
    P.cly = !(uy >= -cam.limy && uy <= cam.limy);
    P.qlen = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float il = 1.0f / P.qlen;
    const float w = q.x * il, x = q.y * il, y = q.z * il, z = q.w * il;
    P.qn[0] = w; P.qn[1] = x; P.qn[2] = y; P.qn[3] = z;
    P.Rg[0] = 1.f - 2.f * (y * y + z * z); P.Rg[1] = 2.f * (x * y - w * z); P.Rg[2] = 2.f * (x * z + w * y);
    P.Rg[3] = 2.f * (x * y + w * z); P.Rg[4] = 1.f - 2.f * (x * x + z * z); P.Rg[5] = 2.f * (y * z - w * x);
    P.Rg[6] = 2.f * (x * z - w * y); P.Rg[7] = 2.f * (y * z + w * x); P.Rg[8] = 1.f - 2.f * (x * x + y * y);
    P.s[0] = expf(ls.x);
    P.s[1] = expf(ls.y);
    P.s[2] = expf(ls.z);
    P.T0 = mul3(sub3(P.W0, mul3(P.W2, P.xz)), cam.fx * P.iz);
    P.T1 = mul3(sub3(P.W1, mul3(P.W2, P.yz)), cam.fy * P.iz);
    // U = T M, M[k][j] = Rg[k][j] s[j]
    float u0[3], u1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        u0[j] = (P.T0.x * P.Rg[j] + P.T0.y * P.Rg[3 + j] + P.T0.z * P.Rg[6 + j]) * P.s[j];
        u1[j] = (P.T1.x * P.Rg[j] + P.T1.y * P.Rg[3 + j] + P.T1.z * P.Rg[6 + j]) * P.s[j];
    }
    P.U0 = make_float3(u0[0], u0[1], u0[2]);
    P.U1 = make_float3(u1[0], u1[1], u1[2]);
    const float aa = dot3(P.U0, P.U0), cc = dot3(P.U1, P.U1);
    P.Sxx = aa + 0.3f;
    P.Syy = cc + 0.3f;
    P.Sxy = dot3(P.U0, P.U1);
    const float3 cr = cross3(P.U0, P.U1);
    P.det = dot3(cr, cr) + 0.3f * (aa + cc) + 0.09f;
}

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
    dval[item] = (uint32_t)item;

    const float3 p = make_float3(means[3 * g], means[3 * g + 1], means[3 * g + 2]);
    // The depth that orders the blend is compensated, so the float32 key is
    // the camera depth rounded once: two Gaussians can only leave exact depth
    // order when their depths round to the same float (ties go by index).
    const FF zf = dot3_plus(cam.R + 6, p, cam.t[2]);
    const float pz = zf.hi;
    if (!(pz > cam.near_z)) {
        touched[item] = 0;
        rects[item] = make_uint2(0, 0);
        dkey[item] = 0xffffffffu;
        return;
    }
    Proj P;
    project_cov(cam, p, quats[g], make_float3(log_scales[3 * g], log_scales[3 * g + 1], log_scales[3 * g + 2]), P);
    const float a = P.Syy / P.det, b = -P.Sxy / P.det, c = P.Sxx / P.det;
    // projected mean, compensated (rounded once from the exact projection of
    // the float32 mean), so pixel-level decisions do not inherit the rounding
    // of the camera transform at large pixel coordinates
    const FF mxf = affine_ff(cam.fx, div_ff(dot3_plus(cam.R, p, cam.t[0]), zf), cam.cx);
    const FF myf = affine_ff(cam.fy, div_ff(dot3_plus(cam.R + 3, p, cam.t[1]), zf), cam.cy);
    const float mx = mxf.hi, my = myf.hi;
    const float o = 1.0f / (1.0f + expf(-logits[g]));
    const float t = 2.0f * logf(255.0f * o);
    const float A = kH * a, B = kH * b, C = kH * c;
    const float detc = (kH * kH) / P.det;
    const float tb = kH * (t * kLevelRel + kLevelAbs);

    // colour from SH along the viewing direction
    float3 dir = sub3(p, make_float3(cam.campos[0], cam.campos[1], cam.campos[2]));
    dir = mul3(dir, rsqrtf(dot3(dir, dir)));
    float Y[K];
    sh_eval<D>(dir.x, dir.y, dir.z, Y);
    float r = 0.5f, gg = 0.5f, bb = 0.5f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        r += Y[k] * shrow[3 * k];
        gg += Y[k] * shrow[3 * k + 1];
        bb += Y[k] * shrow[3 * k + 2];
    }
    r = fmaxf(r, 0.f);
    gg = fmaxf(gg, 0.f);
    bb = fmaxf(bb, 0.f);

    rec[3 * item + 0] = make_float4(mx, my, A, B);
    rec[3 * item + 1] = make_float4(C, log2f(o), P.iz, mxf.lo);
    rec[3 * item + 2] = make_float4(r, gg, bb, myf.lo);
    bin[item] = make_float2(tb, detc);

    uint32_t count = 0;
    int tx0 = 0, ty0 = 0, tx1 = 0, ty1 = 0;
    if (box3) {
        // classic tile box: square of radius ceil(3 sqrt(largest eigenvalue))
        const float mid = 0.5f * (P.Sxx + P.Syy);
        const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - (P.Sxx * P.Syy - P.Sxy * P.Sxy)));
        const float rad = ceilf(3.0f * sqrtf(lam));
        // the tiles holding the pixel centres of the square (the same
        // pixel-centre rule as the SnugBox's rectangle)
        if (snug_rect(mx, my, rad, rad, (float)cam.W, (float)cam.H, &tx0, &ty0, &tx1, &ty1))
            count = (uint32_t)((tx1 - tx0) * (ty1 - ty0));
    } else if (t > 0.0f) {
        BinGeom bg;
        bin_geom(mx, my, A, B, C, detc, tb, bg);
        if (snug_rect(mx, my, bg.rx, bg.ry, (float)cam.W, (float)cam.H, &tx0, &ty0, &tx1, &ty1)) {
            for (int tx = tx0; tx < tx1; ++tx) {
                float xa, xb;
                column_span(tx, (float)cam.W, &xa, &xb);
                int lo, hi;
                count += column_rows(bg, xa, xb, (float)cam.H, ty0, ty1, &lo, &hi);
            }
        }
    }
    if (count == 0) tx0 = ty0 = tx1 = ty1 = 0;
    touched[item] = count;
    rects[item] = pack_rect(tx0, ty0, tx1, ty1);
    dkey[item] = count ? __float_as_uint(pz) : 0xffffffffu;
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
