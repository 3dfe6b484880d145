// Per-(view, Gaussian) preprocess of Sec. 2.1 (Eq. 1-2) as device
// functions, shared by the preprocess kernel and by the neural-Gaussian
// decoder's fused decode + preprocess: real SH, float-float helpers, the EWA
// projection and preprocess_item, which writes one item's blend record,
// binning level set, tile count, tile rectangle and depth key.
#pragma once

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

// One (view, Gaussian) item: cull at the near plane, project, colour from
// the SH row (3 (D + 1)^2 floats, shared or global memory), level set,
// SnugBox (or the classic 3-sigma box when box3) and exact tile count; the
// record layout is that of GS_WS_RECORDS.
template <int D>
__device__ __forceinline__ void preprocess_item(const ViewDev &cam, int64_t item, float3 p, float4 quat, float3 ls,
                                                float logit, const float *shrow, float4 *__restrict__ rec,
                                                float2 *__restrict__ bin, uint32_t *__restrict__ touched,
                                                uint2 *__restrict__ rects, uint32_t *__restrict__ dkey,
                                                uint32_t *__restrict__ dval, int box3) {
    constexpr int K = (D + 1) * (D + 1);
    dval[item] = (uint32_t)item;

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
    project_cov(cam, p, quat, ls, P);
    const float a = P.Syy / P.det, b = -P.Sxy / P.det, c = P.Sxx / P.det;
    // projected mean, compensated (rounded once from the exact projection of
    // the float32 mean), so pixel-level decisions do not inherit the rounding
    // of the camera transform at large pixel coordinates
    const FF mxf = affine_ff(cam.fx, div_ff(dot3_plus(cam.R, p, cam.t[0]), zf), cam.cx);
    const FF myf = affine_ff(cam.fy, div_ff(dot3_plus(cam.R + 3, p, cam.t[1]), zf), cam.cy);
    const float mx = mxf.hi, my = myf.hi;
    const float o = 1.0f / (1.0f + expf(-logit));
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

}  // namespace gs
