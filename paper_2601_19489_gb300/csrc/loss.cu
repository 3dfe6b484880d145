// a6: photometric loss (Eq. 5) and disparity loss (Sec. 3.1) with their
// image gradients.
//
// SSIM uses an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2,
// zero-padded same-size windows per (view, channel) plane, averaged over all
// channels and pixels.  With mu_x = w*x, E_xx = w*(x^2), E_xy = w*(x y) the
// per-pixel SSIM is S(mu_x, E_xx, E_xy); its gradient w.r.t. x is
//   dS/dx(q) = sum_p w(p - q) [dS/dmu_x(p) + 2 x(q) dS/dE_xx(p) + y(q) dS/dE_xy(p)],
// i.e. the same symmetric window applied to three per-pixel maps.  Pass 1
// computes S and the three maps (separable blur of x, y, x^2, y^2, x y in a
// 42x42 shared-memory tile), pass 2 blurs the maps and forms dL/dx.  The
// quantities that share a window weight are summed in packed float32 pairs
// ((mu_x, mu_y), (E_xx, E_yy), (dS/dmu_x, dS/dE_xx)): one f32x2 FMA per tap
// for two of them.  The partial sums of the blocks are reduced in a fixed
// order by the first block of pass 2, after its own tile.
#include <math.h>

#include "gs_internal.cuh"

namespace gs {

constexpr int kSsimT = 32;              // output tile edge
constexpr int kHalo = 5;                // window radius
constexpr int kSsimIn = kSsimT + 2 * kHalo;  // 42
// 11 warps: the horizontal pass (42 rows x 8 groups of 4 outputs = 336
// items) and the vertical pass (256 items) each take one round
constexpr int kSsimThreads = 352;
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct Window {
    float w[11];
};

struct Planes {
    int V;
    int W[GS_MAX_VIEWS], H[GS_MAX_VIEWS];
    int64_t off[GS_MAX_VIEWS];  // pixel offset of each view
};

__device__ __forceinline__ float sgn(float d) { return (float)((d > 0.f) - (d < 0.f)); }

// Plane (view, channel) of a block and its geometry.
__device__ __forceinline__ bool plane_geom(const Planes &pl, int z, int *W, int *H, int64_t *base) {
    const int v = z / 3, c = z - 3 * v;
    *W = pl.W[v];
    *H = pl.H[v];
    *base = 3 * pl.off[v] + (int64_t)c * pl.W[v] * pl.H[v];
    return (int)blockIdx.x * kSsimT < *W && (int)blockIdx.y * kSsimT < *H;
}

__device__ __forceinline__ f2x ld2(const float2 &v) { return pk2(v.x, v.y); }
__device__ __forceinline__ float2 st2(f2x v) {
    float2 r;
    upk2(v, r.x, r.y);
    return r;
}

// Window sums of five quantities per pixel, in packed pairs where the
// quantities share the window weight: (mu_x, mu_y), (E_xx, E_yy) packed and
// E_xy alone.  Maps written for the backward: (dS/dmu_x, dS/dE_xx) packed
// and dS/dE_xy.
__global__ void __launch_bounds__(kSsimThreads)
k_ssim_fwd(Planes pl, Window win, const float *__restrict__ x, const float *__restrict__ y,
           float2 *__restrict__ maps_ab, float *__restrict__ maps_c, float *__restrict__ part_s,
           float *__restrict__ part_l1) {
    __shared__ float2 XY[kSsimIn][kSsimIn + 1];
    __shared__ float2 H2[2][kSsimIn][kSsimT + 1];  // horizontal sums: (mu_x, mu_y), (E_xx, E_yy)
    __shared__ float H1[kSsimIn][kSsimT + 1];      // horizontal sums: E_xy
    __shared__ float red[2][kSsimThreads / 32];
    int W, H;
    int64_t base;
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int tid = threadIdx.x;
    if (!plane_geom(pl, blockIdx.z, &W, &H, &base)) {
        if (tid == 0) {
            part_s[blk] = 0.f;
            part_l1[blk] = 0.f;
        }
        return;
    }
    f2x w2[11];
#pragma unroll
    for (int u = 0; u < 11; ++u) w2[u] = pk2(win.w[u], win.w[u]);
    const int ox = blockIdx.x * kSsimT - kHalo, oy = blockIdx.y * kSsimT - kHalo;
    for (int i = tid; i < kSsimIn * kSsimIn; i += kSsimThreads) {
        const int r = i / kSsimIn, c = i - r * kSsimIn;
        const int gx = ox + c, gy = oy + r;
        float a = 0.f, b = 0.f;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            a = x[base + (int64_t)gy * W + gx];
            b = y[base + (int64_t)gy * W + gx];
        }
        XY[r][c] = make_float2(a, b);
    }
    __syncthreads();
    // horizontal pass: a thread sums 4 adjacent outputs of a row from 14
    // inputs (register blocking: each input and its products are read once
    // for 4 outputs)
    for (int i = tid; i < kSsimIn * (kSsimT / 4); i += kSsimThreads) {
        const int r = i / (kSsimT / 4), c0 = 4 * (i - r * (kSsimT / 4));
        f2x s01[4], s23[4];
        float s4[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            s01[o] = pk2(0.f, 0.f);
            s23[o] = pk2(0.f, 0.f);
            s4[o] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            const float2 v = XY[r][c0 + k];
            const f2x xy = ld2(v), sq = mul2(xy, xy);
            const float p = v.x * v.y;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int u = k - o;  // tap of output c0 + o
                if (u >= 0 && u < 11) {
                    s01[o] = fma2(w2[u], xy, s01[o]);
                    s23[o] = fma2(w2[u], sq, s23[o]);
                    s4[o] = fmaf(win.w[u], p, s4[o]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            H2[0][r][c0 + o] = st2(s01[o]);
            H2[1][r][c0 + o] = st2(s23[o]);
            H1[r][c0 + o] = s4[o];
        }
    }
    __syncthreads();
    float acc_s = 0.f, acc_l1 = 0.f;
    // vertical pass: a thread sums 4 outputs of a column from 14 rows
    for (int i = tid; i < (kSsimT / 4) * kSsimT; i += kSsimThreads) {
        const int r0 = 4 * (i / kSsimT), c = i - (i / kSsimT) * kSsimT;
        f2x s01[4], s23[4];
        float s4[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            s01[o] = pk2(0.f, 0.f);
            s23[o] = pk2(0.f, 0.f);
            s4[o] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            const f2x a = ld2(H2[0][r0 + k][c]), b = ld2(H2[1][r0 + k][c]);
            const float e = H1[r0 + k][c];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int u = k - o;
                if (u >= 0 && u < 11) {
                    s01[o] = fma2(w2[u], a, s01[o]);
                    s23[o] = fma2(w2[u], b, s23[o]);
                    s4[o] = fmaf(win.w[u], e, s4[o]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int r = r0 + o;
            const int gx = blockIdx.x * kSsimT + c, gy = blockIdx.y * kSsimT + r;
            if (gx >= W || gy >= H) continue;
            float mx, my, exx, eyy;
            upk2(s01[o], mx, my);
            upk2(s23[o], exx, eyy);
            const float exy = s4[o];
            const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
            const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
            const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
            const float inv = 1.0f / (B1 * B2);
            const float S = A1 * A2 * inv;
            // partials w.r.t. mu_x, E_xx, E_xy (sxx = E_xx - mu_x^2, sxy = E_xy - mu_x mu_y)
            const float d_mu = 2.f * my * (A2 - A1) * inv - 2.f * mx * S * (1.0f / B1 - 1.0f / B2);
            const float d_exx = -S / B2;
            const float d_exy = 2.f * A1 * inv;
            const int64_t p = base + (int64_t)gy * W + gx;
            maps_ab[p] = make_float2(d_mu, d_exx);
            maps_c[p] = d_exy;
            acc_s += S;
            const float2 v = XY[r + kHalo][c + kHalo];
            acc_l1 += fabsf(v.x - v.y);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_s += __shfl_xor_sync(0xffffffffu, acc_s, o);
        acc_l1 += __shfl_xor_sync(0xffffffffu, acc_l1, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = acc_s;
        red[1][tid >> 5] = acc_l1;
    }
    __syncthreads();
    if (tid == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < kSsimThreads / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        part_s[blk] = a;
        part_l1[blk] = b;
    }
}

// The loss value: fixed-order reduction of the per-block partial sums in
// double by one block of threads (part_* fully written before the launch).
struct LossSums {
    const float *part_s, *part_l1, *part_d;
    int n_s, n_l1, n_d;
    double w_s, w_l1, w_d, s_const;
    float *loss;
};

template <int kThreads>
__device__ __forceinline__ void reduce_loss(const LossSums &L) {
    __shared__ double red[3][kThreads / 32];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < L.n_s; i += kThreads) a += L.part_s[i];
    for (int i = threadIdx.x; i < L.n_l1; i += kThreads) b += L.part_l1[i];
    for (int i = threadIdx.x; i < L.n_d; i += kThreads) c += L.part_d[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = b;
        red[2][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0, sc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            sa += red[0][w];
            sb += red[1][w];
            sc += red[2][w];
        }
        *L.loss = (float)(L.s_const + L.w_s * sa + L.w_l1 * sb + L.w_d * sc);
    }
}

// Gradient: the window sums of the three maps ((dS/dmu_x, dS/dE_xx) packed,
// dS/dE_xy alone) around each pixel.  Block (0, 0, 0) also reduces the loss
// value after its tile (the forward's partial sums and the disparity's are
// complete before this launch).
__global__ void __launch_bounds__(kSsimThreads)
k_ssim_bwd(Planes pl, Window win, const float *__restrict__ x, const float *__restrict__ y,
           const float2 *__restrict__ maps_ab, const float *__restrict__ maps_c, float c_l1, float c_ssim,
           float *__restrict__ grad, LossSums sums) {
    __shared__ float2 M2[kSsimIn][kSsimIn + 1];
    __shared__ float M1[kSsimIn][kSsimIn + 1];
    __shared__ float2 H2[kSsimIn][kSsimT + 1];
    __shared__ float H1[kSsimIn][kSsimT + 1];
    int W, H;
    int64_t base;
    const bool first = blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
    if (plane_geom(pl, blockIdx.z, &W, &H, &base)) {
        const int tid = threadIdx.x;
        f2x w2[11];
#pragma unroll
        for (int u = 0; u < 11; ++u) w2[u] = pk2(win.w[u], win.w[u]);
        const int ox = blockIdx.x * kSsimT - kHalo, oy = blockIdx.y * kSsimT - kHalo;
        for (int i = tid; i < kSsimIn * kSsimIn; i += kSsimThreads) {
            const int r = i / kSsimIn, c = i - r * kSsimIn;
            const int gx = ox + c, gy = oy + r;
            float2 ab = make_float2(0.f, 0.f);
            float d = 0.f;
            if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
                const int64_t p = base + (int64_t)gy * W + gx;
                ab = maps_ab[p];
                d = maps_c[p];
            }
            M2[r][c] = ab;
            M1[r][c] = d;
        }
        __syncthreads();
        // the same two register-blocked passes as the forward, over the maps
        for (int i = tid; i < kSsimIn * (kSsimT / 4); i += kSsimThreads) {
            const int r = i / (kSsimT / 4), c0 = 4 * (i - r * (kSsimT / 4));
            f2x s2[4];
            float s1[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                s2[o] = pk2(0.f, 0.f);
                s1[o] = 0.f;
            }
#pragma unroll
            for (int k = 0; k < 14; ++k) {
                const f2x v = ld2(M2[r][c0 + k]);
                const float e = M1[r][c0 + k];
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int u = k - o;
                    if (u >= 0 && u < 11) {
                        s2[o] = fma2(w2[u], v, s2[o]);
                        s1[o] = fmaf(win.w[u], e, s1[o]);
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                H2[r][c0 + o] = st2(s2[o]);
                H1[r][c0 + o] = s1[o];
            }
        }
        __syncthreads();
        for (int i = tid; i < (kSsimT / 4) * kSsimT; i += kSsimThreads) {
            const int r0 = 4 * (i / kSsimT), c = i - (i / kSsimT) * kSsimT;
            f2x s2[4];
            float s1[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                s2[o] = pk2(0.f, 0.f);
                s1[o] = 0.f;
            }
#pragma unroll
            for (int k = 0; k < 14; ++k) {
                const f2x v = ld2(H2[r0 + k][c]);
                const float e = H1[r0 + k][c];
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int u = k - o;
                    if (u >= 0 && u < 11) {
                        s2[o] = fma2(w2[u], v, s2[o]);
                        s1[o] = fmaf(win.w[u], e, s1[o]);
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int gx = blockIdx.x * kSsimT + c, gy = blockIdx.y * kSsimT + r0 + o;
                if (gx >= W || gy >= H) continue;
                const int64_t p = base + (int64_t)gy * W + gx;
                const float xv = x[p], yv = y[p];
                float dmu, dxx;
                upk2(s2[o], dmu, dxx);
                grad[p] = c_l1 * sgn(xv - yv) + c_ssim * (dmu + 2.f * xv * dxx + yv * s1[o]);
            }
        }
    }
    if (first) {
        __syncthreads();
        reduce_loss<kSsimThreads>(sums);
    }
}

// Plain L1 (lambda = 0): gradient and per-block partial sums.
__global__ void __launch_bounds__(256)
k_l1(const float *__restrict__ x, const float *__restrict__ y, int64_t n, float c_l1,
     float *__restrict__ grad, float *__restrict__ part) {
    __shared__ float red[8];
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const float d = x[i] - y[i];
        acc += fabsf(d);
        grad[i] = c_l1 * sgn(d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int w = 0; w < 8; ++w) a += red[w];
        part[blockIdx.x] = a;
    }
}

// Final loss when no SSIM pass runs (lambda = 0).
__global__ void __launch_bounds__(1024) k_loss_final(LossSums sums) { reduce_loss<1024>(sums); }

static Window make_window() {
    Window w;
    double s = 0.0, g[11];
    for (int u = 0; u < 11; ++u) {
        const double r = u - 5.0;
        g[u] = exp(-(r * r) / (2.0 * 1.5 * 1.5));
        s += g[u];
    }
    for (int u = 0; u < 11; ++u) w.w[u] = (float)(g[u] / s);
    return w;
}

static void ssim_grid(const gs_plan *plan, dim3 *grid) {
    int mw = 0, mh = 0;
    for (int v = 0; v < plan->V; ++v) {
        mw = plan->W[v] > mw ? plan->W[v] : mw;
        mh = plan->H[v] > mh ? plan->H[v] : mh;
    }
    *grid = dim3((mw + kSsimT - 1) / kSsimT, (mh + kSsimT - 1) / kSsimT, 3 * plan->V);
}

static constexpr int kL1Blocks = 4 * 152;

}  // namespace gs

using namespace gs;

extern "C" int64_t gs_loss_scratch_floats(const gs_plan *plan) {
    if (!plan) return 0;
    dim3 g;
    ssim_grid(plan, &g);
    const int64_t nblk = (int64_t)g.x * g.y * g.z;
    return 9 * plan->total_pixels + 2 * nblk + 2 * kL1Blocks + 64;
}

extern "C" int gs_loss(const gs_plan *plan, const float *rgb, const float *target, float lambda,
                       const float *disp, const float *target_disp, float disp_weight, float *dL_drgb,
                       float *dL_ddisp, float *loss, float *scratch, void *stream) {
    if (!plan || !rgb || !target || !dL_drgb || !loss || !scratch || lambda < 0.f || lambda > 1.f)
        return GS_ERR_ARG;
    if (disp && (!target_disp || !dL_ddisp)) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t P = plan->total_pixels;
    const int64_t n3 = 3 * P;
    dim3 grid;
    ssim_grid(plan, &grid);
    const int nblk = (int)(grid.x * grid.y * grid.z);
    float2 *maps_ab = reinterpret_cast<float2 *>(scratch);  // 3P pairs
    float *maps_c = scratch + 6 * P;                         // 3P
    float *part_s = scratch + 9 * P;
    float *part_l1 = part_s + nblk;
    float *part_d = part_l1 + nblk;
    float *part_l1b = part_d + kL1Blocks;
    if (((uintptr_t)scratch & 7) != 0) return GS_ERR_ARG;
    const double inv3p = 1.0 / (double)n3;
    LossSums sums{part_s, part_l1, part_d, 0, 0, 0, -(double)lambda * inv3p, (1.0 - lambda) * inv3p,
                  (double)disp_weight / (double)P, (double)lambda, loss};
    if (disp) {
        k_l1<<<kL1Blocks, 256, 0, s>>>(disp, target_disp, P, (float)(disp_weight / (double)P), dL_ddisp,
                                       part_d);
        sums.n_d = kL1Blocks;
    }
    if (lambda > 0.f) {
        Planes pl;
        pl.V = plan->V;
        for (int v = 0; v < plan->V; ++v) {
            pl.W[v] = plan->W[v];
            pl.H[v] = plan->H[v];
            pl.off[v] = plan->pix_off[v];
        }
        const Window win = make_window();
        k_ssim_fwd<<<grid, kSsimThreads, 0, s>>>(pl, win, rgb, target, maps_ab, maps_c, part_s, part_l1);
        sums.n_s = nblk;
        sums.n_l1 = nblk;
        k_ssim_bwd<<<grid, kSsimThreads, 0, s>>>(pl, win, rgb, target, maps_ab, maps_c,
                                                 (float)((1.0 - lambda) * inv3p), (float)(-lambda * inv3p), dL_drgb,
                                                 sums);
    } else {
        k_l1<<<kL1Blocks, 256, 0, s>>>(rgb, target, n3, (float)inv3p, dL_drgb, part_l1b);
        sums.part_l1 = part_l1b;
        sums.n_l1 = kL1Blocks;
        k_loss_final<<<1, 1024, 0, s>>>(sums);
    }
    return launch_error();
}
