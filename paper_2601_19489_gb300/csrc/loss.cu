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
// 42x42 shared-memory tile), pass 2 blurs the maps and forms dL/dx; partial
// sums per block are reduced in a fixed order by one block.
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

__global__ void __launch_bounds__(kSsimThreads)
k_ssim_fwd(Planes pl, Window win, const float *__restrict__ x, const float *__restrict__ y,
           float *__restrict__ maps, int64_t plane_stride, float *__restrict__ part_s,
           float *__restrict__ part_l1) {
    __shared__ float X[kSsimIn][kSsimIn + 1];
    __shared__ float Yv[kSsimIn][kSsimIn + 1];
    __shared__ float Hs[5][kSsimIn][kSsimT + 1];
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
    const int ox = blockIdx.x * kSsimT - kHalo, oy = blockIdx.y * kSsimT - kHalo;
    for (int i = tid; i < kSsimIn * kSsimIn; i += kSsimThreads) {
        const int r = i / kSsimIn, c = i - r * kSsimIn;
        const int gx = ox + c, gy = oy + r;
        float a = 0.f, b = 0.f;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            a = x[base + (int64_t)gy * W + gx];
            b = y[base + (int64_t)gy * W + gx];
        }
        X[r][c] = a;
        Yv[r][c] = b;
    }
    __syncthreads();
    // horizontal pass: a thread blurs 4 adjacent outputs of a row from 14
    // loaded inputs (register blocking: each input and its products are
    // read once for 4 outputs)
    for (int i = tid; i < kSsimIn * (kSsimT / 4); i += kSsimThreads) {
        const int r = i / (kSsimT / 4), c0 = 4 * (i - r * (kSsimT / 4));
        float s[5][4];
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
            for (int o = 0; o < 4; ++o) s[q][o] = 0.f;
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            const float a = X[r][c0 + k], b = Yv[r][c0 + k];
            const float v[5] = {a, b, a * a, b * b, a * b};
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int u = k - o;  // tap of output c0 + o
                if (u >= 0 && u < 11) {
#pragma unroll
                    for (int q = 0; q < 5; ++q) s[q][o] += win.w[u] * v[q];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
            for (int o = 0; o < 4; ++o) Hs[q][r][c0 + o] = s[q][o];
    }
    __syncthreads();
    float acc_s = 0.f, acc_l1 = 0.f;
    const int64_t npl = (int64_t)W * H;
    // vertical pass: a thread blurs 4 outputs of a column from 14 rows
    for (int i = tid; i < (kSsimT / 4) * kSsimT; i += kSsimThreads) {
        const int r0 = 4 * (i / kSsimT), c = i - (i / kSsimT) * kSsimT;
        float s[5][4];
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
            for (int o = 0; o < 4; ++o) s[q][o] = 0.f;
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            float v[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) v[q] = Hs[q][r0 + k][c];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int u = k - o;
                if (u >= 0 && u < 11) {
#pragma unroll
                    for (int q = 0; q < 5; ++q) s[q][o] += win.w[u] * v[q];
                }
            }
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int r = r0 + o;
            const int gx = blockIdx.x * kSsimT + c, gy = blockIdx.y * kSsimT + r;
            if (gx >= W || gy >= H) continue;
            const float mx = s[0][o], my = s[1][o], exx = s[2][o], eyy = s[3][o], exy = s[4][o];
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
            maps[p] = d_mu;
            maps[plane_stride + p] = d_exx;
            maps[2 * plane_stride + p] = d_exy;
            acc_s += S;
            acc_l1 += fabsf(X[r + kHalo][c + kHalo] - Yv[r + kHalo][c + kHalo]);
        }
    }
    (void)npl;
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

__global__ void __launch_bounds__(kSsimThreads)
k_ssim_bwd(Planes pl, Window win, const float *__restrict__ x, const float *__restrict__ y,
           const float *__restrict__ maps, int64_t plane_stride, float c_l1, float c_ssim,
           float *__restrict__ grad) {
    __shared__ float M[3][kSsimIn][kSsimIn + 1];
    __shared__ float Hs[3][kSsimIn][kSsimT + 1];
    int W, H;
    int64_t base;
    if (!plane_geom(pl, blockIdx.z, &W, &H, &base)) return;
    const int tid = threadIdx.x;
    const int ox = blockIdx.x * kSsimT - kHalo, oy = blockIdx.y * kSsimT - kHalo;
    for (int i = tid; i < kSsimIn * kSsimIn; i += kSsimThreads) {
        const int r = i / kSsimIn, c = i - r * kSsimIn;
        const int gx = ox + c, gy = oy + r;
        float a = 0.f, b = 0.f, d = 0.f;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const int64_t p = base + (int64_t)gy * W + gx;
            a = maps[p];
            b = maps[plane_stride + p];
            d = maps[2 * plane_stride + p];
        }
        M[0][r][c] = a;
        M[1][r][c] = b;
        M[2][r][c] = d;
    }
    __syncthreads();
    // the same two register-blocked passes as the forward, over 3 maps
    for (int i = tid; i < kSsimIn * (kSsimT / 4); i += kSsimThreads) {
        const int r = i / (kSsimT / 4), c0 = 4 * (i - r * (kSsimT / 4));
        float s[3][4];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int o = 0; o < 4; ++o) s[q][o] = 0.f;
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            const float v[3] = {M[0][r][c0 + k], M[1][r][c0 + k], M[2][r][c0 + k]};
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int u = k - o;
                if (u >= 0 && u < 11) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) s[q][o] += win.w[u] * v[q];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int o = 0; o < 4; ++o) Hs[q][r][c0 + o] = s[q][o];
    }
    __syncthreads();
    for (int i = tid; i < (kSsimT / 4) * kSsimT; i += kSsimThreads) {
        const int r0 = 4 * (i / kSsimT), c = i - (i / kSsimT) * kSsimT;
        float s[3][4];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int o = 0; o < 4; ++o) s[q][o] = 0.f;
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            const float v[3] = {Hs[0][r0 + k][c], Hs[1][r0 + k][c], Hs[2][r0 + k][c]};
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int u = k - o;
                if (u >= 0 && u < 11) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) s[q][o] += win.w[u] * v[q];
                }
            }
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int gx = blockIdx.x * kSsimT + c, gy = blockIdx.y * kSsimT + r0 + o;
            if (gx >= W || gy >= H) continue;
            const int64_t p = base + (int64_t)gy * W + gx;
            const float xv = x[p], yv = y[p];
            grad[p] = c_l1 * sgn(xv - yv) + c_ssim * (s[0][o] + 2.f * xv * s[1][o] + yv * s[2][o]);
        }
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

// Final loss: fixed-order reduction of the partial sums in double.
__global__ void __launch_bounds__(1024)
k_loss_final(const float *__restrict__ part_s, int n_s, const float *__restrict__ part_l1, int n_l1,
             const float *__restrict__ part_d, int n_d, double w_s, double w_l1, double w_d,
             double s_const, float *__restrict__ loss) {
    __shared__ double red[3][32];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < n_s; i += 1024) a += part_s[i];
    for (int i = threadIdx.x; i < n_l1; i += 1024) b += part_l1[i];
    for (int i = threadIdx.x; i < n_d; i += 1024) c += part_d[i];
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
        for (int w = 0; w < 32; ++w) {
            sa += red[0][w];
            sb += red[1][w];
            sc += red[2][w];
        }
        *loss = (float)(s_const + w_s * sa + w_l1 * sb + w_d * sc);
    }
}

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
    float *maps = scratch;
    float *part_s = scratch + 9 * P;
    float *part_l1 = part_s + nblk;
    float *part_d = part_l1 + nblk;
    float *part_l1b = part_d + kL1Blocks;
    const double inv3p = 1.0 / (double)n3;
    int n_s = 0, n_l1 = 0, n_d = 0;
    const float *pl1 = part_l1;
    if (lambda > 0.f) {
        Planes pl;
        pl.V = plan->V;
        for (int v = 0; v < plan->V; ++v) {
            pl.W[v] = plan->W[v];
            pl.H[v] = plan->H[v];
            pl.off[v] = plan->pix_off[v];
        }
        const Window win = make_window();
        k_ssim_fwd<<<grid, kSsimThreads, 0, s>>>(pl, win, rgb, target, maps, n3, part_s, part_l1);
        k_ssim_bwd<<<grid, kSsimThreads, 0, s>>>(pl, win, rgb, target, maps, n3, (float)((1.0 - lambda) * inv3p),
                                        (float)(-lambda * inv3p), dL_drgb);
        n_s = nblk;
        n_l1 = nblk;
    } else {
        k_l1<<<kL1Blocks, 256, 0, s>>>(rgb, target, n3, (float)inv3p, dL_drgb, part_l1b);
        pl1 = part_l1b;
        n_l1 = kL1Blocks;
    }
    if (disp) {
        k_l1<<<kL1Blocks, 256, 0, s>>>(disp, target_disp, P, (float)(disp_weight / (double)P), dL_ddisp,
                                       part_d);
        n_d = kL1Blocks;
    }
    k_loss_final<<<1, 1024, 0, s>>>(part_s, n_s, pl1, n_l1, part_d, n_d, -(double)lambda * inv3p,
                                    (1.0 - lambda) * inv3p, (double)disp_weight / (double)P,
                                    (double)lambda, loss);
    return launch_error();
}
