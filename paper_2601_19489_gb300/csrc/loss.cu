// a6: photometric loss (Eq. 5) and disparity loss (Sec. 3.1) with their
// image gradients.
//
// SSIM uses an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2,
// zero-padded same-size windows per (view, channel) plane, averaged over all
// channels and pixels.  With mu_x = w*x, E_xx = w*(x^2), E_xy = w*(x y) the
// per-pixel SSIM is S(mu_x, E_xx, E_xy); its gradient w.r.t. x is
//   dS/dx(q) = sum_p w(p - q) [dS/dmu_x(p) + 2 x(q) dS/dE_xx(p) + y(q) dS/dE_xy(p)],
// i.e. the same symmetric window applied to three per-pixel maps.
//
// One launch does both (k_ssim_fused).  A CTA owns a strip of 32 output
// columns and a segment of output rows of one plane (48 to 256 rows, chosen
// per launch so the grid fills whole waves) and walks down it in chunks of 16
// rows.  Per chunk it loads 16 new input rows, blurs them horizontally (five
// sums per column, over the 42 statistic columns the strip needs), blurs the
// horizontal sums vertically into the statistics of 16 map rows five rows
// behind, forms S and the three maps there, blurs the maps horizontally, and
// blurs those sums vertically into the gradient of 16 output rows ten rows
// behind the input.  The horizontal sums of both blurs live in 32-row rings
// in shared memory, so the rows the window shares with the next chunk are
// kept, not recomputed: only the strip's 10 halo columns and the first
// chunk's 20 halo rows are computed twice.  Nothing but the gradient goes to
// HBM.  Quantities that share a window weight are summed in packed float32
// pairs ((x, y), (x^2, y^2), (dS/dmu_x, dS/dE_xx)): one f32x2 FMA per tap
// for two of them.  Each block writes its partial sums; the last block to
// finish (atomic counter) reduces them in a fixed order.
#include <math.h>

#include "gs_internal.cuh"

namespace gs {

constexpr int kSsimT = 32;                    // output columns of a strip
constexpr int kHalo = 5;                      // window radius
constexpr int kSegHMin = 48, kSegHMax = 256;  // output rows of a CTA (chosen per launch)
constexpr int kR = 16;                        // rows per chunk
constexpr int kRing = 32;                     // rows of the horizontal-sum rings
constexpr int kStatW = kSsimT + 2 * kHalo;    // 42 statistic / map columns
constexpr int kHGroups = (kStatW + 3) / 4;    // 11 groups of 4 horizontal outputs (44 columns)
constexpr int kInW = 4 * kHGroups + 2 * kHalo;  // 54 input columns
constexpr int kSsimThreads = 256;
// outputs per thread in the two gradient passes (128 of the 256 threads
// work in them; 2 outputs per thread keeps all busy but was measured slower:
// 0.147 against 0.142 ms at 1080p)
constexpr int kGB = 4;
// row strides in elements: odd, so that 16 consecutive rows of one column
// fall in 16 different banks
constexpr int kInS = 55, kHS = 45, kMpS = 43, kBhS = 33;
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct SsimSmem {
    union {
        float2 in[kR][kInS];  // this chunk's input rows (x, y)
        struct {
            float2 ab[kR][kMpS];  // this chunk's maps (dS/dmu_x, dS/dE_xx)
            float c[kR][kMpS];    // dS/dE_xy
        } mp;
    } u;
    float2 h01[kRing][kHS];    // horizontal sums of (x, y)
    float2 h23[kRing][kHS];    // of (x^2, y^2)
    float h4[kRing][kHS];      // of x y
    float2 bh01[kRing][kBhS];  // horizontal sums of the maps (dS/dmu_x, dS/dE_xx)
    float bh4[kRing][kBhS];    // of dS/dE_xy
    float red[2][kSsimThreads / 32];
    int last;
};

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
__device__ __forceinline__ bool plane_geom(const Planes &pl, int z, int seg_h, int *W, int *H, int64_t *base) {
    const int v = z / 3, c = z - 3 * v;
    *W = pl.W[v];
    *H = pl.H[v];
    *base = 3 * pl.off[v] + (int64_t)c * pl.W[v] * pl.H[v];
    return (int)blockIdx.x * kSsimT < *W && (int)blockIdx.y * seg_h < *H;
}

__device__ __forceinline__ f2x ld2(const float2 &v) { return *reinterpret_cast<const f2x *>(&v); }
__device__ __forceinline__ float2 st2(f2x v) {
    float2 r;
    upk2(v, r.x, r.y);
    return r;
}

// The loss value: fixed-order reduction of the per-block partial sums in
// double by one block of threads (part_* written by earlier launches, or by
// every other block of this launch before it counted itself done).
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
    for (int i = threadIdx.x; i < L.n_s; i += kThreads) a += __ldcg(L.part_s + i);
    for (int i = threadIdx.x; i < L.n_l1; i += kThreads) b += __ldcg(L.part_l1 + i);
    for (int i = threadIdx.x; i < L.n_d; i += kThreads) c += __ldcg(L.part_d + i);
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

// The whole SSIM pass of one (plane, strip, segment): statistics, maps,
// gradient and the block's partial sums (see the file's header).  Row
// bookkeeping for chunk k with a = y0 - 10 + 16 k: input rows [a, a + 16)
// are loaded and blurred horizontally; map rows [a - 5, a + 11) get their
// statistics (their windows need horizontal sums of rows [a - 10, a + 16));
// output rows [a - 10, a + 6) get their gradient (their windows need the
// maps' horizontal sums of rows [a - 15, a + 11)).
__global__ void __launch_bounds__(kSsimThreads, 4)
k_ssim_fused(Planes pl, Window win, int seg_h, const float *__restrict__ x, const float *__restrict__ y, float c_l1,
             float c_ssim, float *__restrict__ grad, float *__restrict__ part_s, float *__restrict__ part_l1,
             unsigned int *__restrict__ done_ctr, LossSums sums) {
    extern __shared__ __align__(16) unsigned char ssim_smem[];
    SsimSmem &sm = *reinterpret_cast<SsimSmem *>(ssim_smem);
    const int tid = threadIdx.x;
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int nblk = gridDim.x * gridDim.y * gridDim.z;
    int W, H;
    int64_t base;
    float acc_s = 0.f, acc_l1 = 0.f;
    if (plane_geom(pl, blockIdx.z, seg_h, &W, &H, &base)) {
        const float *__restrict__ xp = x + base;
        const float *__restrict__ yp = y + base;
        float *__restrict__ gp = grad + base;
        const int c0 = blockIdx.x * kSsimT, y0 = blockIdx.y * seg_h;
        const int y1 = min(y0 + seg_h, H);
        const int nchunks = (y1 - y0 + 4 + kR - 1) / kR + 1;
        f2x w2[11];
#pragma unroll
        for (int u = 0; u < 11; ++u) w2[u] = pk2(win.w[u], win.w[u]);
        // ring row of an image row (rows from y0 - 20 on)
        auto ring = [y0](int row) { return (row - y0 + 64) & (kRing - 1); };
        // this thread's place in each phase
        const int hr = tid & 15, hg = tid >> 4;              // horizontal passes: row, group of columns
        const int vq = tid / kStatW, vc = tid - vq * kStatW;  // statistics pass: row group, column
        const int gq = tid >> 5, gc = tid & 31;               // gradient pass: row group, column
        for (int k = 0; k < nchunks; ++k) {
            const int a = y0 - 2 * kHalo + kR * k;
            // (1) x, y of this thread's gradient pixels, fetched early
            float gx_[kGB], gy_[kGB];
            const int go0 = a - 2 * kHalo + kGB * gq;
            const bool gcol = c0 + gc < W;
#pragma unroll
            for (int o = 0; o < kGB; ++o) {
                gx_[o] = 0.f;
                gy_[o] = 0.f;
                const int row = go0 + o;
                if (k > 0 && tid < (kR / kGB) * kSsimT && gcol && row >= y0 && row < y1) {
                    const int64_t p = (int64_t)row * W + c0 + gc;
                    gx_[o] = __ldg(xp + p);
                    gy_[o] = __ldg(yp + p);
                }
            }
            // (2) input rows [a, a + 16), columns [c0 - 10, c0 + 44): warp w
            // takes rows 2w and 2w + 1, lanes the columns
            {
                const int lane = tid & 31, w = tid >> 5;
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) {
                    const int r = 2 * w + rr, gyy = a + r;
                    const bool rowin = gyy >= 0 && gyy < H;
                    const int64_t rb = (int64_t)gyy * W;
#pragma unroll
                    for (int cc = lane; cc < kInW; cc += 32) {
                        const int gxx = c0 - 2 * kHalo + cc;
                        float2 v = make_float2(0.f, 0.f);
                        if (rowin && gxx >= 0 && gxx < W) v = make_float2(__ldg(xp + rb + gxx), __ldg(yp + rb + gxx));
                        sm.u.in[r][cc] = v;
                    }
                }
            }
            __syncthreads();
            // (3) horizontal sums of input row a + hr at statistic columns
            // 4 hg .. 4 hg + 3 (column j is image column c0 - 5 + j), from
            // input columns 4 hg .. 4 hg + 13: each input read once for 4 outputs
            if (tid < kR * kHGroups) {
                f2x s01[4], s23[4];
                float s4[4];
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    s01[o] = pk2(0.f, 0.f);
                    s23[o] = pk2(0.f, 0.f);
                    s4[o] = 0.f;
                }
#pragma unroll
                for (int kk = 0; kk < 14; ++kk) {
                    const f2x xy = ld2(sm.u.in[hr][4 * hg + kk]);
                    float xv, yv;
                    upk2(xy, xv, yv);
                    const f2x sq = mul2(xy, xy);
                    const float p = xv * yv;
#pragma unroll
                    for (int o = 0; o < 4; ++o) {
                        const int u = kk - o;
                        if (u >= 0 && u < 11) {
                            s01[o] = fma2(w2[u], xy, s01[o]);
                            s23[o] = fma2(w2[u], sq, s23[o]);
                            s4[o] = fmaf(win.w[u], p, s4[o]);
                        }
                    }
                }
                const int rr = ring(a + hr);
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    sm.h01[rr][4 * hg + o] = st2(s01[o]);
                    sm.h23[rr][4 * hg + o] = st2(s23[o]);
                    sm.h4[rr][4 * hg + o] = s4[o];
                }
            }
            __syncthreads();
            // (4) statistics and maps of map rows m0 .. m0 + 3 at column vc
            // (vertical sums over horizontal-sum rows m0 - 5 .. m0 + 8); rows
            // outside the image, or before y0 - 5 (not needed, their rows of
            // horizontal sums were not computed), get zero maps
            if (tid < 4 * kStatW) {
                const int m0 = a - kHalo + 4 * vq;
                const int gxs = c0 - kHalo + vc;
                f2x s01[4], s23[4];
                float s4[4];
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    s01[o] = pk2(0.f, 0.f);
                    s23[o] = pk2(0.f, 0.f);
                    s4[o] = 0.f;
                }
                if (m0 + 3 >= y0 - kHalo) {
#pragma unroll
                    for (int kk = 0; kk < 14; ++kk) {
                        const int rr = ring(m0 - kHalo + kk);
                        const f2x h01 = ld2(sm.h01[rr][vc]), h23 = ld2(sm.h23[rr][vc]);
                        const float h4 = sm.h4[rr][vc];
#pragma unroll
                        for (int o = 0; o < 4; ++o) {
                            const int u = kk - o;
                            if (u >= 0 && u < 11) {
                                s01[o] = fma2(w2[u], h01, s01[o]);
                                s23[o] = fma2(w2[u], h23, s23[o]);
                                s4[o] = fmaf(win.w[u], h4, s4[o]);
                            }
                        }
                    }
                }
                const bool colin = gxs >= 0 && gxs < W;
                const bool counted = vc >= kHalo && vc < kHalo + kSsimT && colin;
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int m = m0 + o;
                    float d_mu = 0.f, d_exx = 0.f, d_exy = 0.f;
                    if (colin && m >= 0 && m < H && m >= y0 - kHalo) {
                        float mx, my, exx, eyy;
                        upk2(s01[o], mx, my);
                        upk2(s23[o], exx, eyy);
                        const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = s4[o] - mx * my;
                        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
                        const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
                        const float rB1 = fast_rcp(B1), rB2 = fast_rcp(B2);
                        const float inv = rB1 * rB2;
                        const float S = A1 * A2 * inv;
                        // partials w.r.t. mu_x, E_xx, E_xy (sxx = E_xx - mu_x^2, sxy = E_xy - mu_x mu_y)
                        d_mu = 2.f * my * (A2 - A1) * inv - 2.f * mx * S * (rB1 - rB2);
                        d_exx = -S * rB2;
                        d_exy = 2.f * A1 * inv;
                        if (counted && m >= y0 && m < y1) acc_s += S;
                    }
                    sm.u.mp.ab[4 * vq + o][vc] = make_float2(d_mu, d_exx);
                    sm.u.mp.c[4 * vq + o][vc] = d_exy;
                }
            }
            __syncthreads();
            // (5) horizontal sums of the maps of map row a - 5 + hr at output
            // columns kGB hg .. kGB hg + kGB - 1, from map columns kGB hg ..
            // kGB hg + kGB + 9
            if (tid < kR * (kSsimT / kGB)) {
                f2x s2[kGB];
                float s1[kGB];
#pragma unroll
                for (int o = 0; o < kGB; ++o) {
                    s2[o] = pk2(0.f, 0.f);
                    s1[o] = 0.f;
                }
#pragma unroll
                for (int kk = 0; kk < 10 + kGB; ++kk) {
                    const f2x v = ld2(sm.u.mp.ab[hr][kGB * hg + kk]);
                    const float e = sm.u.mp.c[hr][kGB * hg + kk];
#pragma unroll
                    for (int o = 0; o < kGB; ++o) {
                        const int u = kk - o;
                        if (u >= 0 && u < 11) {
                            s2[o] = fma2(w2[u], v, s2[o]);
                            s1[o] = fmaf(win.w[u], e, s1[o]);
                        }
                    }
                }
                const int rr = ring(a - kHalo + hr);
#pragma unroll
                for (int o = 0; o < kGB; ++o) {
                    sm.bh01[rr][kGB * hg + o] = st2(s2[o]);
                    sm.bh4[rr][kGB * hg + o] = s1[o];
                }
            }
            __syncthreads();
            // (6) gradient of output rows go0 .. go0 + kGB - 1 at column gc
            // (vertical sums over map rows go0 - 5 .. go0 + kGB + 4); the
            // first chunk has no output rows inside the segment
            if (k > 0 && tid < (kR / kGB) * kSsimT) {
                f2x s2[kGB];
                float s1[kGB];
#pragma unroll
                for (int o = 0; o < kGB; ++o) {
                    s2[o] = pk2(0.f, 0.f);
                    s1[o] = 0.f;
                }
#pragma unroll
                for (int kk = 0; kk < 10 + kGB; ++kk) {
                    const int rr = ring(go0 - kHalo + kk);
                    const f2x v = ld2(sm.bh01[rr][gc]);
                    const float e = sm.bh4[rr][gc];
#pragma unroll
                    for (int o = 0; o < kGB; ++o) {
                        const int u = kk - o;
                        if (u >= 0 && u < 11) {
                            s2[o] = fma2(w2[u], v, s2[o]);
                            s1[o] = fmaf(win.w[u], e, s1[o]);
                        }
                    }
                }
#pragma unroll
                for (int o = 0; o < kGB; ++o) {
                    const int row = go0 + o;
                    if (gcol && row >= y0 && row < y1) {
                        float dmu, dxx;
                        upk2(s2[o], dmu, dxx);
                        const float xv = gx_[o], yv = gy_[o];
                        gp[(int64_t)row * W + c0 + gc] =
                            c_l1 * sgn(xv - yv) + c_ssim * (dmu + 2.f * xv * dxx + yv * s1[o]);
                        acc_l1 += fabsf(xv - yv);
                    }
                }
            }
            // the next chunk's first write (input rows, aliasing the maps)
            // comes after step 5's barrier; its ring writes come after its
            // own barriers, when this chunk's reads are done
        }
    }
    // block partial sums, then the last block to finish reduces them all
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_s += __shfl_xor_sync(0xffffffffu, acc_s, o);
        acc_l1 += __shfl_xor_sync(0xffffffffu, acc_l1, o);
    }
    if ((tid & 31) == 0) {
        sm.red[0][tid >> 5] = acc_s;
        sm.red[1][tid >> 5] = acc_l1;
    }
    __syncthreads();
    if (tid == 0) {
        float s = 0.f, l = 0.f;
        for (int w = 0; w < kSsimThreads / 32; ++w) {
            s += sm.red[0][w];
            l += sm.red[1][w];
        }
        part_s[blk] = s;
        part_l1[blk] = l;
        __threadfence();
        sm.last = atomicAdd(done_ctr, 1u) == (unsigned int)(nblk - 1);
    }
    __syncthreads();
    if (sm.last) {
        __threadfence();
        reduce_loss<kSsimThreads>(sums);
        if (tid == 0) *done_ctr = 0u;
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

// Grid of the fused SSIM pass: 32-column strips x segments of seg_h rows x
// planes.  seg_h trades the first chunk's halo rows (20 input rows per
// segment) against whole waves of CTAs (4 resident per SM): it minimises
// waves x chunks per CTA.  seg_h = 0 gives the smallest height (the most
// blocks, for sizing the scratch).
static void ssim_grid(const gs_plan *plan, int sms, dim3 *grid, int *seg_h) {
    int mw = 0, mh = 0;
    for (int v = 0; v < plan->V; ++v) {
        mw = plan->W[v] > mw ? plan->W[v] : mw;
        mh = plan->H[v] > mh ? plan->H[v] : mh;
    }
    const int64_t strips = (int64_t)((mw + kSsimT - 1) / kSsimT) * 3 * plan->V;
    int best = kSegHMin;
    if (sms > 0) {
        int64_t best_cost = -1;
        for (int sh = kSegHMin; sh <= kSegHMax; sh += 4) {
            const int64_t ctas = strips * ((mh + sh - 1) / sh);
            const int64_t waves = (ctas + 4 * sms - 1) / (4 * sms);
            const int64_t cost = waves * ((sh + 4 + kR - 1) / kR + 1);
            if (best_cost < 0 || cost < best_cost) {
                best_cost = cost;
                best = sh;
            }
        }
    }
    *seg_h = best;
    *grid = dim3((mw + kSsimT - 1) / kSsimT, (mh + best - 1) / best, 3 * plan->V);
}

static int device_sms() {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev < 0 || dev >= 64) return 152;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms[dev] = 152;
    return sms[dev];
}

// The fused kernel's shared memory exceeds the 48 KB default: raise the
// limit once per device.
static int ssim_smem_setup() {
    static bool done[64] = {};
    int dev = 0;
    int rc = check_cuda(cudaGetDevice(&dev));
    if (rc) return rc;
    if (dev >= 0 && dev < 64 && done[dev]) return GS_OK;
    rc = check_cuda(cudaFuncSetAttribute(k_ssim_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(SsimSmem)));
    if (rc == GS_OK && dev >= 0 && dev < 64) done[dev] = true;
    return rc;
}

static constexpr int kL1Blocks = 4 * 152;

}  // namespace gs

using namespace gs;

extern "C" int64_t gs_loss_scratch_floats(const gs_plan *plan) {
    if (!plan) return 0;
    dim3 g;
    int seg_h;
    ssim_grid(plan, 0, &g, &seg_h);  // the most blocks any launch can have
    const int64_t nblk = (int64_t)g.x * g.y * g.z;
    return 2 * nblk + 2 * kL1Blocks + 64;
}

extern "C" int gs_loss(const gs_plan *plan, const float *rgb, const float *target, float lambda,
                       const float *disp, const float *target_disp, float disp_weight, float *dL_drgb,
                       float *dL_ddisp, float *loss, float *scratch, void *stream) {
    if (!plan || !rgb || !target || !dL_drgb || !loss || !scratch || lambda < 0.f || lambda > 1.f)
        return GS_ERR_ARG;
    if (disp && (!target_disp || !dL_ddisp)) return GS_ERR_ARG;
    if (((uintptr_t)scratch & 7) != 0) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t P = plan->total_pixels;
    const int64_t n3 = 3 * P;
    dim3 grid;
    int seg_h;
    ssim_grid(plan, device_sms(), &grid, &seg_h);
    const int nblk = (int)(grid.x * grid.y * grid.z);
    float *part_s = scratch;
    float *part_l1 = part_s + nblk;
    float *part_d = part_l1 + nblk;
    float *part_l1b = part_d + kL1Blocks;
    unsigned int *done_ctr = reinterpret_cast<unsigned int *>(part_l1b + kL1Blocks);
    const double inv3p = 1.0 / (double)n3;
    LossSums sums{part_s, part_l1, part_d, 0, 0, 0, -(double)lambda * inv3p, (1.0 - lambda) * inv3p,
                  (double)disp_weight / (double)P, (double)lambda, loss};
    if (disp) {
        k_l1<<<kL1Blocks, 256, 0, s>>>(disp, target_disp, P, (float)(disp_weight / (double)P), dL_ddisp,
                                       part_d);
        sums.n_d = kL1Blocks;
    }
    if (lambda > 0.f) {
        int rc = ssim_smem_setup();
        if (rc) return rc;
        Planes pl;
        pl.V = plan->V;
        for (int v = 0; v < plan->V; ++v) {
            pl.W[v] = plan->W[v];
            pl.H[v] = plan->H[v];
            pl.off[v] = plan->pix_off[v];
        }
        const Window win = make_window();
        sums.n_s = nblk;
        sums.n_l1 = nblk;
        rc = check_cuda(cudaMemsetAsync(done_ctr, 0, sizeof(unsigned int), s));
        if (rc) return rc;
        k_ssim_fused<<<grid, kSsimThreads, sizeof(SsimSmem), s>>>(pl, win, seg_h, rgb, target,
                                                                  (float)((1.0 - lambda) * inv3p),
                                                                  (float)(-lambda * inv3p), dL_drgb, part_s, part_l1,
                                                                  done_ctr, sums);
    } else {
        k_l1<<<kL1Blocks, 256, 0, s>>>(rgb, target, n3, (float)inv3p, dL_drgb, part_l1b);
        sums.part_l1 = part_l1b;
        sums.n_l1 = kL1Blocks;
        k_loss_final<<<1, 1024, 0, s>>>(sums);
    }
    return launch_error();
}
