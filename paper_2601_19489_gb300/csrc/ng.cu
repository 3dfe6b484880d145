// a10: neural-Gaussian decoder (Sec. 2.3) on the 5th-generation tensor cores.
//
// An anchor carries a feature f (32), an offset log-scale (3) and a child
// log-scale (3); a shallow MLP shared by all anchors maps x = [f, view
// direction] (35) through h = ReLU(W1 x + b1) (32) to y = W2 h + b2 (140),
// 14 outputs for each of 10 child Gaussians:
//   mean = anchor + tanh(y0..2) e^{s_off};  opacity = tanh(y3) (children with
//   opacity <= 0 are not rendered);  colour = sigmoid(y4..6);
//   log-scale = s_scale + log sigmoid(y7..9);  rotation = y10..13.
// The children are written as ordinary Gaussian parameters (opacity logit,
// SH degree 0) for the splatting step, and the backward maps the children's
// parameter gradients back to the anchors and the MLP.
//
// Both GEMMs of the forward and both per-anchor GEMMs of the backward run as
// tcgen05.mma kind::f16 (bf16 operands, fp32 accumulators in tensor memory),
// M = 128 anchors per CTA, operands staged in shared memory in the canonical
// no-swizzle K-major layout (8 x 16-byte core matrices).  One thread issues
// the MMAs; tcgen05.commit arrives on an mbarrier that the CTA waits on with
// a bounded spin.  The weight gradients (sums over anchors) are formed per CTA
// and reduced over CTAs in a fixed order.
#include <cuda_bf16.h>
#include <stddef.h>

#include "gs_internal.cuh"
#include "preprocess_item.cuh"

namespace gs {
namespace ng {

constexpr int kTileA = 128;             // anchors per CTA = UMMA M
constexpr int kFeat = GS_NG_FEAT;       // 32
constexpr int kIn = kFeat + 3;          // 35
constexpr int kInPad = 48;              // GEMM 1 K (3 x 16)
constexpr int kHid = GS_NG_HIDDEN;      // 32
constexpr int kChild = GS_NG_CHILDREN;  // 10
constexpr int kPer = 14;                // outputs per child
constexpr int kOut = kChild * kPer;     // 140
constexpr int kOutPad = 144;            // GEMM 2 N, backward GEMM K (9 x 16)
constexpr int kFwdThreads = kTileA;    // forward: one thread per anchor
constexpr int kThreads = 3 * kTileA;  // backward: three threads per anchor
constexpr int kTmemCols = 256;
constexpr float kLogitFloor = -30.0f;
constexpr float kOpacityCeil = 1.0f - 1e-6f;
constexpr float kDcScale = 3.5449077018110318f;  // 2 sqrt(pi): SH DC coefficient per unit colour
constexpr int kPartial = kOut * kHid + kHid * kIn + kOut + kHid;  // dW2, dW1, db2, db1 per CTA
constexpr long long kWaitLimit = 1ll << 22;                       // bounded mbarrier spin

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, int ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for the mbarrier phase with the given parity; false after `limit`
// tries (kWaitLimit in every kernel of the decoder).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit = kWaitLimit) {
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Shared-memory matrix descriptor, no swizzle: start address, leading
// (K-direction) and stride (8-row direction) byte offsets, version 1.
__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo) {
    const uint32_t a = smem_u32(p);
    uint64_t d = (uint64_t)((a & 0x3ffffu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3fffu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3fffu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Expect `bytes` of bulk-copy transactions on the mbarrier (one arrival).
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Element (r, k) of an R x K bf16 operand in the canonical no-swizzle
// K-major layout: 8 x 8 core matrices of 128 contiguous bytes, the K chunks of
// a row group adjacent (LBO = 128 B), row groups K * 16 B apart (SBO).
__host__ __device__ constexpr int canon(int r, int k, int K) {
    return (r >> 3) * (K * 8) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// log(sigmoid(x)) = -softplus(-x), stable for large |x|
__device__ __forceinline__ float log_sigmoidf(float x) {
    return x >= 0.0f ? -log1pf(expf(-x)) : x - log1pf(expf(x));
}

struct Args {
    int64_t n;  // anchors
    const float *xyz, *feat, *ls, *b1, *b2;
    float cam[3];
    const __nv_bfloat16 *w1b, *w2b, *w2tb, *w1tb;  // prepared bf16 weights (canonical operand layout, padded)
    __nv_bfloat16 *h_store;                        // bf16 h per anchor (forward -> backward)
    // forward outputs (children)
    float *c_means, *c_ls, *c_quats, *c_logits, *c_sh;
    // backward inputs (children's gradients) and outputs
    float *g_means, *g_ls, *g_quats, *g_logits, *g_sh;
    int zero_g;  // zero the children's gradients after reading them
    int grads_bulk;  // the children's gradient arrays start 16-byte aligned (bulk copies)
    int feat_vec;  // feat and d_feat are 16-byte aligned (float4 rows)
    float *d_feat, *d_ls, *partial;
    int *err;
    // fused decode + preprocess: the plan's view and its preprocess outputs
    ViewDev view;
    float4 *rec;
    float2 *bin;
    uint32_t *touched, *dkey, *dval;
    uint2 *rects;
    int box3;
};

// ------------------------------------------------------------ weight prep
__global__ void __launch_bounds__(256) k_ng_prep(const float *__restrict__ w1, const float *__restrict__ w2,
                                                 __nv_bfloat16 *w1b, __nv_bfloat16 *w2b, __nv_bfloat16 *w2tb,
                                                 __nv_bfloat16 *w1tb) {
    for (int i = threadIdx.x; i < kHid * kInPad; i += blockDim.x) {  // W1 (32 x 48), K-major in the input
        const int r = i / kInPad, k = i % kInPad;
        w1b[canon(r, k, kInPad)] = __float2bfloat16_rn(k < kIn ? w1[r * kIn + k] : 0.0f);
    }
    for (int i = threadIdx.x; i < kOutPad * kHid; i += blockDim.x) {  // W2 (144 x 32)
        const int r = i / kHid, k = i % kHid;
        w2b[canon(r, k, kHid)] = __float2bfloat16_rn(r < kOut ? w2[r * kHid + k] : 0.0f);
    }
    for (int i = threadIdx.x; i < kHid * kOutPad; i += blockDim.x) {  // W2^T (32 x 144)
        const int r = i / kOutPad, k = i % kOutPad;
        w2tb[canon(r, k, kOutPad)] = __float2bfloat16_rn(k < kOut ? w2[k * kHid + r] : 0.0f);
    }
    for (int i = threadIdx.x; i < kInPad * kHid; i += blockDim.x) {  // W1^T (48 x 32)
        const int r = i / kHid, k = i % kHid;
        w1tb[canon(r, k, kHid)] = __float2bfloat16_rn(r < kIn ? w1[k * kIn + r] : 0.0f);
    }
}

// x row of anchor a (bf16-rounded feature and view direction, zero padded)
__device__ __forceinline__ void anchor_input(const Args &A, int64_t a, bool valid, float *x) {
    if (!valid) {
#pragma unroll
        for (int k = 0; k < kInPad; ++k) x[k] = 0.0f;
        return;
    }
    if (A.feat_vec) {
        const float4 *f4 = reinterpret_cast<const float4 *>(A.feat + a * kFeat);
#pragma unroll
        for (int q = 0; q < kFeat / 4; ++q) {
            const float4 f = f4[q];
            x[4 * q] = bf16r(f.x);
            x[4 * q + 1] = bf16r(f.y);
            x[4 * q + 2] = bf16r(f.z);
            x[4 * q + 3] = bf16r(f.w);
        }
    } else {
#pragma unroll
        for (int k = 0; k < kFeat; ++k) x[k] = bf16r(A.feat[a * kFeat + k]);
    }
    float d0 = A.xyz[3 * a] - A.cam[0], d1 = A.xyz[3 * a + 1] - A.cam[1], d2 = A.xyz[3 * a + 2] - A.cam[2];
    const float inv = 1.0f / sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    x[kFeat] = bf16r(d0 * inv);
    x[kFeat + 1] = bf16r(d1 * inv);
    x[kFeat + 2] = bf16r(d2 * inv);
#pragma unroll
    for (int k = kIn; k < kInPad; ++k) x[k] = 0.0f;
}

// Block copy of a prepared operand (already in the canonical layout) into
// shared memory, 16 bytes per thread and step.
template <int kStride = kThreads>
__device__ __forceinline__ void copy16(void *dst, const void *src, int bytes, int tid) {
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (int i = tid; i < bytes / 16; i += kStride) d[i] = s[i];
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- forward
struct FwdSmem {
    __nv_bfloat16 X[kTileA * kInPad];    // GEMM 1 A (M = 128, K = 48)
    __nv_bfloat16 W1[kHid * kInPad];     // GEMM 1 B (N = 32, K = 48)
    __nv_bfloat16 H[kTileA * kHid];      // GEMM 2 A (M = 128, K = 32)
    __nv_bfloat16 W2[kOutPad * kHid];    // GEMM 2 B (N = 144, K = 32)
    float Y[kTileA][kOutPad + 1];        // y = W2 h + b2
    float xyz[kTileA][3], ls[kTileA][6];
    float b1[kHid], b2[kOutPad];
    uint64_t mbar;
    uint32_t tmem;
    int fail;
};

// kPre: also the preprocess of every child (Sec. 2.3's decode fused with the
// per-Gaussian preprocess, the children's parameters passed on in registers)
template <bool kPre>
__global__ void __launch_bounds__(kFwdThreads) k_ng_fwd(Args A) {
    extern __shared__ uint8_t smem_raw[];
    FwdSmem &S = *reinterpret_cast<FwdSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t a0 = (int64_t)blockIdx.x * kTileA;
    const int64_t a = a0 + tid;
    const bool valid = a < A.n;

    if (warp == 0) tmem_alloc(&S.tmem, kTmemCols);
    if (tid == 0) {
        mbar_init(&S.mbar, 1);
        S.fail = 0;
    }
    // operands
    {
        float x[kInPad];
        anchor_input(A, a, valid, x);
#pragma unroll
        for (int k = 0; k < kInPad; ++k) S.X[canon(tid, k, kInPad)] = __float2bfloat16_rn(x[k]);
    }
    copy16<kFwdThreads>(S.W1, A.w1b, kHid * kInPad * 2, tid);
    copy16<kFwdThreads>(S.W2, A.w2b, kOutPad * kHid * 2, tid);
    if (tid < kHid) S.b1[tid] = A.b1[tid];
    for (int i = tid; i < kOutPad; i += kFwdThreads) S.b2[i] = i < kOut ? A.b2[i] : 0.0f;
    for (int j = 0; j < 3; ++j) S.xyz[tid][j] = valid ? A.xyz[3 * a + j] : 0.0f;
    for (int j = 0; j < 6; ++j) S.ls[tid][j] = valid ? A.ls[6 * a + j] : 0.0f;
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;

    // GEMM 1: D[0:32) = X W1^T
    if (tid == 0) {
#pragma unroll
        for (int kk = 0; kk < kInPad / 16; ++kk)
            mma_bf16(tmem, smem_desc(S.X + kk * 128, 128, kInPad * 16), smem_desc(S.W1 + kk * 128, 128, kInPad * 16),
                     idesc_bf16(kTileA, kHid), kk > 0);
        mma_commit(&S.mbar);
    }
    if (!mbar_wait(&S.mbar, 0)) S.fail = 1;
    tc_fence_after();
    __syncthreads();
    if (S.fail) goto cleanup;
    {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
        uint32_t pk[kHid / 2];
#pragma unroll
        for (int c = 0; c < kHid; c += 2) {
            pk[c / 2] = pack_bf16x2(fmaxf(v[c] + S.b1[c], 0.0f), fmaxf(v[c + 1] + S.b1[c + 1], 0.0f));
            // canonical layout: columns c, c + 1 are adjacent (c even)
            *reinterpret_cast<uint32_t *>(&S.H[canon(tid, c, kHid)]) = pk[c / 2];
        }
        if (valid) {
            uint4 *dst = reinterpret_cast<uint4 *>(A.h_store + a * kHid);
#pragma unroll
            for (int q = 0; q < kHid / 8; ++q)
                dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    // GEMM 2: D[32:176) = H W2^T
    if (tid == 0) {
#pragma unroll
        for (int kk = 0; kk < kHid / 16; ++kk)
            mma_bf16(tmem + 32, smem_desc(S.H + kk * 128, 128, kHid * 16), smem_desc(S.W2 + kk * 128, 128, kHid * 16),
                     idesc_bf16(kTileA, kOutPad), kk > 0);
        mma_commit(&S.mbar);
    }
    if (!mbar_wait(&S.mbar, 1)) S.fail = 1;
    tc_fence_after();
    __syncthreads();
    if (S.fail) goto cleanup;
    {
        const uint32_t row = tmem + ((uint32_t)(warp * 32) << 16) + 32;
        float v[32];
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            tmem_ld32(row + ch * 32, v);
#pragma unroll
            for (int c = 0; c < 32; ++c) S.Y[tid][ch * 32 + c] = v[c] + S.b2[ch * 32 + c];
        }
        tmem_ld16(row + 128, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) S.Y[tid][128 + c] = v[c] + S.b2[128 + c];
    }
    __syncthreads();
    {
        // children of the tile, written array by array so consecutive threads
        // store consecutive floats
        const int na = (int)min((int64_t)kTileA, A.n - a0);
        const int nch = na * kChild;
        const int64_t c0 = a0 * kChild;
        if (!kPre) {
            for (int i = tid; i < nch * 3; i += kFwdThreads) {
                const int ch = i / 3, j = i - 3 * ch, r = ch / kChild, c = ch - r * kChild;
                const float u = S.Y[r][c * kPer + j];
                A.c_means[3 * c0 + i] = S.xyz[r][j] + tanhf(u) * expf(S.ls[r][j]);
                A.c_ls[3 * c0 + i] = S.ls[r][3 + j] + log_sigmoidf(S.Y[r][c * kPer + 7 + j]);
                A.c_sh[3 * c0 + i] = (sigmoidf_(S.Y[r][c * kPer + 4 + j]) - 0.5f) * kDcScale;
            }
            for (int i = tid; i < nch * 4; i += kFwdThreads) {
                const int ch = i >> 2, j = i & 3, r = ch / kChild, c = ch - r * kChild;
                A.c_quats[4 * c0 + i] = S.Y[r][c * kPer + 10 + j];
            }
            for (int ch = tid; ch < nch; ch += kFwdThreads) {
                const int r = ch / kChild, c = ch - r * kChild;
                const float o = tanhf(S.Y[r][c * kPer + 3]);
                const float oc = fminf(o, kOpacityCeil);
                A.c_logits[c0 + ch] = o > 0.0f ? logf(oc) - log1pf(-oc) : kLogitFloor;
            }
        } else {
            // child by child: the same parameters (same expressions), written
            // for the backward and preprocessed straight from registers
            for (int ch = tid; ch < nch; ch += kFwdThreads) {
                const int r = ch / kChild, c = ch - r * kChild;
                const float *u = S.Y[r] + c * kPer;
                const int64_t gi = c0 + ch;
                float m[3], ls[3], sh[3];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    m[j] = S.xyz[r][j] + tanhf(u[j]) * expf(S.ls[r][j]);
                    ls[j] = S.ls[r][3 + j] + log_sigmoidf(u[7 + j]);
                    sh[j] = (sigmoidf_(u[4 + j]) - 0.5f) * kDcScale;
                    A.c_means[3 * gi + j] = m[j];
                    A.c_ls[3 * gi + j] = ls[j];
                    A.c_sh[3 * gi + j] = sh[j];
                }
                const float4 q = make_float4(u[10], u[11], u[12], u[13]);
                A.c_quats[4 * gi] = q.x;
                A.c_quats[4 * gi + 1] = q.y;
                A.c_quats[4 * gi + 2] = q.z;
                A.c_quats[4 * gi + 3] = q.w;
                const float o = tanhf(u[3]);
                const float oc = fminf(o, kOpacityCeil);
                const float logit = o > 0.0f ? logf(oc) - log1pf(-oc) : kLogitFloor;
                A.c_logits[gi] = logit;
                preprocess_item<0>(A.view, gi, make_float3(m[0], m[1], m[2]), q, make_float3(ls[0], ls[1], ls[2]), logit,
                                   sh, A.rec, A.bin, A.touched, A.rects, A.dkey, A.dval, A.box3);
            }
        }
    }
cleanup:
    if (S.fail) {
        // give the tensor cores one more bounded wait before the memory goes
        if (tid == 0) atomicCAS(A.err, 0, GS_ERR_TIMEOUT);
        mbar_wait(&S.mbar, 0);
        mbar_wait(&S.mbar, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// --------------------------------------------------------------- backward
// Per CTA of 128 anchors, every contraction on the tensor cores:
//   y  = H W2^T          (recompute, M = 128 anchors, N = 144, K = 32)
//   dh = dY W2           (M = 128 anchors, N = 32, K = 144)
//   dW2 = dY^T H         (outputs 0..127 and 128..143 as two M = 128 tiles,
//                         N = 32, K = 128 anchors)
//   dx = dH W1           (M = 128 anchors, N = 48, K = 32)
//   dW1^T = x^T dH       (M = 128 input rows of which 48 exist, N = 32,
//                         K = 128 anchors)
// An M = 128 operand with fewer real rows (dW2's last 16 outputs, dW1's 48
// inputs) is followed in shared memory by other operand buffers: the MMA reads
// them as its remaining rows, whose results land in TMEM lanes nobody reads.
// TMEM columns: y 0..143, then dh 0..31, dx 32..79, dW2 128..159 and
// 160..191, dW1^T 192..223.
// Three threads per anchor (warps w, w + 4 and w + 8 read the same TMEM
// lanes): the per-child work, the operand packing and the TMEM read-backs
// are split between the three thirds of the CTA.
struct BwdSmem {
    __nv_bfloat16 W2T[kHid * kOutPad];   // dh B (N = 32, K = 144)
    __nv_bfloat16 W1T[kInPad * kHid];    // dx B (N = 48, K = 32)
    // DY, DYT2 and DYT first hold the tile's children's gradients (copied
    // in while y is recomputed); the A operands with fewer than 128 rows
    // (DYT2, XT) read their missing rows from the buffers after them
    __nv_bfloat16 DY[kTileA * kOutPad];  // dh A (M = 128 anchors, K = 144)
    __nv_bfloat16 DYT2[16 * kTileA];     // dW2 A, outputs 128..143 (+112 rows read past the end)
    __nv_bfloat16 DYT[kTileA * kTileA];  // dW2 A, outputs 0..127
    __nv_bfloat16 XT[kInPad * kTileA];   // dW1^T A, inputs 0..47 (+80 rows read past the end)
    __nv_bfloat16 HT[kHid * kTileA];     // dW2 B (N = 32 hidden, K = 128 anchors)
    union {
        struct {
            __nv_bfloat16 H[kTileA * kHid];    // y A (M = 128, K = 32)
            __nv_bfloat16 W2[kOutPad * kHid];  // y B (N = 144, K = 32)
        } p1;
        struct {
            __nv_bfloat16 DH[kTileA * kHid];   // dx A (M = 128, K = 32)
            __nv_bfloat16 DHT[kHid * kTileA];  // dW1^T B (N = 32 hidden, K = 128 anchors)
        } p2;
    } u;
    float Y[kTileA][kOutPad + 1];  // y, then dL/dy (fp32)
    float xyz[kTileA][3], ls[kTileA][6], dls[3][kTileA][6];  // dls: per third of the children
    float db1w[kTileA / 32][kHid];    // per-warp sums of db1
    float b2[kOutPad];
    uint64_t mbar, gbar;  // MMA completion; children's gradients copied in
    uint32_t tmem;
    int fail;
};

// staged children's gradients (floats from the start of DY): means, SH DC,
// log-scales (3 per child), quaternions (4), opacity logits (1)
constexpr int kStM = 0, kStS = kTileA * kChild * 3, kStL = 2 * kStS, kStQ = 3 * kStS;
constexpr int kStO = kStQ + kTileA * kChild * 4, kStEnd = kStO + kTileA * kChild;
static_assert(offsetof(BwdSmem, DY) + 4 * kStEnd <= offsetof(BwdSmem, XT), "children's gradients fit the staging");
static_assert(offsetof(BwdSmem, DYT2) + 2 * kTileA * kTileA <= sizeof(BwdSmem), "dW2 tail operand rows");
static_assert(offsetof(BwdSmem, XT) + 2 * kTileA * kTileA <= sizeof(BwdSmem), "dW1 operand rows");
static_assert(sizeof(BwdSmem) + 1024 <= 227 * 1024, "one backward CTA fits the shared memory of an SM");

__device__ __forceinline__ float bf16f(__nv_bfloat16 v) { return __bfloat162float(v); }

__global__ void __launch_bounds__(kThreads) k_ng_bwd(Args A) {
    extern __shared__ uint8_t smem_raw[];
    BwdSmem &S = *reinterpret_cast<BwdSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // anchor row of the tile (= TMEM lane) and which third of its work this
    // thread does; warps w, w + 4 and w + 8 share TMEM lanes 32 (w mod 4) ..
    const int r = tid & (kTileA - 1), grp = tid >> 7;
    const int64_t a0 = (int64_t)blockIdx.x * kTileA;
    const int64_t a = a0 + r;
    const bool valid = a < A.n;
    const int na = (int)min((int64_t)kTileA, A.n - a0);
    float *part = A.partial + (size_t)blockIdx.x * kPartial;

    if (warp == 0) tmem_alloc(&S.tmem, kTmemCols);
    // the tile's children's gradients into shared memory: five bulk copies
    // that run while the operands load and y is recomputed (a partial last
    // tile or unaligned arrays take plain loads instead)
    float *stg = reinterpret_cast<float *>(S.DY);
    const int nch = na * kChild;
    const int64_t c0 = a0 * kChild;
    const bool bulk = A.grads_bulk && na == kTileA;
    if (tid == 0) {
        mbar_init(&S.mbar, 1);
        mbar_init(&S.gbar, 1);
        S.fail = 0;
        if (bulk) {
            constexpr uint32_t b3 = kTileA * kChild * 3 * 4, b4 = kTileA * kChild * 4 * 4, b1 = kTileA * kChild * 4;
            mbar_expect_tx(&S.gbar, 3 * b3 + b4 + b1);
            bulk_g2s(stg + kStM, A.g_means + 3 * c0, b3, &S.gbar);
            bulk_g2s(stg + kStS, A.g_sh + 3 * c0, b3, &S.gbar);
            bulk_g2s(stg + kStL, A.g_ls + 3 * c0, b3, &S.gbar);
            bulk_g2s(stg + kStQ, A.g_quats + 4 * c0, b4, &S.gbar);
            bulk_g2s(stg + kStO, A.g_logits + c0, b1, &S.gbar);
        }
    }
    if (!bulk) {
        for (int i = tid; i < nch * 3; i += kThreads) {
            stg[kStM + i] = A.g_means[3 * c0 + i];
            stg[kStS + i] = A.g_sh[3 * c0 + i];
            stg[kStL + i] = A.g_ls[3 * c0 + i];
        }
        for (int i = tid; i < nch * 4; i += kThreads) stg[kStQ + i] = A.g_quats[4 * c0 + i];
        for (int i = tid; i < nch; i += kThreads) stg[kStO + i] = A.g_logits[c0 + i];
    }
    if (grp == 0) {
        // h of this anchor into the y GEMM's A (row = anchor) and the dW2
        // GEMM's B (row = hidden unit, K = anchors)
        const uint4 *src = reinterpret_cast<const uint4 *>(A.h_store + a * kHid);
#pragma unroll
        for (int q = 0; q < kHid / 8; ++q) {
            const uint4 w = valid ? src[q] : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 8 * q + 2 * e;
                *reinterpret_cast<uint32_t *>(&S.u.p1.H[canon(r, c, kHid)]) = u[e];
                S.HT[canon(c, r, kTileA)] = __ushort_as_bfloat16((unsigned short)(u[e] & 0xffffu));
                S.HT[canon(c + 1, r, kTileA)] = __ushort_as_bfloat16((unsigned short)(u[e] >> 16));
            }
        }
        for (int j = 0; j < 3; ++j) S.xyz[r][j] = valid ? A.xyz[3 * a + j] : 0.0f;
        for (int j = 0; j < 6; ++j) S.ls[r][j] = valid ? A.ls[6 * a + j] : 0.0f;
    } else if (grp == 1) {
        // x of this anchor as the dW1^T GEMM's A (row = input, K = anchors)
        float x[kInPad];
        anchor_input(A, a, valid, x);
#pragma unroll
        for (int k = 0; k < kInPad; ++k) S.XT[canon(k, r, kTileA)] = __float2bfloat16_rn(x[k]);
    }
    copy16(S.u.p1.W2, A.w2b, kOutPad * kHid * 2, tid);
    copy16(S.W2T, A.w2tb, kHid * kOutPad * 2, tid);
    copy16(S.W1T, A.w1tb, kInPad * kHid * 2, tid);
    for (int i = tid; i < kOutPad; i += kThreads) S.b2[i] = i < kOut ? A.b2[i] : 0.0f;
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t my_lanes = tmem + ((uint32_t)((warp & 3) * 32) << 16);

    // y = W2 h + b2, recomputed exactly as in the forward
    if (tid == 0) {
#pragma unroll
        for (int kk = 0; kk < kHid / 16; ++kk)
            mma_bf16(tmem, smem_desc(S.u.p1.H + kk * 128, 128, kHid * 16),
                     smem_desc(S.u.p1.W2 + kk * 128, 128, kHid * 16), idesc_bf16(kTileA, kOutPad), kk > 0);
        mma_commit(&S.mbar);
    }
    if (!mbar_wait(&S.mbar, 0)) S.fail = 1;
    tc_fence_after();
    __syncthreads();
    if (S.fail) goto cleanup;
    {
        // columns 0..63 by the first third, 64..127 by the second, 128..143
        // by the last
        float v[32];
        if (grp < 2) {
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int ch = 2 * grp + cc;
                tmem_ld32(my_lanes + ch * 32, v);
#pragma unroll
                for (int c = 0; c < 32; ++c) S.Y[r][ch * 32 + c] = v[c] + S.b2[ch * 32 + c];
            }
        } else {
            tmem_ld16(my_lanes + 128, v);
#pragma unroll
            for (int c = 0; c < 16; ++c) S.Y[r][128 + c] = v[c] + S.b2[128 + c];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (bulk && !mbar_wait(&S.gbar, 0)) S.fail = 1;
    __syncthreads();
    if (S.fail) goto cleanup;
    if (A.zero_g) {
        // the children's gradients are consumed: clear them (coalesced)
        if (bulk) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = tid; i < nch * 3 / 4; i += kThreads) {
                reinterpret_cast<float4 *>(A.g_means + 3 * c0)[i] = z;
                reinterpret_cast<float4 *>(A.g_sh + 3 * c0)[i] = z;
                reinterpret_cast<float4 *>(A.g_ls + 3 * c0)[i] = z;
            }
            for (int i = tid; i < nch; i += kThreads) reinterpret_cast<float4 *>(A.g_quats + 4 * c0)[i] = z;
            for (int i = tid; i < nch / 4; i += kThreads) reinterpret_cast<float4 *>(A.g_logits + c0)[i] = z;
        } else {
            for (int i = tid; i < nch * 3; i += kThreads) {
                A.g_means[3 * c0 + i] = 0.0f;
                A.g_sh[3 * c0 + i] = 0.0f;
                A.g_ls[3 * c0 + i] = 0.0f;
            }
            for (int i = tid; i < nch * 4; i += kThreads) A.g_quats[4 * c0 + i] = 0.0f;
            for (int i = tid; i < nch; i += kThreads) A.g_logits[c0 + i] = 0.0f;
        }
    }
    if (r < na) {
        // dL/dy of a third of this anchor's children (4, 3, 3) in place of y
        // (every element depends on its own y only), and that third's share
        // of the anchor's log-scale gradients, children in order
        float *yr = S.Y[r];
        float so[3], dl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; ++j) so[j] = expf(S.ls[r][j]);
#pragma unroll 1
        const int cb = grp == 0 ? 0 : (grp == 1 ? 4 : 7), ce = grp == 0 ? 4 : (grp == 1 ? 7 : kChild);
        for (int c = cb; c < ce; ++c) {
            const int ch = r * kChild + c;
            float *u = yr + c * kPer;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float gm = stg[kStM + 3 * ch + j], gs = stg[kStS + 3 * ch + j], gl = stg[kStL + 3 * ch + j];
                const float th = tanhf(u[j]);
                dl[j] += gm * th * so[j];
                u[j] = gm * so[j] * (1.0f - th * th);
                const float rgb = sigmoidf_(u[4 + j]);
                u[4 + j] = gs * kDcScale * rgb * (1.0f - rgb);
                dl[3 + j] += gl;
                u[7 + j] = gl * sigmoidf_(-u[7 + j]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) u[10 + j] = stg[kStQ + 4 * ch + j];
            const float o = tanhf(u[3]);
            const float oc = fminf(o, kOpacityCeil);
            u[3] = (o > 0.0f && o < kOpacityCeil) ? stg[kStO + ch] / (oc * (1.0f - oc)) * (1.0f - o * o) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) S.dls[grp][r][k] = dl[k];
    }
    __syncthreads();
    // db2 (unrounded dy of the present anchors)
    for (int o = tid; o < kOut; o += kThreads) {
        // four interleaved running sums (independent loads in flight), then
        // combined in a fixed order
        float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int rr = 0; rr < na; ++rr) s4[rr & 3] += S.Y[rr][o];
        part[kOut * kHid + kHid * kIn + o] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    }
    __syncthreads();
    {
        // this anchor's rounded dy (zero for an absent anchor and the padding
        // outputs) as its row of the dh GEMM's A and its column (K index) of
        // the dW2 GEMMs' A operands
        const bool live = r < na;
        constexpr int kPartOut = kOutPad / 3;  // outputs per third (even)
        static_assert(kPartOut % 2 == 0 && 3 * kPartOut == kOutPad, "outputs split in thirds of pairs");
#pragma unroll 4
        for (int o = grp * kPartOut; o < (grp + 1) * kPartOut; o += 2) {
            const float v0 = live && o < kOut ? S.Y[r][o] : 0.0f;
            const float v1 = live && o + 1 < kOut ? S.Y[r][o + 1] : 0.0f;
            const uint32_t pk = pack_bf16x2(v0, v1);
            *reinterpret_cast<uint32_t *>(&S.DY[canon(r, o, kOutPad)]) = pk;
            const __nv_bfloat16 b0 = __ushort_as_bfloat16((unsigned short)(pk & 0xffffu));
            const __nv_bfloat16 b1 = __ushort_as_bfloat16((unsigned short)(pk >> 16));
            if (o < kTileA) {
                S.DYT[canon(o, r, kTileA)] = b0;
                S.DYT[canon(o + 1, r, kTileA)] = b1;
            } else {
                S.DYT2[canon(o - kTileA, r, kTileA)] = b0;
                S.DYT2[canon(o + 1 - kTileA, r, kTileA)] = b1;
            }
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // dh = dy W2 (contraction over the 144 outputs), dW2 = dy^T h (over the
    // 128 anchors) for outputs 0..127 and 128..143
    if (tid == 0) {
#pragma unroll
        for (int kk = 0; kk < kOutPad / 16; ++kk)
            mma_bf16(tmem, smem_desc(S.DY + kk * 128, 128, kOutPad * 16), smem_desc(S.W2T + kk * 128, 128, kOutPad * 16),
                     idesc_bf16(kTileA, kHid), kk > 0);
#pragma unroll
        for (int kk = 0; kk < kTileA / 16; ++kk) {
            const uint64_t hb = smem_desc(S.HT + kk * 128, 128, kTileA * 16);
            mma_bf16(tmem + 128, smem_desc(S.DYT + kk * 128, 128, kTileA * 16), hb, idesc_bf16(kTileA, kHid), kk > 0);
            mma_bf16(tmem + 160, smem_desc(S.DYT2 + kk * 128, 128, kTileA * 16), hb, idesc_bf16(kTileA, kHid), kk > 0);
        }
        mma_commit(&S.mbar);
    }
    if (!mbar_wait(&S.mbar, 1)) S.fail = 1;
    tc_fence_after();
    __syncthreads();
    if (S.fail) goto cleanup;
    if (grp == 0) {
        // dh after the ReLU mask, rounded, as the dx GEMM's A (row = anchor)
        // and the dW1^T GEMM's B (row = hidden unit, K = anchors); the
        // y-recompute operands it overwrites are no longer read
        float v[32];
        tmem_ld32(my_lanes, v);
#pragma unroll
        for (int c = 0; c < kHid; c += 2) {
            const float d0 = bf16f(S.HT[canon(c, r, kTileA)]) > 0.0f ? v[c] : 0.0f;
            const float d1 = bf16f(S.HT[canon(c + 1, r, kTileA)]) > 0.0f ? v[c + 1] : 0.0f;
            const float w0 = warp_sum(d0), w1 = warp_sum(d1);
            if (lane == 0) {
                S.db1w[warp][c] = w0;
                S.db1w[warp][c + 1] = w1;
            }
            const uint32_t pk = pack_bf16x2(d0, d1);
            *reinterpret_cast<uint32_t *>(&S.u.p2.DH[canon(r, c, kHid)]) = pk;
            S.u.p2.DHT[canon(c, r, kTileA)] = __ushort_as_bfloat16((unsigned short)(pk & 0xffffu));
            S.u.p2.DHT[canon(c + 1, r, kTileA)] = __ushort_as_bfloat16((unsigned short)(pk >> 16));
        }
    } else if (grp == 1) {
        // this thread's row (output r) of dW2
        float v[32];
        tmem_ld32(my_lanes + 128, v);
        float4 *dst = reinterpret_cast<float4 *>(part + r * kHid);
#pragma unroll
        for (int q = 0; q < kHid / 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
        float v[32];
        if (warp == 8) {  // outputs 128..139
            tmem_ld32(my_lanes + 160, v);
            if (lane < kOut - kTileA) {
                float4 *d2 = reinterpret_cast<float4 *>(part + (kTileA + lane) * kHid);
#pragma unroll
                for (int q = 0; q < kHid / 4; ++q)
                    d2[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // dx = dh W1 (over the 32 hidden units); dW1^T = x^T dh (over the anchors)
    if (tid == 0) {
#pragma unroll
        for (int kk = 0; kk < kHid / 16; ++kk)
            mma_bf16(tmem + 32, smem_desc(S.u.p2.DH + kk * 128, 128, kHid * 16),
                     smem_desc(S.W1T + kk * 128, 128, kHid * 16), idesc_bf16(kTileA, kInPad), kk > 0);
#pragma unroll
        for (int kk = 0; kk < kTileA / 16; ++kk)
            mma_bf16(tmem + 192, smem_desc(S.XT + kk * 128, 128, kTileA * 16),
                     smem_desc(S.u.p2.DHT + kk * 128, 128, kTileA * 16), idesc_bf16(kTileA, kHid), kk > 0);
        mma_commit(&S.mbar);
    }
    if (tid < kHid) {  // db1, warps in order
        float sum = 0.0f;
#pragma unroll
        for (int w = 0; w < kTileA / 32; ++w) sum += S.db1w[w][tid];
        part[kOut * kHid + kHid * kIn + kOut + tid] = sum;
    }
    if (!mbar_wait(&S.mbar, 0)) S.fail = 1;
    tc_fence_after();
    __syncthreads();
    if (S.fail) goto cleanup;
    if (grp == 0) {
        float v[32];
        tmem_ld32(my_lanes + 32, v);
        if (valid) {
            if (A.feat_vec) {
                float4 *df = reinterpret_cast<float4 *>(A.d_feat + a * kFeat);
#pragma unroll
                for (int q = 0; q < kFeat / 4; ++q) {
                    float4 d = df[q];
                    d.x += v[4 * q];
                    d.y += v[4 * q + 1];
                    d.z += v[4 * q + 2];
                    d.w += v[4 * q + 3];
                    df[q] = d;
                }
            } else {
#pragma unroll
                for (int c = 0; c < kFeat; ++c) A.d_feat[a * kFeat + c] += v[c];
            }
#pragma unroll
            for (int j = 0; j < 6; ++j) A.d_ls[6 * a + j] += S.dls[0][r][j] + S.dls[1][r][j] + S.dls[2][r][j];
        }
    } else if (warp < 6) {  // dW1[h][i] = (dW1^T)[i][h] for the 35 inputs (TMEM lanes 0..63)
        float v[32];
        tmem_ld32(my_lanes + 192, v);
        if (r < kIn)
#pragma unroll
            for (int h = 0; h < kHid; ++h) part[kOut * kHid + h * kIn + r] = v[h];
    }
cleanup:
    if (S.fail) {
        // give the tensor cores and the copies one more bounded wait before
        // the memory goes
        if (tid == 0) atomicCAS(A.err, 0, GS_ERR_TIMEOUT);
        mbar_wait(&S.mbar, 0);
        mbar_wait(&S.mbar, 1);
        if (bulk) mbar_wait(&S.gbar, 0);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// Sum of the per-CTA partials, added to the grads.  A block owns 32
// consecutive partial entries (a warp reads them as one 128-byte row); its 32
// warps take the CTAs t = warp, warp + 32, ... (four running sums each, for
// independent loads in flight), then one warp adds the 32 warp sums in warp
// order.  The order is fixed, so the result is deterministic.
constexpr int kRedCols = 32, kRedRows = 32;
__global__ void __launch_bounds__(kRedCols * kRedRows) k_ng_reduce(const float *__restrict__ partial, int n_tiles,
                                                                   float *dw2, float *dw1, float *db2, float *db1) {
    __shared__ float red[kRedRows][kRedCols + 1];
    const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int i = blockIdx.x * kRedCols + c;
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (i < kPartial) {
        int t = g;
        for (; t + 3 * kRedRows < n_tiles; t += 4 * kRedRows)
#pragma unroll
            for (int u = 0; u < 4; ++u) s[u] += partial[(size_t)(t + u * kRedRows) * kPartial + i];
        for (int u = 0; t < n_tiles; t += kRedRows, ++u) s[u & 3] += partial[(size_t)t * kPartial + i];
    }
    red[g][c] = (s[0] + s[1]) + (s[2] + s[3]);
    __syncthreads();
    if (g != 0 || i >= kPartial) return;
    float tot = 0.0f;
    for (int r = 0; r < kRedRows; ++r) tot += red[r][c];
    if (i < kOut * kHid) dw2[i] += tot;
    else if (i < kOut * kHid + kHid * kIn) dw1[i - kOut * kHid] += tot;
    else if (i < kOut * kHid + kHid * kIn + kOut) db2[i - kOut * kHid - kHid * kIn] += tot;
    else db1[i - kOut * kHid - kHid * kIn - kOut] += tot;
}

// ---------------------------------------------------------------- workspace
struct Layout {
    size_t w1b, w2b, w2tb, w1tb, h, partial, err, bytes;
};

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

static Layout layout(int64_t n) {
    Layout L;
    size_t o = 0;
    const int64_t tiles = (n + kTileA - 1) / kTileA;
    L.err = o;
    o = al(o + 256);
    L.w1b = o;
    o = al(o + kHid * kInPad * 2);
    L.w2b = o;
    o = al(o + kOutPad * kHid * 2);
    L.w2tb = o;
    o = al(o + kHid * kOutPad * 2);
    L.w1tb = o;
    o = al(o + kInPad * kHid * 2);
    L.h = o;
    o = al(o + (size_t)n * kHid * 2);
    L.partial = o;
    o = al(o + (size_t)tiles * kPartial * 4);
    L.bytes = o;
    return L;
}

static int check_ng(const gs_ng_params *p) {
    if (!p || p->n_anchors <= 0 || p->n_anchors * (int64_t)kChild >= (1ll << 31) || !p->anchor_xyz || !p->feat ||
        !p->anchor_ls || !p->w1 || !p->b1 || !p->w2 || !p->b2)
        return GS_ERR_ARG;
    return GS_OK;
}

// Raise a kernel's dynamic shared-memory limit once per device (the
// attribute is per device context); `done` is the caller's per-kernel table.
static int smem_opt_in(const void *kernel, size_t bytes, bool *done) {
    int dev = 0;
    int rc = check_cuda(cudaGetDevice(&dev));
    if (rc) return rc;
    const bool cache = dev >= 0 && dev < 64;
    if (cache && done[dev]) return GS_OK;
    rc = check_cuda(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (rc == GS_OK && cache) done[dev] = true;
    return rc;
}

static Args base_args(const gs_ng_params *p, const gs_camera *cam, void *ws) {
    const Layout L = layout(p->n_anchors);
    Args A{};
    A.n = p->n_anchors;
    A.xyz = p->anchor_xyz;
    A.feat = p->feat;
    A.feat_vec = ((uintptr_t)p->feat & 15) == 0;
    A.ls = p->anchor_ls;
    A.b1 = p->b1;
    A.b2 = p->b2;
    // camera centre = -R^T t
    for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int i = 0; i < 3; ++i) s -= (double)cam->w2c[i * 4 + j] * (double)cam->w2c[i * 4 + 3];
        A.cam[j] = (float)s;
    }
    char *w = (char *)ws;
    A.w1b = (const __nv_bfloat16 *)(w + L.w1b);
    A.w2b = (const __nv_bfloat16 *)(w + L.w2b);
    A.w2tb = (const __nv_bfloat16 *)(w + L.w2tb);
    A.w1tb = (const __nv_bfloat16 *)(w + L.w1tb);
    A.h_store = (__nv_bfloat16 *)(w + L.h);
    A.partial = (float *)(w + L.partial);
    A.err = (int *)(w + L.err);
    return A;
}

}  // namespace ng
}  // namespace gs

using namespace gs;

extern "C" size_t gs_ng_workspace_bytes(int64_t n_anchors) {
    return n_anchors > 0 ? ng::layout(n_anchors).bytes : 0;
}

extern "C" int gs_ng_decode_fwd(const gs_ng_params *p, const gs_camera *cam, gs_params *children, void *ws,
                                void *stream) {
    int rc = ng::check_ng(p);
    if (rc) return rc;
    if (!cam || !ws || !children || children->n != p->n_anchors * ng::kChild || children->sh_degree != 0 ||
        !children->means || !children->log_scales || !children->quats || !children->opacity_logits || !children->sh)
        return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = sizeof(ng::FwdSmem) + 1024;
    static bool opted[64] = {};
    rc = ng::smem_opt_in((const void *)ng::k_ng_fwd<false>, smem, opted);
    if (rc) return rc;
    ng::Args A = ng::base_args(p, cam, ws);
    char *w = (char *)ws;
    const ng::Layout L = ng::layout(p->n_anchors);
    ng::k_ng_prep<<<1, 256, 0, s>>>(p->w1, p->w2, (__nv_bfloat16 *)(w + L.w1b), (__nv_bfloat16 *)(w + L.w2b),
                                    (__nv_bfloat16 *)(w + L.w2tb), (__nv_bfloat16 *)(w + L.w1tb));
    A.c_means = children->means;
    A.c_ls = children->log_scales;
    A.c_quats = children->quats;
    A.c_logits = children->opacity_logits;
    A.c_sh = children->sh;
    const unsigned tiles = (unsigned)((p->n_anchors + ng::kTileA - 1) / ng::kTileA);
    ng::k_ng_fwd<false><<<tiles, ng::kFwdThreads, smem, s>>>(A);
    return launch_error();
}

extern "C" int gs_ng_decode_preprocess(const gs_ng_params *p, const gs_camera *cam, gs_params *children, void *ws,
                                       const gs_plan *plan, void *plan_ws, void *stream) {
    int rc = ng::check_ng(p);
    if (rc) return rc;
    if (!cam || !ws || !children || children->n != p->n_anchors * ng::kChild || children->sh_degree != 0 ||
        !children->means || !children->log_scales || !children->quats || !children->opacity_logits || !children->sh ||
        !plan || !plan_ws || plan->V != 1 || plan->n != children->n || plan->sh_degree != 0 || plan->pose)
        return GS_ERR_ARG;
    rc = check_cams(plan, cam);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = sizeof(ng::FwdSmem) + 1024;
    static bool opted[64] = {};
    rc = ng::smem_opt_in((const void *)ng::k_ng_fwd<true>, smem, opted);
    if (rc) return rc;
    ng::Args A = ng::base_args(p, cam, ws);
    char *w = (char *)ws;
    const ng::Layout L = ng::layout(p->n_anchors);
    ng::k_ng_prep<<<1, 256, 0, s>>>(p->w1, p->w2, (__nv_bfloat16 *)(w + L.w1b), (__nv_bfloat16 *)(w + L.w2b),
                                    (__nv_bfloat16 *)(w + L.w2tb), (__nv_bfloat16 *)(w + L.w1tb));
    A.c_means = children->means;
    A.c_ls = children->log_scales;
    A.c_quats = children->quats;
    A.c_logits = children->opacity_logits;
    A.c_sh = children->sh;
    A.view = make_views(plan, cam).v[0];
    A.rec = ws_at<float4>(plan_ws, plan->o_rec);
    A.bin = ws_at<float2>(plan_ws, plan->o_bin);
    A.touched = ws_at<uint32_t>(plan_ws, plan->o_touched);
    A.rects = ws_at<uint2>(plan_ws, plan->o_rect);
    A.dkey = ws_at<uint32_t>(plan_ws, plan->o_dkey[0]);
    A.dval = ws_at<uint32_t>(plan_ws, plan->o_dval[0]);
    A.box3 = plan->bbox_3sigma;
    const unsigned tiles = (unsigned)((p->n_anchors + ng::kTileA - 1) / ng::kTileA);
    ng::k_ng_fwd<true><<<tiles, ng::kFwdThreads, smem, s>>>(A);
    return launch_error();
}

extern "C" int gs_ng_decode_bwd(const gs_ng_params *p, const gs_camera *cam, const gs_params *child_grads,
                                int32_t zero_child_grads, gs_ng_params *grads, void *ws, void *stream) {
    int rc = ng::check_ng(p);
    if (rc) return rc;
    if (!cam || !ws || !child_grads || !grads || child_grads->n != p->n_anchors * ng::kChild ||
        child_grads->sh_degree != 0 || !child_grads->means || !child_grads->log_scales || !child_grads->quats ||
        !child_grads->opacity_logits || !child_grads->sh || !grads->feat || !grads->anchor_ls || !grads->w1 ||
        !grads->b1 || !grads->w2 || !grads->b2)
        return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = sizeof(ng::BwdSmem) + 1024;
    static bool opted[64] = {};
    rc = ng::smem_opt_in((const void *)ng::k_ng_bwd, smem, opted);
    if (rc) return rc;
    ng::Args A = ng::base_args(p, cam, ws);
    A.g_means = child_grads->means;
    A.g_ls = child_grads->log_scales;
    A.g_quats = child_grads->quats;
    A.g_logits = child_grads->opacity_logits;
    A.g_sh = child_grads->sh;
    A.zero_g = zero_child_grads != 0;
    A.grads_bulk = ((((uintptr_t)A.g_means) | ((uintptr_t)A.g_ls) | ((uintptr_t)A.g_quats) |
                     ((uintptr_t)A.g_logits) | ((uintptr_t)A.g_sh)) & 15) == 0;
    A.d_feat = grads->feat;
    A.feat_vec = A.feat_vec && ((uintptr_t)grads->feat & 15) == 0;
    A.d_ls = grads->anchor_ls;
    const int tiles = (int)((p->n_anchors + ng::kTileA - 1) / ng::kTileA);
    ng::k_ng_bwd<<<tiles, ng::kThreads, smem, s>>>(A);
    ng::k_ng_reduce<<<(ng::kPartial + ng::kRedCols - 1) / ng::kRedCols, ng::kRedCols * ng::kRedRows, 0, s>>>(
        A.partial, tiles, grads->w2, grads->w1, grads->b2, grads->b1);
    return launch_error();
}

namespace gs {
namespace ng {

// The bounded wait on its own: one thread initialises an mbarrier for one
// arrival and waits for its first phase.  With arrive = 0 nothing ever
// arrives (no thread, no copy, no MMA is in flight), so the wait must give
// up after `limit` tries and record GS_ERR_TIMEOUT; with arrive = 1 the
// thread arrives first and the wait must succeed.
__global__ void k_wait_probe(int32_t *err, long long limit, int arrive) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    if (arrive) {
        uint64_t state;
        asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(smem_u32(&bar)) : "memory");
        (void)state;
    }
    if (!mbar_wait(&bar, 0, limit)) atomicCAS(err, 0, GS_ERR_TIMEOUT);
}

}  // namespace ng
}  // namespace gs

extern "C" int gs_ng_wait_probe(int32_t *d_err, int64_t limit, int32_t arrive, void *stream) {
    if (!d_err || limit < 1 || limit > ng::kWaitLimit || (arrive != 0 && arrive != 1)) return GS_ERR_ARG;
    ng::k_wait_probe<<<1, 32, 0, (cudaStream_t)stream>>>(d_err, (long long)limit, arrive);
    return launch_error();
}

extern "C" int gs_ng_read_status(void *ws, int32_t *out_error, void *stream) {
    if (!ws || !out_error) return GS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int e = 0;
    int rc = check_cuda(cudaMemcpyAsync(&e, ws, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (rc) return rc;
    rc = check_cuda(cudaStreamSynchronize(s));
    if (rc) return rc;
    *out_error = e;
    return e ? e : GS_OK;
}
