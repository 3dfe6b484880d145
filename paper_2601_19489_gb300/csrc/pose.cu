// Global pose refinement (Sec. 2.5): one correction (Delta_R, Delta_t)
// shared by every camera, applied on the camera side, [W | t] ->
// [Delta_R W | Delta_R t + Delta_t]; its loss gradient is accumulated by the
// preprocess backward (preprocess.cu) and turned into an update here.
//
// State buffer (doubles): [0..8] Delta_R row-major, [9..11] Delta_t,
// [12..17] Adam m, [18..23] Adam v, [24] Adam step, [32 + 8 s + k] partial
// gradient sums, s < GS_POSE_SLOTS, k < 6 (omega, tau).
#include <math.h>

#include "gs_internal.cuh"

namespace gs {

constexpr int kPoseR = 0, kPoseT = 9, kPoseM = 12, kPoseV = 18, kPoseStep = 24, kPoseAcc = 32;

__global__ void k_pose_init(double *st) {
    for (int i = threadIdx.x; i < GS_POSE_STATE_DOUBLES; i += blockDim.x)
        st[i] = (i == kPoseR || i == kPoseR + 4 || i == kPoseR + 8) ? 1.0 : 0.0;
}

// One thread per view: the corrected transform in double precision, rounded
// once to float32; the camera centre -R^T t from the rounded values (as the
// host computes it for an uncorrected camera).
__global__ void k_pose_compose(ViewsDev views, const double *__restrict__ st, ViewDev *__restrict__ out) {
    const int v = threadIdx.x;
    if (v >= views.V) return;
    ViewDev d = views.v[v];
    double R[9], t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double a = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) a += st[kPoseR + 3 * i + k] * (double)d.R[3 * k + j];
            R[3 * i + j] = a;
        }
        double b = st[kPoseT + i];
#pragma unroll
        for (int k = 0; k < 3; ++k) b += st[kPoseR + 3 * i + k] * (double)d.t[k];
        t[i] = b;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) d.R[i] = (float)R[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) d.t[i] = (float)t[i];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double c = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) c -= (double)d.R[3 * i + j] * (double)d.t[i];
        d.campos[j] = (float)c;
    }
    out[v] = d;
}

// exp([w]_x) by Rodrigues' formula, I + a K + b K^2 with a = sin(th)/th and
// b = (1 - cos th)/th^2; below th = 1e-4 both from their Taylor series (to
// th^4), where the quotients would lose digits.
__device__ void so3_exp(const double w[3], double E[9]) {
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double a, b;
    if (th2 < 1e-8) {
        a = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        b = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    } else {
        const double th = sqrt(th2);
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
    }
    const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double k2 = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) k2 += K[3 * i + k] * K[3 * k + j];
            E[3 * i + j] = (i == j ? 1.0 : 0.0) + a * K[3 * i + j] + b * k2;
        }
}

// One block of GS_POSE_SLOTS threads: thread s takes slot s (and clears it);
// the block sums the slots; thread 0 runs Adam and folds the increment in.
__global__ void __launch_bounds__(GS_POSE_SLOTS) k_pose_step(double *st, gs_pose_hparams hp) {
    __shared__ double part[GS_POSE_SLOTS / 32][6];
    const int s = threadIdx.x, lane = s & 31, warp = s >> 5;
    double g[6];
    double *slot = st + kPoseAcc + 8 * s;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        g[k] = slot[k];
        slot[k] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) g[k] += __shfl_xor_sync(0xffffffffu, g[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) part[warp][k] = g[k];
    __syncthreads();
    if (s != 0) return;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        double a = 0.0;
        for (int w = 0; w < GS_POSE_SLOTS / 32; ++w) a += part[w][k];
        g[k] = a;
    }
    const double step = st[kPoseStep] + 1.0;
    st[kPoseStep] = step;
    const double bc1 = 1.0 - pow(hp.b1, step), bc2 = 1.0 - pow(hp.b2, step);
    double xi[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double m = hp.b1 * st[kPoseM + k] + (1.0 - hp.b1) * g[k];
        const double v = hp.b2 * st[kPoseV + k] + (1.0 - hp.b2) * g[k] * g[k];
        st[kPoseM + k] = m;
        st[kPoseV + k] = v;
        const double lr = k < 3 ? hp.lr_rot : hp.lr_trans;
        xi[k] = -lr * (m / bc1) / (sqrt(v / bc2) + hp.eps);
    }
    double E[9];
    so3_exp(xi, E);
    double R[9], t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double a = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) a += E[3 * i + k] * st[kPoseR + 3 * k + j];
            R[3 * i + j] = a;
        }
        double b = xi[3 + i];
#pragma unroll
        for (int k = 0; k < 3; ++k) b += E[3 * i + k] * st[kPoseT + k];
        t[i] = b;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) st[kPoseR + i] = R[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) st[kPoseT + i] = t[i];
}

int pose_compose(const gs_plan *plan, void *ws, const ViewsDev &vd, cudaStream_t s) {
    k_pose_compose<<<1, 32, 0, s>>>(vd, plan->pose, ws_at<ViewDev>(ws, plan->o_posed));
    return launch_error();
}

}  // namespace gs

using namespace gs;

static_assert(GS_MAX_VIEWS <= 32, "one compose thread per view");
static_assert(GS_POSE_SLOTS % 32 == 0 && GS_POSE_SLOTS <= 1024, "one step block, whole warps");

extern "C" int gs_pose_init(double *d_state, void *stream) {
    if (!d_state || ((uintptr_t)d_state & 15)) return GS_ERR_ARG;
    k_pose_init<<<1, 256, 0, (cudaStream_t)stream>>>(d_state);
    return launch_error();
}

extern "C" int gs_plan_set_pose(gs_plan *plan, double *d_state) {
    if (!plan || ((uintptr_t)d_state & 15)) return GS_ERR_ARG;
    plan->pose = d_state;
    return GS_OK;
}

extern "C" int gs_pose_step(double *d_state, const gs_pose_hparams *hp, void *stream) {
    if (!d_state || ((uintptr_t)d_state & 15) || !hp) return GS_ERR_ARG;
    if (!(hp->b1 >= 0.5 && hp->b1 < 1.0) || !(hp->b2 >= 0.5 && hp->b2 < 1.0) || !(hp->eps >= 0.0) ||
        !(hp->lr_rot >= 0.0) || !(hp->lr_trans >= 0.0))
        return GS_ERR_ARG;
    k_pose_step<<<1, GS_POSE_SLOTS, 0, (cudaStream_t)stream>>>(d_state, *hp);
    return launch_error();
}
