/*
 * Oracle for the per-pixel part of the 3DGS training step, in float64.
 *
 * TEST INFRASTRUCTURE.  This file is the slow, plain CPU definition that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may build, load or call it; the product path
 * never does.  It shares no code, header or constant with the CUDA sources.
 *
 * What it computes (paper Sec. 2.1 "renderCUDA" and Sec. 2.2):
 *   for every pixel of a window, all projected Gaussians whose opacity-aware
 *   level set (Eq. 1) can reach the pixel centre are visited in ascending
 *   camera depth (ties by ascending Gaussian index) and alpha-blended front to
 *   back.  The gradient is the classic per-pixel back-to-front recursion that
 *   Sec. 2.2 describes as the baseline the per-Gaussian backward replaces; it
 *   is the same sum, evaluated in the other order.
 *
 * Readings where the paper is silent (the classic 3DGS conventions it builds
 * on): pixel (i, j) has its centre at (i + 0.5, j + 0.5); with
 * d = centre - mean2d, power = -(a dx^2 + 2 b dx dy + c dy^2) / 2 for the conic
 * (a, b, c); a pair with power > 0 is skipped; alpha = min(0.99, o e^power); a
 * pair with alpha < 1/255 is skipped; if T (1 - alpha) < 1e-4 the pixel stops
 * before blending that pair; C += rgb alpha T, D += alpha T / z (blended
 * disparity, Sec. 3.1), T *= 1 - alpha; the output colour is C + T bg.
 *
 * The per-pixel candidate set is every Gaussian whose level-set bounding box
 * (half-extents sqrt(t Sxx), sqrt(t Syy), t = 2 ln(255 o), widened by one
 * pixel) holds the pixel centre.  Outside the level set alpha < 1/255, so the
 * cull cannot change any result; it only keeps the oracle's cost at the sum of
 * box areas instead of pixels x Gaussians.
 *
 * Ambiguity flags: a pixel is flagged when a float32 evaluation of the same
 * definition could take another branch: some candidate has alpha within a
 * band of the 1/255 cut, the clamp switches within a band of 0.99, the stop
 * test T (1 - alpha) is within a band of 1e-4, or two blended candidates have
 * depths within a relative band (their order could flip).  The alpha and
 * clamp bands are a relative part plus the change of ln(alpha) that a shift
 * of the projected mean by pos_abs pixels causes (|d power / d mean| pos_abs);
 * the stop band adds the same shifts and the relative alpha error cond_eps,
 * both propagated through T (a long chain of high-alpha splats widens it
 * through the factors alpha / (1 - alpha)).  A pixel is also
 * flagged when its value is ill-conditioned: when relative errors of cond_eps
 * in every blended alpha could move a colour channel, D or T by more than half
 * of the per-pixel tolerance 1e-4 |v| + 1e-7 (first-order bound
 * sum_k alpha_k |dv/dalpha_k| cond_eps, where a long chain of high-alpha
 * splats amplifies the error of T through the factors 1 / (1 - alpha)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Projected Gaussian record, one row of ORC_STRIDE doubles per Gaussian. */
enum {
    ORC_MX = 0, ORC_MY, ORC_A, ORC_B, ORC_C, ORC_O, ORC_R, ORC_G, ORC_BL,
    ORC_Z, ORC_T, ORC_VALID, ORC_STRIDE
};

#define ORC_ALPHA_MIN (1.0 / 255.0)
#define ORC_ALPHA_MAX 0.99
#define ORC_T_STOP 1e-4

typedef struct {
    double alpha_rel;  /* band around the 1/255 cut, relative */
    double clamp_rel;  /* band around the 0.99 clamp, relative */
    double tstop_rel;  /* band around the 1e-4 stop, relative */
    double depth_rel;  /* relative depth gap under which order may flip */
    double pos_abs;    /* absolute uncertainty of a float32 mean2d, pixels */
    double cond_eps;   /* relative float32 error of each alpha (conditioning flag) */
} orc_amb;

typedef struct {
    int64_t *start;  /* (npix + 1) CSR offsets */
    int64_t *ids;    /* candidate Gaussian ids, per pixel sorted by (z, id) */
} orc_lists;

static const double *g_sort_proj; /* read-only during the sorts below */

static int cmp_depth_id(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    double za = g_sort_proj[a * ORC_STRIDE + ORC_Z];
    double zb = g_sort_proj[b * ORC_STRIDE + ORC_Z];
    if (za < zb) return -1;
    if (za > zb) return 1;
    return (a > b) - (a < b);
}

/* Pixel-index range [lo, hi] of a Gaussian's widened level-set box, or 0 if
 * it reaches no pixel of the window. */
static int orc_box(const double *g, int x0, int y0, int x1, int y1,
                   int *ix0, int *iy0, int *ix1, int *iy1) {
    if (g[ORC_VALID] == 0.0 || !(g[ORC_T] > 0.0)) return 0;
    double a = g[ORC_A], b = g[ORC_B], c = g[ORC_C];
    double det = a * c - b * b;
    if (!(det > 0.0)) return 0;
    double sxx = c / det, syy = a / det; /* inverse of the conic */
    double rx = sqrt(g[ORC_T] * sxx) + 1.0, ry = sqrt(g[ORC_T] * syy) + 1.0;
    double lo_x = ceil(g[ORC_MX] - rx - 0.5), hi_x = floor(g[ORC_MX] + rx - 0.5);
    double lo_y = ceil(g[ORC_MY] - ry - 0.5), hi_y = floor(g[ORC_MY] + ry - 0.5);
    if (lo_x < x0) lo_x = x0;
    if (lo_y < y0) lo_y = y0;
    if (hi_x > x1 - 1) hi_x = x1 - 1;
    if (hi_y > y1 - 1) hi_y = y1 - 1;
    if (lo_x > hi_x || lo_y > hi_y) return 0;
    *ix0 = (int)lo_x; *iy0 = (int)lo_y; *ix1 = (int)hi_x; *iy1 = (int)hi_y;
    return 1;
}

static void orc_build_lists(int64_t n, const double *proj, int x0, int y0, int x1, int y1,
                            orc_lists *L) {
    int w = x1 - x0, h = y1 - y0;
    int64_t npix = (int64_t)w * h;
    L->start = (int64_t *)calloc((size_t)npix + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int ax, ay, bx, by;
        if (!orc_box(proj + i * ORC_STRIDE, x0, y0, x1, y1, &ax, &ay, &bx, &by)) continue;
        for (int y = ay; y <= by; ++y)
            for (int x = ax; x <= bx; ++x)
                L->start[(int64_t)(y - y0) * w + (x - x0) + 1] += 1;
    }
    for (int64_t p = 0; p < npix; ++p) L->start[p + 1] += L->start[p];
    L->ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L->start[npix] > 0 ? L->start[npix] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(npix > 0 ? npix : 1));
    for (int64_t p = 0; p < npix; ++p) fill[p] = L->start[p];
    for (int64_t i = 0; i < n; ++i) { /* ascending id order */
        int ax, ay, bx, by;
        if (!orc_box(proj + i * ORC_STRIDE, x0, y0, x1, y1, &ax, &ay, &bx, &by)) continue;
        for (int y = ay; y <= by; ++y)
            for (int x = ax; x <= bx; ++x) {
                int64_t p = (int64_t)(y - y0) * w + (x - x0);
                L->ids[fill[p]++] = i;
            }
    }
    free(fill);
    g_sort_proj = proj;
    for (int64_t p = 0; p < npix; ++p)
        qsort(L->ids + L->start[p], (size_t)(L->start[p + 1] - L->start[p]), sizeof(int64_t),
              cmp_depth_id);
}

static void orc_free_lists(orc_lists *L) {
    free(L->start);
    free(L->ids);
}

/* Per-pair evaluation shared by the forward and the backward. */
typedef struct {
    double dx, dy, power, G, raw, alpha;
    int clamped;
} orc_pair;

static void orc_eval(const double *g, double px, double py, orc_pair *e) {
    e->dx = px - g[ORC_MX];
    e->dy = py - g[ORC_MY];
    double q = g[ORC_A] * e->dx * e->dx + 2.0 * g[ORC_B] * e->dx * e->dy + g[ORC_C] * e->dy * e->dy;
    e->power = -0.5 * q;
    e->G = exp(e->power);
    e->raw = g[ORC_O] * e->G;
    e->clamped = e->raw > ORC_ALPHA_MAX;
    e->alpha = e->clamped ? ORC_ALPHA_MAX : e->raw;
}

/*
 * Forward over the window [x0, x1) x [y0, y1).
 * out_rgb: planar 3 x h x w; out_disp, out_T: h x w; out_count: number of
 * blended Gaussians per pixel; out_amb: ambiguity flag per pixel.
 * Any output pointer may be NULL.  Returns the total number of candidates.
 */
int64_t orc_render_fwd(int64_t n, const double *proj, const double *bg,
                       int x0, int y0, int x1, int y1, const orc_amb *amb,
                       double *out_rgb, double *out_disp, double *out_T,
                       int32_t *out_count, uint8_t *out_amb, int n_threads) {
    orc_lists L;
    orc_build_lists(n, proj, x0, y0, x1, y1, &L);
    int w = x1 - x0, h = y1 - y0;
    int64_t npix = (int64_t)w * h;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
    int64_t cap = 64;
    int64_t *blist = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    double *bal = (double *)malloc(sizeof(double) * (size_t)cap);
    double *bT = (double *)malloc(sizeof(double) * (size_t)cap);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
    for (int64_t p = 0; p < npix; ++p) {
        double px = (double)(x0 + p % w) + 0.5, py = (double)(y0 + p / w) + 0.5;
        double T = 1.0, C[3] = {0.0, 0.0, 0.0}, D = 0.0, prev_z = -1.0, t_sens = 0.0;
        int64_t ncand = L.start[p + 1] - L.start[p];
        if (ncand > cap) {
            cap = ncand;
            blist = (int64_t *)realloc(blist, sizeof(int64_t) * (size_t)cap);
            bal = (double *)realloc(bal, sizeof(double) * (size_t)cap);
            bT = (double *)realloc(bT, sizeof(double) * (size_t)cap);
        }
        int32_t count = 0;
        uint8_t flag = 0;
        for (int64_t k = L.start[p]; k < L.start[p + 1]; ++k) {
            const double *g = proj + L.ids[k] * ORC_STRIDE;
            orc_pair e;
            orc_eval(g, px, py, &e);
            double shift = 0.0;
            if (amb) {
                /* |d ln alpha| for a mean2d shift of pos_abs in x and y */
                shift = amb->pos_abs * (fabs(g[ORC_A] * e.dx + g[ORC_B] * e.dy) +
                                        fabs(g[ORC_B] * e.dx + g[ORC_C] * e.dy));
                if (fabs(log(e.raw * 255.0)) < amb->alpha_rel + shift) flag = 1;
                if (fabs(log(e.raw / ORC_ALPHA_MAX)) < amb->clamp_rel + shift) flag = 1;
            }
            if (amb && e.raw * 255.0 >= 1.0 - 2.0 * (amb->alpha_rel + shift)) {
                /* a candidate that blends (or nearly does) with a depth tie
                 * against the previous such candidate: float32 may swap them */
                if (prev_z > 0.0 && fabs(g[ORC_Z] - prev_z) < amb->depth_rel * g[ORC_Z]) flag = 1;
                prev_z = g[ORC_Z];
            }
            if (e.power > 0.0) continue;
            if (e.alpha < ORC_ALPHA_MIN) continue;
            double test_T = T * (1.0 - e.alpha);
            if (amb) {
                /* ln T moves by alpha / (1 - alpha) times the relative change of
                 * alpha: from a mean2d shift, and from the relative float32 error
                 * cond_eps that every alpha carries (a clamped alpha is exact) */
                double s_here = t_sens + (e.clamped ? 0.0 : e.alpha / (1.0 - e.alpha) * (shift + amb->cond_eps));
                if (fabs(log(test_T / ORC_T_STOP)) < amb->tstop_rel + s_here) flag = 1;
                t_sens = s_here;
            }
            if (test_T < ORC_T_STOP) {
                /* the candidate right after the stopping one could take its
                 * place under a depth tie */
                for (int64_t k2 = k + 1; amb && k2 < L.start[p + 1]; ++k2) {
                    const double *g2 = proj + L.ids[k2] * ORC_STRIDE;
                    orc_pair e2;
                    orc_eval(g2, px, py, &e2);
                    if (e2.raw * 255.0 < 1.0 - 2.0 * amb->alpha_rel) continue;
                    if (fabs(g2[ORC_Z] - g[ORC_Z]) < amb->depth_rel * g2[ORC_Z]) flag = 1;
                    break;
                }
                break;
            }
            double wgt = e.alpha * T;
            C[0] += g[ORC_R] * wgt;
            C[1] += g[ORC_G] * wgt;
            C[2] += g[ORC_BL] * wgt;
            D += wgt / g[ORC_Z];
            blist[count] = e.clamped ? -1 - L.ids[k] : L.ids[k];
            bal[count] = e.alpha;
            bT[count] = T;
            T = test_T;
            ++count;
        }
        if (amb && amb->cond_eps > 0.0 && !flag) {
            /* first-order sensitivity of C (3), D and T to relative alpha errors */
            double behind[4] = {T * bg[0], T * bg[1], T * bg[2], 0.0};
            double sens[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            double sumT = 0.0;
            for (int32_t j = count - 1; j >= 0; --j) {
                int64_t id = blist[j] < 0 ? -1 - blist[j] : blist[j];
                const double *g = proj + id * ORC_STRIDE;
                double vals[4] = {g[ORC_R], g[ORC_G], g[ORC_BL], 1.0 / g[ORC_Z]};
                double a = bal[j], Tj = bT[j];
                for (int c = 0; c < 4; ++c) {
                    if (blist[j] >= 0) sens[c] += a * fabs(vals[c] * Tj - behind[c] / (1.0 - a));
                    behind[c] += vals[c] * a * Tj;
                }
                if (blist[j] >= 0) sumT += a / (1.0 - a);
            }
            sens[4] = T * sumT;
            double v[5] = {C[0] + T * bg[0], C[1] + T * bg[1], C[2] + T * bg[2], D, T};
            for (int c = 0; c < 5; ++c)
                if (sens[c] * amb->cond_eps > 0.5 * (1e-4 * fabs(v[c]) + 1e-7)) flag = 1;
        }
        if (out_rgb) {
            out_rgb[p] = C[0] + T * bg[0];
            out_rgb[npix + p] = C[1] + T * bg[1];
            out_rgb[2 * npix + p] = C[2] + T * bg[2];
        }
        if (out_disp) out_disp[p] = D;
        if (out_T) out_T[p] = T;
        if (out_count) out_count[p] = count;
        if (out_amb) out_amb[p] = flag;
    }
    free(blist);
    free(bal);
    free(bT);
    }
    int64_t total = L.start[npix];
    orc_free_lists(&L);
    return total;
}

/*
 * Backward over the window.  g_rgb (3 x h x w planar) and g_disp (h x w) are
 * dL/d(output colour) and dL/d(blended disparity).  Gradients are ADDED into
 * the per-Gaussian accumulators, ORC_G2D doubles per Gaussian:
 *   [0, 1] mean2d (x, y); [2, 3, 4] conic (a, b, c); [5] opacity;
 *   [6, 7, 8] rgb; [9] inverse depth 1/z.
 * The conic gradient is taken with respect to the entries a, b, c of
 * q = a dx^2 + 2 b dx dy + c dy^2.
 */
#define ORC_G2D 10
void orc_render_bwd(int64_t n, const double *proj, const double *bg,
                    int x0, int y0, int x1, int y1,
                    const double *g_rgb, const double *g_disp, double *grad2d, int n_threads) {
    orc_lists L;
    orc_build_lists(n, proj, x0, y0, x1, y1, &L);
    int w = x1 - x0, h = y1 - y0;
    int64_t npix = (int64_t)w * h;
    int nt = 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
    nt = omp_get_max_threads();
#endif
    /* Per-thread accumulators over the Gaussians that reach the window. */
    int64_t *local = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t n_local = 0;
    for (int64_t i = 0; i < n; ++i) local[i] = -1;
    for (int64_t k = 0; k < L.start[npix]; ++k)
        if (local[L.ids[k]] < 0) local[L.ids[k]] = n_local++;
    int64_t *global_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_local > 0 ? n_local : 1));
    for (int64_t i = 0; i < n; ++i)
        if (local[i] >= 0) global_of[local[i]] = i;
    double *acc = (double *)calloc((size_t)nt * (size_t)(n_local > 0 ? n_local : 1) * ORC_G2D,
                                   sizeof(double));
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = acc + (size_t)tid * (size_t)n_local * ORC_G2D;
        int64_t cap = 64;
        int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        orc_pair *pairs = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)cap);
        double *Ts = (double *)malloc(sizeof(double) * (size_t)cap);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t p = 0; p < npix; ++p) {
            double px = (double)(x0 + p % w) + 0.5, py = (double)(y0 + p / w) + 0.5;
            int64_t ncand = L.start[p + 1] - L.start[p];
            if (ncand > cap) {
                cap = ncand;
                list = (int64_t *)realloc(list, sizeof(int64_t) * (size_t)cap);
                pairs = (orc_pair *)realloc(pairs, sizeof(orc_pair) * (size_t)cap);
                Ts = (double *)realloc(Ts, sizeof(double) * (size_t)cap);
            }
            /* Forward again, recording the blended pairs. */
            double T = 1.0;
            int64_t m = 0;
            for (int64_t k = L.start[p]; k < L.start[p + 1]; ++k) {
                const double *g = proj + L.ids[k] * ORC_STRIDE;
                orc_pair e;
                orc_eval(g, px, py, &e);
                if (e.power > 0.0 || e.alpha < ORC_ALPHA_MIN) continue;
                double test_T = T * (1.0 - e.alpha);
                if (test_T < ORC_T_STOP) break;
                list[m] = L.ids[k];
                pairs[m] = e;
                Ts[m] = T;
                ++m;
                T = test_T;
            }
            double gC[3] = {g_rgb[p], g_rgb[npix + p], g_rgb[2 * npix + p]};
            double gD = g_disp[p];
            /* Back to front: suffix sums of what lies behind splat k. */
            double behindC[3] = {T * bg[0], T * bg[1], T * bg[2]};
            double behindD = 0.0;
            for (int64_t j = m - 1; j >= 0; --j) {
                const double *g = proj + list[j] * ORC_STRIDE;
                const orc_pair *e = &pairs[j];
                double Tk = Ts[j], a = e->alpha;
                double rgb[3] = {g[ORC_R], g[ORC_G], g[ORC_BL]};
                double invz = 1.0 / g[ORC_Z];
                double *out = my + (size_t)local[list[j]] * ORC_G2D;
                double dL_dalpha = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    out[6 + ch] += a * Tk * gC[ch];
                    dL_dalpha += gC[ch] * (rgb[ch] * Tk - behindC[ch] / (1.0 - a));
                }
                out[9] += a * Tk * gD;
                dL_dalpha += gD * (invz * Tk - behindD / (1.0 - a));
                for (int ch = 0; ch < 3; ++ch) behindC[ch] += rgb[ch] * a * Tk;
                behindD += invz * a * Tk;
                if (e->clamped) continue; /* alpha = 0.99 does not depend on o or power */
                out[5] += dL_dalpha * e->G;
                double dL_dpower = dL_dalpha * e->raw;
                double dx = e->dx, dy = e->dy;
                /* power = -(a dx^2 + 2 b dx dy + c dy^2)/2, dx = px - mx */
                out[0] += dL_dpower * (g[ORC_A] * dx + g[ORC_B] * dy);
                out[1] += dL_dpower * (g[ORC_B] * dx + g[ORC_C] * dy);
                out[2] += dL_dpower * (-0.5 * dx * dx);
                out[3] += dL_dpower * (-dx * dy);
                out[4] += dL_dpower * (-0.5 * dy * dy);
            }
        }
        free(list);
        free(pairs);
        free(Ts);
    }
    for (int64_t li = 0; li < n_local; ++li)
        for (int t = 0; t < nt; ++t)
            for (int c = 0; c < ORC_G2D; ++c)
                grad2d[global_of[li] * ORC_G2D + c] += acc[((size_t)t * n_local + li) * ORC_G2D + c];
    free(acc);
    free(global_of);
    free(local);
    orc_free_lists(&L);
}

/*
 * Contributor-weighted sums for score-guided densification (Sec. 3.2, Eq. 4
 * and Eq. 6): for every pixel of the window and every Gaussian the forward
 * blends there (the same rules as orc_render_fwd: alpha >= 1/255, before the
 * transmittance stop), ADD the pixel's weight weight[p] (h x w) to
 * out_score[id].  Serial over pixels, in pixel order.
 */
void orc_contrib_score(int64_t n, const double *proj, int x0, int y0, int x1, int y1,
                       const double *weight, double *out_score) {
    orc_lists L;
    orc_build_lists(n, proj, x0, y0, x1, y1, &L);
    int w = x1 - x0, h = y1 - y0;
    int64_t npix = (int64_t)w * h;
    for (int64_t p = 0; p < npix; ++p) {
        if (weight[p] == 0.0) continue;
        double px = (double)(x0 + p % w) + 0.5, py = (double)(y0 + p / w) + 0.5;
        double T = 1.0;
        for (int64_t k = L.start[p]; k < L.start[p + 1]; ++k) {
            const double *g = proj + L.ids[k] * ORC_STRIDE;
            orc_pair e;
            orc_eval(g, px, py, &e);
            if (e.power > 0.0 || e.alpha < ORC_ALPHA_MIN) continue;
            double test_T = T * (1.0 - e.alpha);
            if (test_T < ORC_T_STOP) break;
            out_score[L.ids[k]] += weight[p];
            T = test_T;
        }
    }
    (void)h;
    orc_free_lists(&L);
}

int orc_stride(void) { return ORC_STRIDE; }
int orc_g2d(void) { return ORC_G2D; }
