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
 *   level set (Eq. 1) can reach the pixel centre are visited in depth order
 *   and alpha-blended front to back.  The gradient is the classic per-pixel
 *   back-to-front recursion that Sec. 2.2 describes as the baseline the
 *   per-Gaussian backward replaces; it is the same sum, evaluated in the other
 *   order.
 *
 * Readings where the paper is silent (the classic 3DGS conventions it builds
 * on): pixel (i, j) has its centre at (i + 0.5, j + 0.5); with
 * d = centre - mean2d, power = -(a dx^2 + 2 b dx dy + c dy^2) / 2 for the conic
 * (a, b, c); a pair with power > 0 is skipped; alpha = min(0.99, o e^power); a
 * pair with alpha < 1/255 is skipped; if T (1 - alpha) < 1e-4 the pixel stops
 * before blending that pair; C += rgb alpha T, D += alpha T / z (blended
 * disparity, Sec. 3.1), T *= 1 - alpha; the output colour is C + T bg.
 * The depth order is the order of the float32 depth (the sort key of
 * Sec. 2.1 holds the bits of a float32 depth), equal float32 depths by
 * ascending Gaussian index.
 *
 * The per-pixel candidate set is every Gaussian whose level-set bounding box
 * (half-extents sqrt(t Sxx), sqrt(t Syy), t = 2 ln(255 o), widened by one
 * pixel) holds the pixel centre.  Outside the level set alpha < 1/255, so the
 * cull cannot change any result; it only keeps the oracle's cost at the sum of
 * box areas instead of pixels x Gaussians.
 *
 * Where float32 decides a branch.  A float32 evaluation of the same
 * definition may decide a threshold differently when the float64 value lies
 * close to it.  For every pair the oracle bounds the float32 error of
 * ln alpha (orc_amb below: a fixed part, the rounding of the quadratic form
 * relative to the sum of its absolute terms, the relative error of the
 * float32 conic, which grows with its condition number, and the rounding of
 * a tile-local projected mean) and carries the bounds through T.  A pixel is
 * flagged, by reason (ORC_F_* bits), when the 1/255 cut, the 0.99 clamp or
 * the 1e-4 stop of some candidate lies inside its band, or when a depth order
 * could change (a float32 depth within z_rel of a rounding midpoint, or, with
 * depth_rel > 0, two blended depths within depth_rel of each other).  For a
 * flagged pixel with at most ORC_MAX_DEC uncertain cut / clamp / stop
 * decisions, the oracle evaluates every combination of those decisions taken
 * the other way ("alternatives"): a float32 result must then match the
 * canonical branch or one of them.  Pixels with a possible depth swap or more
 * decisions are flagged as unresolved.
 *
 * Conditioning.  With the same per-pair bounds the oracle returns, per pixel
 * and value (C, D, T), the first-order bound sum_k |dv/d ln alpha_k| eps_k
 * plus the rounding of T at each blended splat; a pixel whose bound exceeds
 * the per-pixel tolerance 1e-4 |v| + 1e-7 is flagged ORC_F_COND (there the
 * tolerance alone does not cover a float32 evaluation; a comparison adds the
 * bound to it).
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
#define ORC_DILATION 0.3
#define ORC_TILE 16.0

/* flag bits */
#define ORC_F_CUT 1
#define ORC_F_CLAMP 2
#define ORC_F_STOP 4
#define ORC_F_DEPTH 8
#define ORC_F_COND 16
#define ORC_F_UNRESOLVED 32

/* decision kinds */
#define ORC_D_CUT 0
#define ORC_D_CLAMP 1
#define ORC_D_STOP 2
#define ORC_MAX_DEC 4

typedef struct {
    double ln_abs;     /* fixed band of ln alpha (absolute) */
    double tstop_abs;  /* fixed band of ln T at the stop (absolute) */
    double depth_rel;  /* two blended depths closer than this (relative) may swap */
    double q_rel;      /* rounding of q per unit of |a dx^2| + 2 |b dx dy| + |c dy^2| */
    double conic_rel;  /* relative error of the float32 conic in its worst direction ... */
    double kappa_rel;  /* ... plus this much per unit of the conic's condition number */
    double pos_rel;    /* rounding of a tile-local mean, relative to its distance from the tile origin + 16 */
    double t_rel;      /* rounding of T at each blended splat (relative) */
    double z_rel;      /* band around a float32 rounding midpoint of the depth (relative) */
} orc_amb;

typedef struct {
    int64_t *start;  /* (npix + 1) CSR offsets */
    int64_t *ids;    /* candidate Gaussian ids, per pixel sorted by (float32 z, id) */
} orc_lists;

static const double *g_sort_proj; /* read-only during the sorts below */

static int cmp_depth_id(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    float za = (float)g_sort_proj[a * ORC_STRIDE + ORC_Z];
    float zb = (float)g_sort_proj[b * ORC_STRIDE + ORC_Z];
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
    double dx, dy, power, G, raw;
} orc_pair;

static void orc_eval(const double *g, double px, double py, orc_pair *e) {
    e->dx = px - g[ORC_MX];
    e->dy = py - g[ORC_MY];
    double q = g[ORC_A] * e->dx * e->dx + 2.0 * g[ORC_B] * e->dx * e->dy + g[ORC_C] * e->dy * e->dy;
    e->power = -0.5 * q;
    e->G = exp(e->power);
    e->raw = g[ORC_O] * e->G;
}

/* Bound on the float32 error of ln alpha for one pair (see the header):
 *   ln_abs + (E_eval + E_conic) / 2 + E_pos, with
 *   E_eval  = q_rel (|a| dx^2 + 2 |b dx dy| + |c| dy^2): rounding of the
 *             quadratic form evaluated from float32 conic entries,
 *   E_conic = (conic_rel + kappa_rel kappa) q: the float32 conic's relative
 *             error in its worst direction, which grows with the condition
 *             number kappa of the conic (a needle's conic entries are far
 *             larger than its quadratic form along the needle),
 *   E_pos   = pos_rel [(|mx - x0| + 16) |a dx + b dy| + (|my - y0| + 16) |b dx + c dy|]
 *             for the tile origin (x0, y0) of the pixel: a tile-local mean
 *             rounded once. */
static double orc_pair_eps(const double *g, const orc_pair *e, double tx0, double ty0, const orc_amb *amb) {
    double a = g[ORC_A], b = g[ORC_B], c = g[ORC_C];
    double dx = e->dx, dy = e->dy;
    double sabs = fabs(a) * dx * dx + 2.0 * fabs(b * dx * dy) + fabs(c) * dy * dy;
    double q = -2.0 * e->power;
    double tr = a + c, det = a * c - b * b;
    double kappa = 1.0;
    if (det > 0.0) {
        double disc = sqrt(fmax(tr * tr - 4.0 * det, 0.0));
        kappa = (tr + disc) / fmax(tr - disc, 1e-300 * tr);
        if (tr - disc <= 0.0) kappa = (tr + disc) * (tr + disc) / (4.0 * det); /* cancellation-free form */
    }
    double eps = amb->ln_abs + 0.5 * (amb->q_rel * sabs + (amb->conic_rel + amb->kappa_rel * kappa) * q);
    if (amb->pos_rel > 0.0) {
        double ex = amb->pos_rel * (fabs(g[ORC_MX] - tx0) + ORC_TILE);
        double ey = amb->pos_rel * (fabs(g[ORC_MY] - ty0) + ORC_TILE);
        eps += ex * fabs(a * dx + b * dy) + ey * fabs(b * dx + c * dy);
    }
    return eps;
}

/* Is z within z_rel of a midpoint between two adjacent float32 values (its
 * float32 rounding could go either way)?  A depth exactly on a midpoint is
 * not: it arises when the camera transform of the float32 inputs is exact
 * (an axis-aligned camera), and then a compensated evaluation is exact too
 * and both round it to even. */
static int orc_z_near_midpoint(double z, double z_rel) {
    if (z_rel <= 0.0) return 0;
    float f = (float)z;
    double lo = (double)nextafterf(f, -INFINITY), hi = (double)nextafterf(f, INFINITY);
    double d1 = fabs(z - 0.5 * ((double)f + lo)), d2 = fabs(z - 0.5 * ((double)f + hi));
    double band = z_rel * fabs(z);
    return (d1 > 0.0 && d1 < band) || (d2 > 0.0 && d2 < band);
}

/* Per-thread scratch of one pixel's blend. */
typedef struct {
    int64_t cap;
    int64_t *pos;     /* candidate position of each blended splat */
    double *alpha;    /* its alpha */
    double *Tb;       /* T in front of it */
    double *eps;      /* its ln alpha band (0 when clamped) */
    int *clamped;
    orc_pair *pair;
    double *contrib;  /* backward: ORC_G2D values per candidate position */
} orc_scratch;

#define ORC_G2D 10

static void orc_scratch_reserve(orc_scratch *s, int64_t n) {
    if (n <= s->cap) return;
    s->cap = n;
    s->pos = (int64_t *)realloc(s->pos, sizeof(int64_t) * (size_t)n);
    s->alpha = (double *)realloc(s->alpha, sizeof(double) * (size_t)n);
    s->Tb = (double *)realloc(s->Tb, sizeof(double) * (size_t)n);
    s->eps = (double *)realloc(s->eps, sizeof(double) * (size_t)n);
    s->clamped = (int *)realloc(s->clamped, sizeof(int) * (size_t)n);
    s->pair = (orc_pair *)realloc(s->pair, sizeof(orc_pair) * (size_t)n);
    s->contrib = (double *)realloc(s->contrib, sizeof(double) * ORC_G2D * (size_t)n);
}

static void orc_scratch_free(orc_scratch *s) {
    free(s->pos); free(s->alpha); free(s->Tb); free(s->eps); free(s->clamped); free(s->pair);
    free(s->contrib);
}

typedef struct { int64_t pos; int kind; } orc_dec;

typedef struct {
    double C[3], D, T;
    int64_t nblend;
    int64_t last_id;     /* id of the last blended Gaussian, -1 if none */
    uint8_t flags;
    int nd;              /* uncertain decisions found (canonical run) */
    orc_dec dec[ORC_MAX_DEC];
} orc_result;

static int orc_flipped(const orc_dec *fl, int nfl, int64_t pos, int kind) {
    for (int i = 0; i < nfl; ++i)
        if (fl[i].pos == pos && fl[i].kind == kind) return 1;
    return 0;
}

static void orc_add_dec(orc_result *r, int64_t pos, int kind) {
    if (r->nd < ORC_MAX_DEC) {
        r->dec[r->nd].pos = pos;
        r->dec[r->nd].kind = kind;
    }
    r->nd++;
}

/* Blend one pixel over its candidates ids[0 .. ncand) with the decisions in
 * `fl` taken the other way.  With amb (canonical run) the uncertain decisions
 * and the flags are recorded.  The blended splats are left in s. */
static void orc_blend_pixel(const double *proj, const int64_t *ids, int64_t ncand, double px, double py,
                            double tx0, double ty0, const double *bg, const orc_amb *amb,
                            const orc_dec *fl, int nfl, orc_scratch *s, orc_result *r) {
    orc_scratch_reserve(s, ncand > 0 ? ncand : 1);
    double T = 1.0, C[3] = {0.0, 0.0, 0.0}, D = 0.0, epsT = 0.0, prev_z = -1.0;
    int64_t m = 0;
    r->flags = 0;
    r->nd = 0;
    r->last_id = -1;
    for (int64_t k = 0; k < ncand; ++k) {
        const double *g = proj + ids[k] * ORC_STRIDE;
        orc_pair e;
        orc_eval(g, px, py, &e);
        double eps = 0.0;
        if (amb) {
            eps = orc_pair_eps(g, &e, tx0, ty0, amb);
            double lr = log(e.raw);
            if (fabs(lr - log(ORC_ALPHA_MIN)) < eps) orc_add_dec(r, k, ORC_D_CUT), r->flags |= ORC_F_CUT;
            if (fabs(lr - log(ORC_ALPHA_MAX)) < eps) orc_add_dec(r, k, ORC_D_CLAMP), r->flags |= ORC_F_CLAMP;
            if (lr > log(ORC_ALPHA_MIN) - eps) {
                /* a candidate that blends or nearly does: its depth order */
                if (orc_z_near_midpoint(g[ORC_Z], amb->z_rel)) r->flags |= ORC_F_DEPTH;
                if (amb->depth_rel > 0.0 && prev_z > 0.0 && fabs(g[ORC_Z] - prev_z) < amb->depth_rel * g[ORC_Z])
                    r->flags |= ORC_F_DEPTH;
                prev_z = g[ORC_Z];
            }
        }
        if (e.power > 0.0) continue;
        int clamped = (e.raw > ORC_ALPHA_MAX) ^ orc_flipped(fl, nfl, k, ORC_D_CLAMP);
        double alpha = clamped ? ORC_ALPHA_MAX : e.raw;
        int pass = !(alpha < ORC_ALPHA_MIN) ^ orc_flipped(fl, nfl, k, ORC_D_CUT);
        if (!pass) continue;
        double test_T = T * (1.0 - alpha);
        double eps_here = 0.0;
        if (amb) {
            eps_here = epsT + amb->t_rel + (clamped ? 0.0 : alpha / (1.0 - alpha) * eps);
            if (fabs(log(test_T / ORC_T_STOP)) < amb->tstop_abs + eps_here) {
                orc_add_dec(r, k, ORC_D_STOP);
                r->flags |= ORC_F_STOP;
            }
        }
        int stop = (test_T < ORC_T_STOP) ^ orc_flipped(fl, nfl, k, ORC_D_STOP);
        if (stop) {
            /* the next candidate that blends or nearly does could take the
             * stopping one's place if its float32 depth rounds the other way */
            for (int64_t k2 = k + 1; amb && k2 < ncand; ++k2) {
                const double *g2 = proj + ids[k2] * ORC_STRIDE;
                orc_pair e2;
                orc_eval(g2, px, py, &e2);
                if (log(e2.raw) <= log(ORC_ALPHA_MIN) - orc_pair_eps(g2, &e2, tx0, ty0, amb)) continue;
                if (orc_z_near_midpoint(g2[ORC_Z], amb->z_rel)) r->flags |= ORC_F_DEPTH;
                if (amb->depth_rel > 0.0 && fabs(g2[ORC_Z] - g[ORC_Z]) < amb->depth_rel * g2[ORC_Z])
                    r->flags |= ORC_F_DEPTH;
                break;
            }
            break;
        }
        double wgt = alpha * T;
        C[0] += g[ORC_R] * wgt;
        C[1] += g[ORC_G] * wgt;
        C[2] += g[ORC_BL] * wgt;
        D += wgt / g[ORC_Z];
        s->pos[m] = k;
        s->alpha[m] = alpha;
        s->Tb[m] = T;
        s->eps[m] = clamped ? 0.0 : eps;
        s->clamped[m] = clamped;
        s->pair[m] = e;
        ++m;
        T = test_T;
        epsT = eps_here;
        r->last_id = ids[k];
    }
    if (r->nd > ORC_MAX_DEC) r->flags |= ORC_F_UNRESOLVED;
    if (r->flags & ORC_F_DEPTH) r->flags |= ORC_F_UNRESOLVED;
    r->C[0] = C[0] + T * bg[0];
    r->C[1] = C[1] + T * bg[1];
    r->C[2] = C[2] + T * bg[2];
    r->D = D;
    r->T = T;
    r->nblend = m;
}

/* First-order bound of the float32 error of (C r, g, b, D, T) of a blended
 * pixel: sum over blended splats of |dv / d ln alpha_k| eps_k plus the
 * rounding t_rel of T at each splat, carried to everything behind it. */
static void orc_bound(const double *proj, const int64_t *ids, const orc_scratch *s, const orc_result *r,
                      const double *bg, const orc_amb *amb, double *bound) {
    double behind[4] = {r->T * bg[0], r->T * bg[1], r->T * bg[2], 0.0};
    double b[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    double sum_ln_T = 0.0;
    for (int64_t j = r->nblend - 1; j >= 0; --j) {
        const double *g = proj + ids[s->pos[j]] * ORC_STRIDE;
        double vals[4] = {g[ORC_R], g[ORC_G], g[ORC_BL], 1.0 / g[ORC_Z]};
        double a = s->alpha[j], Tj = s->Tb[j];
        for (int c = 0; c < 4; ++c) {
            /* d v / d ln alpha_j = alpha_j (v_j T_j - behind / (1 - alpha_j)) */
            b[c] += a * fabs(vals[c] * Tj - behind[c] / (1.0 - a)) * s->eps[j] + behind[c] * amb->t_rel;
            behind[c] += vals[c] * a * Tj;
        }
        sum_ln_T += a / (1.0 - a) * s->eps[j] + amb->t_rel;
    }
    b[4] = r->T * sum_ln_T;
    for (int c = 0; c < 5; ++c) bound[c] = b[c];
}

/* Magnitudes of one pixel's gradient terms, ADDED into mag at each blended
 * splat's candidate position: every term of orc_pixel_backward with each
 * factor replaced by its absolute value and the colour behind a splat by
 * the pixel's whole absolute composited colour (a float32 backward that
 * recovers what lies behind a splat from the pixel's totals carries an
 * absolute error of the order of those totals).  A float32 evaluation of
 * the terms, summed in any order, is within a small multiple of the unit
 * roundoff times these magnitudes of the exact sums. */
static void orc_pixel_magnitude(const double *proj, const int64_t *ids, const orc_scratch *s,
                                const orc_result *r, const double *bg, const double *gC, double gD,
                                double *mag) {
    double Cabs[3] = {r->T * fabs(bg[0]), r->T * fabs(bg[1]), r->T * fabs(bg[2])};
    double Dabs = 0.0;
    for (int64_t j = 0; j < r->nblend; ++j) {
        const double *g = proj + ids[s->pos[j]] * ORC_STRIDE;
        double w = s->alpha[j] * s->Tb[j];
        Cabs[0] += fabs(g[ORC_R]) * w;
        Cabs[1] += fabs(g[ORC_G]) * w;
        Cabs[2] += fabs(g[ORC_BL]) * w;
        Dabs += fabs(1.0 / g[ORC_Z]) * w;
    }
    for (int64_t j = 0; j < r->nblend; ++j) {
        const double *g = proj + ids[s->pos[j]] * ORC_STRIDE;
        const orc_pair *e = &s->pair[j];
        double Tk = s->Tb[j], a = s->alpha[j];
        double rgb[3] = {g[ORC_R], g[ORC_G], g[ORC_BL]};
        double *out = mag + (size_t)s->pos[j] * ORC_G2D;
        double m_alpha = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            out[6 + ch] += a * Tk * fabs(gC[ch]);
            m_alpha += fabs(gC[ch]) * (fabs(rgb[ch]) * Tk + Cabs[ch] / (1.0 - a));
        }
        out[9] += a * Tk * fabs(gD);
        m_alpha += fabs(gD) * (fabs(1.0 / g[ORC_Z]) * Tk + Dabs / (1.0 - a));
        if (s->clamped[j]) continue;
        out[5] += m_alpha * e->G;
        double m_power = m_alpha * e->raw;
        double dx = fabs(e->dx), dy = fabs(e->dy);
        out[0] += m_power * (fabs(g[ORC_A]) * dx + fabs(g[ORC_B]) * dy);
        out[1] += m_power * (fabs(g[ORC_B]) * dx + fabs(g[ORC_C]) * dy);
        out[2] += m_power * 0.5 * dx * dx;
        out[3] += m_power * dx * dy;
        out[4] += m_power * 0.5 * dy * dy;
    }
}

/* Backward of one pixel for the blended splats in s: ADD the ORC_G2D
 * gradient values of each into s->contrib at its candidate position. */
static void orc_pixel_backward(const double *proj, const int64_t *ids, const orc_scratch *s,
                               const orc_result *r, const double *bg, const double *gC, double gD,
                               double *contrib) {
    double behindC[3] = {r->T * bg[0], r->T * bg[1], r->T * bg[2]};
    double behindD = 0.0;
    for (int64_t j = r->nblend - 1; j >= 0; --j) {
        const double *g = proj + ids[s->pos[j]] * ORC_STRIDE;
        const orc_pair *e = &s->pair[j];
        double Tk = s->Tb[j], a = s->alpha[j];
        double rgb[3] = {g[ORC_R], g[ORC_G], g[ORC_BL]};
        double invz = 1.0 / g[ORC_Z];
        double *out = contrib + (size_t)s->pos[j] * ORC_G2D;
        double dL_dalpha = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            out[6 + ch] += a * Tk * gC[ch];
            dL_dalpha += gC[ch] * (rgb[ch] * Tk - behindC[ch] / (1.0 - a));
        }
        out[9] += a * Tk * gD;
        dL_dalpha += gD * (invz * Tk - behindD / (1.0 - a));
        for (int ch = 0; ch < 3; ++ch) behindC[ch] += rgb[ch] * a * Tk;
        behindD += invz * a * Tk;
        if (s->clamped[j]) continue; /* alpha = 0.99 does not depend on o or power */
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

static void orc_alt_flips(const orc_result *r, int mask, orc_dec *fl, int *nfl) {
    *nfl = 0;
    for (int i = 0; i < r->nd && i < ORC_MAX_DEC; ++i)
        if (mask & (1 << i)) fl[(*nfl)++] = r->dec[i];
}

/*
 * Forward over the window [x0, x1) x [y0, y1).
 * out_rgb: planar 3 x h x w; out_disp, out_T: h x w; out_count: number of
 * blended Gaussians per pixel; out_last: id of the last blended Gaussian
 * (-1: none); out_flags: ORC_F_* bits per pixel; out_bound: 5 x h x w
 * first-order error bounds of (C r, g, b, D, T).  With amb and alt_cap > 0,
 * the alternatives of every flagged, resolved pixel are written to
 * alt_pix (pixel index), alt_val (5 values: C r, g, b, D, T) and alt_last
 * (last blended id) up to alt_cap rows; *n_alt receives the number of rows
 * needed (rows beyond alt_cap are dropped: call again with a larger buffer).
 * Any output pointer may be NULL.  Returns the total number of candidates.
 */
int64_t orc_render_fwd2(int64_t n, const double *proj, const double *bg,
                        int x0, int y0, int x1, int y1, const orc_amb *amb,
                        double *out_rgb, double *out_disp, double *out_T,
                        int32_t *out_count, int64_t *out_last, uint8_t *out_flags, double *out_bound,
                        int64_t alt_cap, int64_t *alt_pix, double *alt_val, int64_t *alt_last,
                        int64_t *n_alt, int n_threads) {
    orc_lists L;
    orc_build_lists(n, proj, x0, y0, x1, y1, &L);
    int w = x1 - x0, h = y1 - y0;
    int64_t npix = (int64_t)w * h;
    int64_t alt_rows = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
    orc_scratch s = {0};
    orc_scratch s2 = {0};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
    for (int64_t p = 0; p < npix; ++p) {
        int ix = x0 + (int)(p % w), iy = y0 + (int)(p / w);
        double px = (double)ix + 0.5, py = (double)iy + 0.5;
        double tx0 = floor(ix / ORC_TILE) * ORC_TILE, ty0 = floor(iy / ORC_TILE) * ORC_TILE;
        const int64_t *ids = L.ids + L.start[p];
        int64_t ncand = L.start[p + 1] - L.start[p];
        orc_result r;
        orc_blend_pixel(proj, ids, ncand, px, py, tx0, ty0, bg, amb, NULL, 0, &s, &r);
        double bound[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        if (amb) {
            orc_bound(proj, ids, &s, &r, bg, amb, bound);
            double v[5] = {r.C[0], r.C[1], r.C[2], r.D, r.T};
            for (int c = 0; c < 5; ++c)
                if (bound[c] > 1e-4 * fabs(v[c]) + 1e-7) r.flags |= ORC_F_COND;
        }
        if (amb && r.nd > 0 && !(r.flags & ORC_F_UNRESOLVED) && alt_cap >= 0) {
            int nalt = (1 << r.nd) - 1;
            int64_t row;
#ifdef _OPENMP
#pragma omp atomic capture
#endif
            { row = alt_rows; alt_rows += nalt; }
            for (int mask = 1; mask <= nalt; ++mask, ++row) {
                orc_dec fl[ORC_MAX_DEC];
                int nfl;
                orc_alt_flips(&r, mask, fl, &nfl);
                orc_result ra;
                orc_blend_pixel(proj, ids, ncand, px, py, tx0, ty0, bg, NULL, fl, nfl, &s2, &ra);
                if (row < alt_cap) {
                    alt_pix[row] = p;
                    alt_val[5 * row + 0] = ra.C[0];
                    alt_val[5 * row + 1] = ra.C[1];
                    alt_val[5 * row + 2] = ra.C[2];
                    alt_val[5 * row + 3] = ra.D;
                    alt_val[5 * row + 4] = ra.T;
                    alt_last[row] = ra.last_id;
                }
            }
        }
        if (out_rgb) {
            out_rgb[p] = r.C[0];
            out_rgb[npix + p] = r.C[1];
            out_rgb[2 * npix + p] = r.C[2];
        }
        if (out_disp) out_disp[p] = r.D;
        if (out_T) out_T[p] = r.T;
        if (out_count) out_count[p] = (int32_t)r.nblend;
        if (out_last) out_last[p] = r.last_id;
        if (out_flags) out_flags[p] = r.flags;
        if (out_bound)
            for (int c = 0; c < 5; ++c) out_bound[(int64_t)c * npix + p] = bound[c];
    }
    orc_scratch_free(&s);
    orc_scratch_free(&s2);
    }
    if (n_alt) *n_alt = alt_rows;
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
 * q = a dx^2 + 2 b dx dy + c dy^2.  grad2d takes the canonical branch at
 * every pixel.  With amb and slack, for every flagged pixel the largest
 * change of each Gaussian's ORC_G2D values over the pixel's alternatives is
 * ADDED to slack (N x ORC_G2D); a Gaussian that is a candidate of an
 * unresolved pixel gets slack = +inf.  With mag, the magnitudes of the
 * canonical branch's terms (orc_pixel_magnitude) are ADDED to mag
 * (N x ORC_G2D).
 */
void orc_render_bwd2(int64_t n, const double *proj, const double *bg,
                     int x0, int y0, int x1, int y1,
                     const double *g_rgb, const double *g_disp, const orc_amb *amb,
                     double *grad2d, double *slack, double *mag, int n_threads) {
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
    size_t per = (size_t)(n_local > 0 ? n_local : 1) * ORC_G2D;
    double *acc = (double *)calloc((size_t)nt * per, sizeof(double));
    double *sacc = (amb && slack) ? (double *)calloc((size_t)nt * per, sizeof(double)) : NULL;
    double *macc = mag ? (double *)calloc((size_t)nt * per, sizeof(double)) : NULL;
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = acc + (size_t)tid * per;
        double *mys = sacc ? sacc + (size_t)tid * per : NULL;
        double *mym = macc ? macc + (size_t)tid * per : NULL;
        orc_scratch s = {0};
        orc_scratch s2 = {0};
        double *canon = NULL;
        int64_t canon_cap = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t p = 0; p < npix; ++p) {
            int ix = x0 + (int)(p % w), iy = y0 + (int)(p / w);
            double px = (double)ix + 0.5, py = (double)iy + 0.5;
            double tx0 = floor(ix / ORC_TILE) * ORC_TILE, ty0 = floor(iy / ORC_TILE) * ORC_TILE;
            const int64_t *ids = L.ids + L.start[p];
            int64_t ncand = L.start[p + 1] - L.start[p];
            double gC[3] = {g_rgb[p], g_rgb[npix + p], g_rgb[2 * npix + p]};
            double gD = g_disp[p];
            orc_result r;
            orc_blend_pixel(proj, ids, ncand, px, py, tx0, ty0, bg, mys ? amb : NULL, NULL, 0, &s, &r);
            if (ncand > canon_cap) {
                canon_cap = ncand;
                canon = (double *)realloc(canon, sizeof(double) * ORC_G2D * (size_t)ncand);
            }
            memset(canon, 0, sizeof(double) * ORC_G2D * (size_t)(ncand > 0 ? ncand : 0));
            orc_pixel_backward(proj, ids, &s, &r, bg, gC, gD, canon);
            for (int64_t k = 0; k < ncand; ++k) {
                double *out = my + (size_t)local[ids[k]] * ORC_G2D;
                for (int c = 0; c < ORC_G2D; ++c) out[c] += canon[k * ORC_G2D + c];
            }
            if (mym) {
                memset(canon, 0, sizeof(double) * ORC_G2D * (size_t)(ncand > 0 ? ncand : 0));
                orc_pixel_magnitude(proj, ids, &s, &r, bg, gC, gD, canon);
                for (int64_t k = 0; k < ncand; ++k) {
                    double *out = mym + (size_t)local[ids[k]] * ORC_G2D;
                    for (int c = 0; c < ORC_G2D; ++c) out[c] += canon[k * ORC_G2D + c];
                }
            }
            if (!mys || (r.nd == 0 && !(r.flags & ORC_F_UNRESOLVED))) continue;
            if (r.flags & ORC_F_UNRESOLVED) {
                for (int64_t k = 0; k < ncand; ++k)
                    for (int c = 0; c < ORC_G2D; ++c) mys[(size_t)local[ids[k]] * ORC_G2D + c] = INFINITY;
                continue;
            }
            /* largest change of each candidate's values over the alternatives */
            int nalt = (1 << r.nd) - 1;
            orc_scratch_reserve(&s2, ncand > 0 ? ncand : 1);
            double *dev = (double *)calloc((size_t)ORC_G2D * (size_t)(ncand > 0 ? ncand : 1), sizeof(double));
            for (int mask = 1; mask <= nalt; ++mask) {
                orc_dec fl[ORC_MAX_DEC];
                int nfl;
                orc_alt_flips(&r, mask, fl, &nfl);
                orc_result ra;
                orc_blend_pixel(proj, ids, ncand, px, py, tx0, ty0, bg, NULL, fl, nfl, &s2, &ra);
                memset(s2.contrib, 0, sizeof(double) * ORC_G2D * (size_t)(ncand > 0 ? ncand : 1));
                orc_pixel_backward(proj, ids, &s2, &ra, bg, gC, gD, s2.contrib);
                for (int64_t k = 0; k < ncand * ORC_G2D; ++k) {
                    double d = fabs(s2.contrib[k] - canon[k]);
                    if (d > dev[k]) dev[k] = d;
                }
            }
            for (int64_t k = 0; k < ncand; ++k)
                for (int c = 0; c < ORC_G2D; ++c) mys[(size_t)local[ids[k]] * ORC_G2D + c] += dev[k * ORC_G2D + c];
            free(dev);
        }
        free(canon);
        orc_scratch_free(&s);
        orc_scratch_free(&s2);
    }
    for (int64_t li = 0; li < n_local; ++li)
        for (int t = 0; t < nt; ++t)
            for (int c = 0; c < ORC_G2D; ++c) {
                grad2d[global_of[li] * ORC_G2D + c] += acc[((size_t)t * n_local + li) * ORC_G2D + c];
                if (sacc) slack[global_of[li] * ORC_G2D + c] += sacc[((size_t)t * n_local + li) * ORC_G2D + c];
                if (macc) mag[global_of[li] * ORC_G2D + c] += macc[((size_t)t * n_local + li) * ORC_G2D + c];
            }
    free(acc);
    free(sacc);
    free(macc);
    free(global_of);
    free(local);
    orc_free_lists(&L);
}

/*
 * Contributor-weighted sums for score-guided densification (Sec. 3.2, Eq. 4
 * and Eq. 6): for every pixel of the window and every Gaussian the forward
 * blends there (the same rules as orc_render_fwd2), ADD the pixel's weight
 * weight[p] (h x w) to out_score[id].  Serial over pixels, in pixel order.
 */
void orc_contrib_score(int64_t n, const double *proj, int x0, int y0, int x1, int y1,
                       const double *weight, double *out_score) {
    orc_lists L;
    orc_build_lists(n, proj, x0, y0, x1, y1, &L);
    int w = x1 - x0;
    int64_t npix = (int64_t)w * (y1 - y0);
    const double zero_bg[3] = {0.0, 0.0, 0.0};
    orc_scratch s = {0};
    for (int64_t p = 0; p < npix; ++p) {
        if (weight[p] == 0.0) continue;
        double px = (double)(x0 + p % w) + 0.5, py = (double)(y0 + p / w) + 0.5;
        const int64_t *ids = L.ids + L.start[p];
        orc_result r;
        orc_blend_pixel(proj, ids, L.start[p + 1] - L.start[p], px, py, 0.0, 0.0, zero_bg, NULL, NULL, 0, &s, &r);
        for (int64_t j = 0; j < r.nblend; ++j) out_score[ids[s.pos[j]]] += weight[p];
    }
    orc_scratch_free(&s);
    orc_free_lists(&L);
}

int orc_stride(void) { return ORC_STRIDE; }
int orc_g2d(void) { return ORC_G2D; }
