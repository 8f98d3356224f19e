/*
 * FP64 CPU oracle for the FUSE-Flow per-frame fusion path (arXiv 2602.01035).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU baseline
 * of the benchmark, never by the product path.  Plain, slow, sequential double
 * precision; library qsort is the only non-trivial primitive.
 *
 * Readings of the paper taken here (each one is also used, independently written, by
 * the CUDA path):
 *  - Eq. 8 has an unbalanced parenthesis; it is read as P = T_i^-1 pi^-1(K_i, u_h, D_i(u_h))
 *    with u_h = [x, y, 1] at the pixel centre, depth being z-depth.
 *  - Eq. 9 sets a rejected point to 0; a rejected point is dropped instead.
 *  - Eq. 4 writes T_ji; it is T_j T_i^-1, evaluated here through world coordinates.
 *  - The depth D_j(u_j) of Eq. 5 is read at the nearest pixel floor(u + 1/2); a view
 *    enters Eq. 7 only if a_z > 0, the pixel lies inside image j and D_j there is valid.
 *    Views that fail are skipped while the printed 1/(K-1) is kept.
 *  - K counts camera i (Eq. 7 divides by K-1); the K-1 views are a static per-camera
 *    list (Sec. II.5(2)b): other cameras by optical-axis angle, then centre distance,
 *    then index.  K-1 = 0 gives V = 1.
 *  - Sec. II.5(1): coarse grid anchored at the world origin; refinement level of a coarse
 *    cell with n_c points is the largest l <= Lmax with n_c >= n_min 4^l (else 0); cell
 *    edge s0 / 2^l.  Points whose finest-level index leaves [-2^19, 2^19) are dropped.
 *  - Sec. II.5(2)a keeps every gated member of a cell in the fusion; the representative
 *    is the member of largest C, ties to the lowest pixel index.
 *  - Eq. 8's preprocessed depth D^r has no stated rule; orc_screen_depth gives the
 *    one read here (a depth range and a relative-jump screen against 4-neighbours), off
 *    by default so that D^r = D.
 *  - Eq. 11 is read as the normalised weighted mean over the cell's members (positions
 *    and colours).  The mean is evaluated with weights divided by the cell's largest
 *    weight, which leaves it unchanged and keeps it defined when every weight underflows.
 */
#include "fuseflow_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define KEY_NONE (~(uint64_t)0)
#define KEY_BIAS ((int64_t)1 << 19)

void orc_default_params(orc_params *p) {
    memset(p, 0, sizeof(*p));
    p->tau = 0.6f;              /* Eq. 9: tau = 0.6 */
    p->k_views = 4;
    p->sigma_m = 0.03;
    p->coarse_cell_m = 0.32;
    p->max_level = 4;
    p->n_min = 32;
    p->depth_format = ORC_DEPTH_U16;
    p->depth_scale = 0.001;
    p->use_conf = 1;
    p->use_consistency = 1;
    p->row_step = 1;
    p->band_m = 1e-5;
    p->band_px = 1e-6;
    p->band_az = 1e-6;
    p->top_k = 0;
}

/* ---------------------------------------------------------------- small linear algebra */
/* x_cam = R x_world + t */
static void to_camera(const orc_camera *c, const double w[3], double a[3]) {
    for (int r = 0; r < 3; ++r)
        a[r] = c->R[3 * r + 0] * w[0] + c->R[3 * r + 1] * w[1] + c->R[3 * r + 2] * w[2] + c->t[r];
}

/* x_world = R^T (x_cam - t), the inverse pose T^-1 of Eq. 5 and Eq. 8 */
static void to_world(const orc_camera *c, const double a[3], double w[3]) {
    double d[3] = {a[0] - c->t[0], a[1] - c->t[1], a[2] - c->t[2]};
    for (int k = 0; k < 3; ++k)
        w[k] = c->R[0 + k] * d[0] + c->R[3 + k] * d[1] + c->R[6 + k] * d[2];
}

/* pi^-1(K, [x, y, 1], z): point at z-depth z on the ray through pixel centre (x, y) */
static void unproject(const orc_camera *c, double x, double y, double z, double p[3]) {
    p[0] = z * (x - c->cx) / c->fx;
    p[1] = z * (y - c->cy) / c->fy;
    p[2] = z;
}

/* Raw depth sample, its validity (D > 0 and finite) and its z in metres. */
static int depth_at(const void *buf, int fmt, int64_t idx, double scale, double *z) {
    double raw;
    if (fmt == ORC_DEPTH_U16) raw = (double)((const uint16_t *)buf)[idx];
    else if (fmt == ORC_DEPTH_F32) raw = (double)((const float *)buf)[idx];
    else raw = ((const double *)buf)[idx];
    if (!(raw > 0.0) || !isfinite(raw)) return 0;
    *z = raw * scale;
    return 1;
}

/* ---------------------------------------------------------------- depth screen (D^r) */
static float raw_as_float(const void *buf, int fmt, int64_t idx) {
    if (fmt == ORC_DEPTH_U16) return (float)((const uint16_t *)buf)[idx];
    if (fmt == ORC_DEPTH_F32) return ((const float *)buf)[idx];
    return (float)((const double *)buf)[idx];
}

/* valid and within the screen's bounds (float32 comparisons on depth units) */
static int screen_in_bounds(float d, float min_u, float max_u) {
    if (!(d > 0.0f) || !isfinite(d)) return 0;
    if (min_u > 0.0f && !(d >= min_u)) return 0;
    if (max_u > 0.0f && !(d <= max_u)) return 0;
    return 1;
}

int orc_screen_depth(const orc_params *p, int32_t w, int32_t h, const void *in, void *out) {
    if (!p || !in || !out || w < 1 || h < 1 || p->depth_scale <= 0) return ORC_ERR_ARG;
    const float min_u = p->screen_min_m > 0 ? (float)(p->screen_min_m / p->depth_scale) : 0.0f;
    const float max_u = p->screen_max_m > 0 ? (float)(p->screen_max_m / p->depth_scale) : 0.0f;
    const float rel = p->screen_edge_rel > 0.0f ? p->screen_edge_rel : 0.0f;
    const int dx[4] = {-1, 1, 0, 0}, dy[4] = {0, 0, -1, 1};
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            const int64_t i = (int64_t)y * w + x;
            const float d = raw_as_float(in, p->depth_format, i);
            int keep = screen_in_bounds(d, min_u, max_u);
            if (keep && rel > 0.0f) {
                const float thr = rel * d;
                for (int k = 0; k < 4 && keep; ++k) {
                    const int xn = x + dx[k], yn = y + dy[k];
                    if (xn < 0 || xn >= w || yn < 0 || yn >= h) continue;
                    const float dn = raw_as_float(in, p->depth_format, (int64_t)yn * w + xn);
                    if (screen_in_bounds(dn, min_u, max_u) && fabsf(d - dn) > thr) keep = 0;
                }
            }
            if (p->depth_format == ORC_DEPTH_U16)
                ((uint16_t *)out)[i] = keep ? ((const uint16_t *)in)[i] : 0;
            else if (p->depth_format == ORC_DEPTH_F32)
                ((float *)out)[i] = keep ? ((const float *)in)[i] : 0.0f;
            else
                ((double *)out)[i] = keep ? ((const double *)in)[i] : 0.0;
        }
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- neighbour table */
typedef struct { double angle, dist; int32_t j; } nb_cand;

static int nb_before(const nb_cand *a, const nb_cand *b) {
    const double tol = 1e-9;
    if (fabs(a->angle - b->angle) > tol) return a->angle < b->angle;
    if (fabs(a->dist - b->dist) > tol) return a->dist < b->dist;
    return a->j < b->j;
}

/* Sec. II.5(2)b: "cameras whose views overlap ... or are spatially closest", read as a
 * static list per camera: the other cameras ordered by the angle between optical axes,
 * then by centre distance, then by index; the first min(K, N) - 1 are kept. */
int orc_neighbours(const orc_camera *cams, int32_t n, int32_t k_views, int32_t *out) {
    if (n < 1 || k_views < 1) return ORC_ERR_ARG;
    int K = k_views < n ? k_views : n;
    nb_cand *c = (nb_cand *)malloc(sizeof(nb_cand) * (size_t)(n > 1 ? n : 1));
    if (!c) return ORC_ERR_NOMEM;
    for (int i = 0; i < n; ++i) {
        double ai[3], ci[3], zero[3] = {0, 0, 0}, ez[3] = {0, 0, 1};
        double wi0[3], wi1[3];
        to_world(&cams[i], zero, wi0);   /* camera centre */
        to_world(&cams[i], ez, wi1);     /* a point one metre down the optical axis */
        for (int k = 0; k < 3; ++k) { ci[k] = wi0[k]; ai[k] = wi1[k] - wi0[k]; }
        int m = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double wj0[3], wj1[3], aj[3], dot = 0, dist2 = 0;
            to_world(&cams[j], zero, wj0);
            to_world(&cams[j], ez, wj1);
            for (int k = 0; k < 3; ++k) {
                aj[k] = wj1[k] - wj0[k];
                dot += ai[k] * aj[k];
                dist2 += (wj0[k] - ci[k]) * (wj0[k] - ci[k]);
            }
            double na = sqrt(ai[0] * ai[0] + ai[1] * ai[1] + ai[2] * ai[2]);
            double nb = sqrt(aj[0] * aj[0] + aj[1] * aj[1] + aj[2] * aj[2]);
            double cs = dot / (na * nb);
            if (cs > 1) cs = 1;
            if (cs < -1) cs = -1;
            c[m].angle = acos(cs);
            c[m].dist = sqrt(dist2);
            c[m].j = j;
            ++m;
        }
        /* insertion sort: stable and deterministic for the tolerance-based order */
        for (int a = 1; a < m; ++a) {
            nb_cand v = c[a];
            int b = a - 1;
            while (b >= 0 && nb_before(&v, &c[b])) { c[b + 1] = c[b]; --b; }
            c[b + 1] = v;
        }
        for (int k = 0; k < K - 1; ++k) out[i * (K - 1) + k] = c[k].j;
    }
    free(c);
    return ORC_OK;
}

/* ---------------------------------------------------------------- sorting helpers */
typedef struct { uint64_t key; uint32_t g; uint32_t idx; } sort_item;

static int cmp_item(const void *pa, const void *pb) {
    const sort_item *a = (const sort_item *)pa, *b = (const sort_item *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->g != b->g) return a->g < b->g ? -1 : 1;
    return 0;
}

static uint64_t pack_key(int level, int64_t kx, int64_t ky, int64_t kz) {
    return ((uint64_t)level << 60) | ((uint64_t)(kx + KEY_BIAS) << 40) |
           ((uint64_t)(ky + KEY_BIAS) << 20) | (uint64_t)(kz + KEY_BIAS);
}

/* Sec. II.5(1)d: smaller cells where the coarse density is high. */
static int level_of(int64_t n_c, int n_min, int max_level) {
    int l = 0;
    for (int cand = 0; cand <= max_level; ++cand) {
        double thr = (double)n_min * ldexp(1.0, 2 * cand);   /* n_min 4^l */
        if ((double)n_c >= thr) l = cand;
    }
    return l;
}

static int64_t find_key(const uint64_t *keys, int64_t n, uint64_t k) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (keys[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && keys[lo] == k) ? lo : -1;
}

typedef struct { uint32_t rep; int64_t cell; } rep_item;

/* camera index of global pixel g */
static int camera_of(const int64_t *off, int n, int64_t g) {
    int i = 0;
    while (i + 1 < n && g >= off[i + 1]) ++i;
    return i;
}

static float conf_of(const float *const *conf, const int64_t *off, int n, int64_t g) {
    const int i = camera_of(off, n, g);
    return conf[i][g - off[i]];
}

static int cmp_rep(const void *pa, const void *pb) {
    const rep_item *a = (const rep_item *)pa, *b = (const rep_item *)pb;
    return a->rep < b->rep ? -1 : (a->rep > b->rep ? 1 : 0);
}

/* ---------------------------------------------------------------- the frame */
static int fuse_frame_on(const orc_camera *cams, int32_t n, const orc_params *p,
                         const void *const *depth, const float *const *conf,
                         const uint8_t *const *rgb, orc_points *pts, orc_cells *cells,
                         int64_t cell_capacity, orc_stats *st);

/* Eq. 8's D^r first (when a screen is set), then the frame on it */
int orc_fuse_frame(const orc_camera *cams, int32_t n, const orc_params *p,
                   const void *const *depth, const float *const *conf,
                   const uint8_t *const *rgb, orc_points *pts, orc_cells *cells,
                   int64_t cell_capacity, orc_stats *st) {
    if (!cams || n < 1 || !p || !depth) return ORC_ERR_ARG;
    if (!(p->screen_min_m > 0) && !(p->screen_max_m > 0) && !(p->screen_edge_rel > 0.0f))
        return fuse_frame_on(cams, n, p, depth, conf, rgb, pts, cells, cell_capacity, st);
    const size_t esz = p->depth_format == ORC_DEPTH_U16 ? 2 : p->depth_format == ORC_DEPTH_F32 ? 4 : 8;
    void **dr = (void **)calloc((size_t)n, sizeof(void *));
    int rc = dr ? ORC_OK : ORC_ERR_NOMEM;
    for (int i = 0; i < n && rc == ORC_OK; ++i) {
        dr[i] = malloc(esz * (size_t)cams[i].width * (size_t)cams[i].height);
        rc = dr[i] ? orc_screen_depth(p, cams[i].width, cams[i].height, depth[i], dr[i]) : ORC_ERR_NOMEM;
    }
    if (rc == ORC_OK)
        rc = fuse_frame_on(cams, n, p, (const void *const *)dr, conf, rgb, pts, cells, cell_capacity, st);
    for (int i = 0; dr && i < n; ++i) free(dr[i]);
    free(dr);
    return rc;
}

static int fuse_frame_on(const orc_camera *cams, int32_t n, const orc_params *p,
                         const void *const *depth, const float *const *conf,
                         const uint8_t *const *rgb, orc_points *pts, orc_cells *cells,
                         int64_t cell_capacity, orc_stats *st) {
    if (!cams || n < 1 || !p || !depth || !conf || !rgb || !st) return ORC_ERR_ARG;
    if (p->k_views < 1 || p->sigma_m <= 0 || p->coarse_cell_m <= 0 || p->max_level < 0 ||
        p->max_level > 14 || p->n_min < 1 || p->depth_scale <= 0 || p->top_k < 0)
        return ORC_ERR_ARG;
    const int K = p->k_views < n ? p->k_views : n;
    const int K1 = K - 1;
    const int row_step = p->row_step > 0 ? p->row_step : 1;

    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!off) return ORC_ERR_NOMEM;
    off[0] = 0;
    for (int i = 0; i < n; ++i) off[i + 1] = off[i] + (int64_t)cams[i].width * cams[i].height;
    const int64_t npx = off[n];

    int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * (K1 > 0 ? K1 : 1)));
    double *pw = (double *)malloc(sizeof(double) * 3 * (size_t)npx);
    double *lw = (double *)malloc(sizeof(double) * (size_t)npx);      /* ln omega */
    double *om = (double *)malloc(sizeof(double) * (size_t)npx);      /* omega */
    uint8_t *flag = (uint8_t *)calloc((size_t)npx, 1);                /* 1 gated, 2 in range, 4 tie */
    if (!nbr || !pw || !lw || !om || !flag) {
        free(off); free(nbr); free(pw); free(lw); free(om); free(flag);
        return ORC_ERR_NOMEM;
    }
    if (K1 > 0) orc_neighbours(cams, n, p->k_views, nbr);

    memset(st, 0, sizeof(*st));
    for (int k = 0; k < 3; ++k) { st->bbox[k] = INFINITY; st->bbox[3 + k] = -INFINITY; }
    const double sigma2 = p->sigma_m * p->sigma_m;

    /* Eq. 8-10 per pixel, camera by camera, row by row */
    for (int i = 0; i < n; ++i) {
        const orc_camera *ci = &cams[i];
        for (int y = 0; y < ci->height; ++y) {
            for (int x = 0; x < ci->width; ++x) {
                const int64_t li = (int64_t)y * ci->width + x;
                const int64_t g = off[i] + li;
                double z = 0;
                int valid = (y % row_step == 0) &&
                            depth_at(depth[i], p->depth_format, li, p->depth_scale, &z);
                const float C = conf[i][li];
                int gated = valid && (p->use_conf ? (C > p->tau) : 1);   /* Eq. 9 */
                if (pts && pts->valid) pts->valid[g] = (uint8_t)valid;
                if (pts && pts->gated) pts->gated[g] = (uint8_t)gated;
                if (pts && pts->nview) pts->nview[g] = -1;
                if (pts && pts->margin_tie_px) pts->margin_tie_px[g] = INFINITY;
                if (pts && pts->min_az) pts->min_az[g] = INFINITY;
                st->n_valid += valid;
                if (!gated) continue;
                st->n_gated += 1;
                flag[g] |= 1;

                /* Eq. 8: P = T_i^-1 pi^-1(K_i, [x, y, 1], D) */
                double pc[3], P[3];
                unproject(ci, (double)x, (double)y, z, pc);
                to_world(ci, pc, P);
                for (int k = 0; k < 3; ++k) {
                    pw[3 * g + k] = P[k];
                    if (P[k] < st->bbox[k]) st->bbox[k] = P[k];
                    if (P[k] > st->bbox[3 + k]) st->bbox[3 + k] = P[k];
                }

                /* Eq. 4-7 over the K-1 neighbour views */
                double sum = 0.0, tie = INFINITY, minaz = INFINITY;
                int nview = 0;
                if (p->use_consistency && K1 > 0) {
                    for (int q = 0; q < K1; ++q) {
                        const int j = nbr[i * K1 + q];
                        const orc_camera *cj = &cams[j];
                        double a[3];
                        to_camera(cj, P, a);                    /* T_ji P via the world */
                        if (fabs(a[2]) < minaz) minaz = fabs(a[2]);
                        if (!(a[2] > 0.0)) continue;            /* behind camera j */
                        double u = cj->fx * a[0] / a[2] + cj->cx; /* Eq. 4 */
                        double v = cj->fy * a[1] / a[2] + cj->cy;
                        double fu = u + 0.5, fv = v + 0.5;
                        double mu = fabs(fu - nearbyint(fu)), mv = fabs(fv - nearbyint(fv));
                        if (mu < tie) tie = mu;
                        if (mv < tie) tie = mv;
                        double px = floor(fu), py = floor(fv);
                        if (!(px >= 0.0 && px < (double)cj->width && py >= 0.0 &&
                              py < (double)cj->height))
                            continue;                           /* field-of-view check */
                        const int64_t lj = (int64_t)py * cj->width + (int64_t)px;
                        double zj;
                        if (!depth_at(depth[j], p->depth_format, lj, p->depth_scale, &zj))
                            continue;
                        double qc[3], Q[3];                     /* Eq. 5 */
                        unproject(cj, px, py, zj, qc);
                        to_world(cj, qc, Q);
                        double d2 = 0.0;                        /* Eq. 6 */
                        for (int k = 0; k < 3; ++k) d2 += (P[k] - Q[k]) * (P[k] - Q[k]);
                        sum += d2 / sigma2;
                        nview += 1;
                    }
                }
                double e = (K1 > 0 && p->use_consistency) ? sum / (double)K1 : 0.0;  /* Eq. 7 */
                double V = exp(-e);
                double omega = p->use_conf ? (double)C * V : V;                    /* Eq. 10 */
                double logw = (p->use_conf ? log((double)C) : 0.0) - e;
                om[g] = omega;
                lw[g] = logw;
                if (tie < p->band_px || minaz < p->band_az) flag[g] |= 4;
                if (pts) {
                    if (pts->pw) for (int k = 0; k < 3; ++k) pts->pw[3 * g + k] = P[k];
                    if (pts->e) pts->e[g] = e;
                    if (pts->omega) pts->omega[g] = omega;
                    if (pts->log_omega) pts->log_omega[g] = logw;
                    if (pts->nview) pts->nview[g] = nview;
                    if (pts->margin_tie_px) pts->margin_tie_px[g] = tie;
                    if (pts->min_az) pts->min_az[g] = minaz;
                }
            }
        }
    }
    st->n_tie_points = 0;
    for (int64_t g = 0; g < npx; ++g) st->n_tie_points += (flag[g] & 4) ? 1 : 0;

    /* Sec. II.5(1)b-c: coarse grid of edge s0 anchored at the world origin */
    const double s0 = p->coarse_cell_m;
    const int L = p->max_level;
    int64_t n_pts = 0;
    for (int64_t g = 0; g < npx; ++g) {
        if (!(flag[g] & 1)) continue;
        int ok = 1;
        for (int k = 0; k < 3; ++k) {
            double f = floor(ldexp(pw[3 * g + k] / s0, L));
            if (!(f >= -(double)KEY_BIAS && f < (double)KEY_BIAS)) ok = 0;
        }
        if (ok) { flag[g] |= 2; ++n_pts; }
        else st->n_out_of_range += 1;
    }
    sort_item *items = (sort_item *)malloc(sizeof(sort_item) * (size_t)(n_pts > 0 ? n_pts : 1));
    uint64_t *ckeys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_pts > 0 ? n_pts : 1));
    int64_t *ccount = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_pts > 0 ? n_pts : 1));
    int64_t *b_in = (int64_t *)calloc((size_t)(n_pts > 0 ? n_pts : 1), sizeof(int64_t));
    int64_t *b_out = (int64_t *)calloc((size_t)(n_pts > 0 ? n_pts : 1), sizeof(int64_t));
    uint8_t *amb = (uint8_t *)calloc((size_t)(n_pts > 0 ? n_pts : 1), 1);
    uint64_t *pkey = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(npx > 0 ? npx : 1));
    if (!items || !ckeys || !ccount || !b_in || !b_out || !amb || !pkey) {
        free(off); free(nbr); free(pw); free(lw); free(om); free(flag); free(items);
        free(ckeys); free(ccount); free(b_in); free(b_out); free(amb); free(pkey);
        return ORC_ERR_NOMEM;
    }
    int64_t m = 0;
    for (int64_t g = 0; g < npx; ++g) {
        pkey[g] = KEY_NONE;
        if (!(flag[g] & 2)) continue;
        int64_t kc[3];
        for (int k = 0; k < 3; ++k) kc[k] = (int64_t)floor(pw[3 * g + k] / s0);
        items[m].key = pack_key(0, kc[0], kc[1], kc[2]);
        items[m].g = (uint32_t)g;
        items[m].idx = (uint32_t)m;
        ++m;
    }
    qsort(items, (size_t)n_pts, sizeof(sort_item), cmp_item);
    int64_t n_coarse = 0;
    for (int64_t a = 0; a < n_pts;) {
        int64_t b = a;
        while (b < n_pts && items[b].key == items[a].key) ++b;
        ckeys[n_coarse] = items[a].key;
        ccount[n_coarse] = b - a;        /* density estimate n_c */
        ++n_coarse;
        a = b;
    }
    st->n_coarse = n_coarse;

    /* Coarse cells whose level could change when points within band_m of a coarse
     * boundary fall on the other side (reported, never silently passed). */
    const double dband = p->band_m / s0;
    for (int64_t g = 0; g < npx; ++g) {
        if (!(flag[g] & 2)) continue;
        double r[3];
        int64_t lo[3], hi[3], own[3];
        int near = 0;
        for (int k = 0; k < 3; ++k) {
            r[k] = pw[3 * g + k] / s0;
            own[k] = (int64_t)floor(r[k]);
            lo[k] = (int64_t)floor(r[k] - dband);
            hi[k] = (int64_t)floor(r[k] + dband);
            if (lo[k] != hi[k]) near = 1;
        }
        if (!near) continue;
        int64_t ci = find_key(ckeys, n_coarse, pack_key(0, own[0], own[1], own[2]));
        if (ci >= 0) b_in[ci] += 1;
        for (int64_t ax = lo[0]; ax <= hi[0]; ++ax)
            for (int64_t ay = lo[1]; ay <= hi[1]; ++ay)
                for (int64_t az = lo[2]; az <= hi[2]; ++az) {
                    if (ax == own[0] && ay == own[1] && az == own[2]) continue;
                    int64_t cj = find_key(ckeys, n_coarse, pack_key(0, ax, ay, az));
                    if (cj >= 0) b_out[cj] += 1;
                }
    }
    for (int64_t c = 0; c < n_coarse; ++c) {
        int l0 = level_of(ccount[c] - b_in[c], p->n_min, L);
        int l1 = level_of(ccount[c] + b_out[c], p->n_min, L);
        amb[c] = (l0 != l1);
        st->n_ambiguous_coarse += amb[c];
    }

    /* Sec. II.5(1)d-e: level per coarse cell, then each point's cell key */
    for (int64_t t = 0; t < n_pts; ++t) {
        const uint32_t g = items[t].g;
        int64_t ci = find_key(ckeys, n_coarse, items[t].key);
        int l = level_of(ccount[ci], p->n_min, L);
        int64_t k3[3];
        double margin = INFINITY;
        const double edge = ldexp(s0, -l);
        for (int k = 0; k < 3; ++k) {
            double f = ldexp(pw[3 * g + k] / s0, l);
            k3[k] = (int64_t)floor(f);
            double dist = fabs(f - nearbyint(f)) * edge;
            if (dist < margin) margin = dist;
        }
        uint64_t key = pack_key(l, k3[0], k3[1], k3[2]);
        pkey[g] = key;
        items[t].key = key;
        if (margin < p->band_m) { st->n_boundary_points += 1; flag[g] |= 8; }
        if (amb[ci]) flag[g] |= 16;
        if (pts && pts->level) pts->level[g] = l;
        if (pts && pts->margin_cell_m) pts->margin_cell_m[g] = margin;
    }
    if (pts) {
        for (int64_t g = 0; g < npx; ++g) {
            if (pts->key) pts->key[g] = pkey[g];
            if (pts->in_range) pts->in_range[g] = (flag[g] & 2) ? 1 : 0;
            if (pts->level && !(flag[g] & 2)) pts->level[g] = -1;
            if (pts->margin_cell_m && !(flag[g] & 2)) pts->margin_cell_m[g] = INFINITY;
        }
    }

    /* Cells: group members by key (members in ascending pixel order) */
    qsort(items, (size_t)n_pts, sizeof(sort_item), cmp_item);
    int64_t n_cells = 0;
    for (int64_t a = 0; a < n_pts;) {
        int64_t b = a;
        while (b < n_pts && items[b].key == items[a].key) ++b;
        ++n_cells;
        a = b;
    }
    st->n_cells = n_cells;
    int rc = ORC_OK;
    if (cells && n_cells > cell_capacity) rc = ORC_ERR_CAPACITY;
    if (cells && rc == ORC_OK) {
        rep_item *order = (rep_item *)malloc(sizeof(rep_item) * (size_t)(n_cells > 0 ? n_cells : 1));
        int64_t *start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_cells + 1));
        if (!order || !start) { free(order); free(start); rc = ORC_ERR_NOMEM; }
        else {
            int64_t c = 0;
            for (int64_t a = 0; a < n_pts;) {
                int64_t b = a;
                while (b < n_pts && items[b].key == items[a].key) ++b;
                start[c] = a;
                /* Sec. II.5(2)a: representative = largest C, ties to the lowest index */
                uint32_t rep = items[a].g;
                float best = conf_of(conf, off, n, rep);
                for (int64_t t = a + 1; t < b; ++t) {
                    const uint32_t g = items[t].g;
                    const float Cg = conf_of(conf, off, n, g);
                    if (Cg > best) { best = Cg; rep = g; }
                }
                order[c].rep = rep;
                order[c].cell = c;
                ++c;
                a = b;
            }
            start[n_cells] = n_pts;
            qsort(order, (size_t)n_cells, sizeof(rep_item), cmp_rep);
            uint32_t *fused = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n_pts > 0 ? n_pts : 1));
            for (int64_t o = 0; fused && o < n_cells; ++o) {
                const int64_t c0 = order[o].cell;
                const int64_t a = start[c0], b = start[c0 + 1];
                /* the members that enter Eq. 11: all of them, or (Sec. II.5(2)a) the top_k
                   by C, ties to the lowest pixel index, taken by repeated selection */
                int64_t nf = 0;
                if (p->top_k == 0 || b - a <= p->top_k) {
                    for (int64_t t = a; t < b; ++t) fused[nf++] = items[t].g;
                } else {
                    for (int k = 0; k < p->top_k; ++k) {
                        int64_t best = -1;
                        float bc = 0.0f;
                        for (int64_t t = a; t < b; ++t) {
                            const uint32_t g = items[t].g;
                            int taken = 0;
                            for (int64_t q = 0; q < nf; ++q) taken |= fused[q] == g;
                            if (taken) continue;
                            const float Cg = conf_of(conf, off, n, g);
                            if (best < 0 || Cg > bc || (Cg == bc && g < (uint32_t)best)) {
                                best = g;
                                bc = Cg;
                            }
                        }
                        fused[nf++] = (uint32_t)best;
                    }
                }
                double lmax = -INFINITY, W = 0.0;
                uint32_t fl = 0;
                for (int64_t t = a; t < b; ++t) {
                    uint32_t g = items[t].g;
                    if (flag[g] & 8) fl |= ORC_CELL_BOUNDARY;
                    if (flag[g] & 16) fl |= ORC_CELL_AMBIGUOUS_LEVEL;
                }
                for (int64_t q = 0; q < nf; ++q) {
                    const uint32_t g = fused[q];
                    if (lw[g] > lmax) lmax = lw[g];
                    W += om[g];
                    if (flag[g] & 4) fl |= ORC_CELL_TIE;
                }
                /* Eq. 11, normalised; weights scaled by the largest one */
                double sw = 0.0, sp[3] = {0, 0, 0}, sc[3] = {0, 0, 0};
                for (int64_t q = 0; q < nf; ++q) {
                    const uint32_t g = fused[q];
                    const int ci = camera_of(off, n, g);
                    const uint8_t *px = rgb[ci] + 3 * (g - off[ci]);
                    double w = exp(lw[g] - lmax);
                    sw += w;
                    for (int k = 0; k < 3; ++k) {
                        sp[k] += w * pw[3 * g + k];
                        sc[k] += w * (double)px[k];
                    }
                }
                if (cells->key) cells->key[o] = items[a].key;
                if (cells->count) cells->count[o] = (uint32_t)(b - a);
                if (cells->rep) cells->rep[o] = order[o].rep;
                if (cells->weight) cells->weight[o] = W;
                for (int k = 0; k < 3; ++k) {
                    if (cells->pos) cells->pos[3 * o + k] = sp[k] / sw;
                    if (cells->rgb) cells->rgb[3 * o + k] = sc[k] / sw;
                }
                if (cells->flags) cells->flags[o] = fl;
            }
            if (!fused) rc = ORC_ERR_NOMEM;
            free(fused);
            free(order);
            free(start);
        }
    }
    free(off); free(nbr); free(pw); free(lw); free(om); free(flag); free(items);
    free(ckeys); free(ccount); free(b_in); free(b_out); free(amb); free(pkey);
    return rc;
}

/* ---------------------------------------------------------------- Eq. 12 MC error */
int orc_mc_error(const orc_camera *cams, int32_t n, const orc_params *p,
                 const void *const *depth, const double *pts, int64_t n_pts,
                 double occlusion_m, double *err, int32_t *nvis, double *tie_px, double *mc_m,
                 int64_t *n_used) {
    if (!cams || n < 1 || !p || !depth || (n_pts > 0 && !pts) || !mc_m || !n_used)
        return ORC_ERR_ARG;
    double total = 0.0;
    int64_t used = 0;
    for (int64_t k = 0; k < n_pts; ++k) {
        const double *P = pts + 3 * k;
        double sum = 0.0, tie = INFINITY;
        int32_t vis = 0;
        for (int32_t i = 0; i < n; ++i) {
            const orc_camera *c = &cams[i];
            double a[3];
            to_camera(c, P, a);                       /* T_i P_k */
            if (!(a[2] > 0.0)) continue;              /* behind camera i */
            const double u = c->fx * a[0] / a[2] + c->cx;   /* pi(T_i P_k) */
            const double v = c->fy * a[1] / a[2] + c->cy;
            const double px = floor(u + 0.5), py = floor(v + 0.5);
            if (px >= -1.0 && py >= -1.0 && px <= c->width && py <= c->height) {
                /* the pixel decision matters here (inside the image or at its border) */
                const double fu = u + 0.5 - px, fv = v + 0.5 - py;
                const double tu = fu < 1.0 - fu ? fu : 1.0 - fu, tv = fv < 1.0 - fv ? fv : 1.0 - fv;
                if (tu < tie) tie = tu;
                if (tv < tie) tie = tv;
            }
            if (px < 0.0 || py < 0.0 || px >= c->width || py >= c->height) continue;
            double D;
            if (!depth_at(depth[i], p->depth_format, (int64_t)py * c->width + (int64_t)px,
                          p->depth_scale, &D))
                continue;                             /* no observed depth there */
            if (a[2] > D + occlusion_m) continue;     /* behind the observed surface: occluded */
            sum += fabs(a[2] - D);                    /* |z(T_i P_k) - D_i(pi(T_i P_k))| */
            ++vis;
        }
        const double e = vis ? sum / vis : NAN;
        if (err) err[k] = e;
        if (nvis) nvis[k] = vis;
        if (tie_px) tie_px[k] = tie;
        if (vis) {
            total += e;
            ++used;
        }
    }
    *mc_m = used ? total / (double)used : NAN;
    *n_used = used;
    return ORC_OK;
}

/* ---------------------------------------------------------------- Eq. 3 confidence */
int orc_confidence(const void *depth, int32_t w, int32_t h, const orc_params *p, double alpha,
                   double beta, double gamma, double delta, double *out) {
    if (!depth || w < 1 || h < 1 || !p || !out || !(alpha + gamma > 0.0)) return ORC_ERR_ARG;
    for (int32_t y = 0; y < h; ++y) {
        for (int32_t x = 0; x < w; ++x) {
            double z;
            if (!depth_at(depth, p->depth_format, (int64_t)y * w + x, p->depth_scale, &z)) {
                out[(int64_t)y * w + x] = 0.0;
                continue;
            }
            /* depth gradient G from central (or one-sided) differences */
            double g[2];
            for (int axis = 0; axis < 2; ++axis) {
                const int dx = axis == 0, dy = axis == 1;
                double zm = 0.0, zp = 0.0;
                const int xm = x - dx, ym = y - dy, xp = x + dx, yp = y + dy;
                const int vm = xm >= 0 && ym >= 0 &&
                               depth_at(depth, p->depth_format, (int64_t)ym * w + xm, p->depth_scale, &zm);
                const int vp = xp < w && yp < h &&
                               depth_at(depth, p->depth_format, (int64_t)yp * w + xp, p->depth_scale, &zp);
                if (vm && vp) g[axis] = (zp - zm) / 2.0;
                else if (vp) g[axis] = zp - z;
                else if (vm) g[axis] = z - zm;
                else g[axis] = 0.0;
            }
            const double G = sqrt(g[0] * g[0] + g[1] * g[1]);
            /* local variance of the valid depths of the 3x3 window (two passes) */
            double vals[9];
            int n = 0;
            for (int v = -1; v <= 1; ++v)
                for (int u = -1; u <= 1; ++u) {
                    const int xx = x + u, yy = y + v;
                    double zz;
                    if (xx < 0 || yy < 0 || xx >= w || yy >= h) continue;
                    if (depth_at(depth, p->depth_format, (int64_t)yy * w + xx, p->depth_scale, &zz))
                        vals[n++] = zz;
                }
            double mean = 0.0, var = 0.0;
            for (int k = 0; k < n; ++k) mean += vals[k];
            mean /= n;
            for (int k = 0; k < n; ++k) var += (vals[k] - mean) * (vals[k] - mean);
            var /= n;
            out[(int64_t)y * w + x] =
                (alpha / (1.0 + beta * G) + gamma / (1.0 + delta * var)) / (alpha + gamma);
        }
    }
    return ORC_OK;
}
