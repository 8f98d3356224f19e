/*
 * FP64 CPU oracle for the FUSE-Flow per-frame fusion path (arXiv 2602.01035).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code, header,
 * table or constant with the CUDA path and must never be used as a fallback for it.
 *
 * Every quantity is computed in double precision, step by step in the order of the
 * paper: Eq. 8 back-projection, Eq. 9 gating, Eq. 4-7 distance consistency, Eq. 10
 * joint weight, Sec. II.5(1) adaptive partition, Sec. II.5(2)a representative,
 * Eq. 11 weighted fusion.  The readings taken where the paper is silent are listed
 * at each function in fuseflow_oracle.c.
 */
#ifndef FUSEFLOW_ORACLE_H
#define FUSEFLOW_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_DEPTH_U16 = 0, ORC_DEPTH_F32 = 1, ORC_DEPTH_F64 = 2 };

/* Pinhole intrinsics K_i and camera-from-world pose T_i (x_cam = R x_world + t). */
typedef struct {
    double fx, fy, cx, cy;
    int32_t width, height;
    double R[9]; /* row-major */
    double t[3];
} orc_camera;

typedef struct {
    float tau;             /* Eq. 9 threshold, compared in float32 */
    int32_t k_views;       /* K of Eq. 7, counting camera i itself */
    double sigma_m;        /* sigma of Eq. 7, metres */
    double coarse_cell_m;  /* edge of the coarse grid cell, metres */
    int32_t max_level;     /* finest refinement level */
    int32_t n_min;         /* density threshold of level 0 */
    int32_t depth_format;  /* ORC_DEPTH_* */
    int32_t use_conf;      /* 0: no measurement confidence (no gate, omega = V) */
    double depth_scale;    /* metres per depth unit */
    int32_t use_consistency; /* 0: V = 1 */
    int32_t row_step;      /* process rows y % row_step == 0 only (timing samples); 1 = all */
    double band_m;         /* report points within band_m of a cell boundary */
    double band_px;        /* report projections within band_px of a half-pixel tie */
    double band_az;        /* report projections with |a_z| below band_az metres */
    int32_t top_k;         /* Sec. II.5(2)a: fuse only the top_k members of a cell by C
                              (ties to the lowest pixel index); 0 = every member */
    double screen_min_m;   /* D^r of Eq. 8 (see orc_screen_depth); <= 0: no lower bound */
    double screen_max_m;   /* <= 0: no upper bound */
    float screen_edge_rel; /* <= 0: no edge screen */
} orc_params;

/* Per-pixel outputs, arrays of n_pixels entries in global pixel order
 * g = off_i + y * W_i + x.  Any pointer may be NULL. */
typedef struct {
    uint8_t *valid, *gated, *in_range;
    double *pw;           /* [n][3] world point P_i(x, y), metres (gated pixels) */
    double *e;            /* exponent of Eq. 7: sum_j d_ij^2 / sigma^2 / (K-1) */
    double *omega;        /* Eq. 10 */
    double *log_omega;    /* ln(omega), finite even when omega underflows */
    int32_t *nview;       /* number of views entering the sum of Eq. 7 */
    uint64_t *key;        /* cell key, ~0 if not gated or out of range */
    int32_t *level;       /* refinement level of the point's coarse cell, -1 if none */
    double *margin_cell_m;/* distance to the nearest boundary of the point's cell, metres */
    double *margin_tie_px;/* min over views of the distance of u+1/2, v+1/2 to an integer */
    double *min_az;       /* min over views of |a_z| (metres) */
} orc_points;

/* Per-cell outputs ordered by representative pixel index, ascending. */
typedef struct {
    uint64_t *key;
    uint32_t *count, *rep;
    double *weight;       /* W = sum of member omegas */
    double *pos;          /* [n][3] fused position, metres */
    double *rgb;          /* [n][3] fused colour, 0..255 */
    uint32_t *flags;      /* ORC_CELL_* */
} orc_cells;

enum { ORC_CELL_BOUNDARY = 1, ORC_CELL_AMBIGUOUS_LEVEL = 2, ORC_CELL_TIE = 4 };

typedef struct {
    int64_t n_valid, n_gated, n_out_of_range, n_cells;
    double bbox[6];        /* min xyz, max xyz over gated points; +inf/-inf if none */
    int64_t n_boundary_points, n_tie_points, n_ambiguous_coarse, n_coarse;
} orc_stats;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NOMEM = 2, ORC_ERR_CAPACITY = 3 };

void orc_default_params(orc_params *p);

/* Static neighbour table: for each camera the K-1 other cameras used in Eq. 7. */
int orc_neighbours(const orc_camera *cams, int32_t n_cams, int32_t k_views, int32_t *out);

/* D^r of Eq. 8: the depth after a preprocessing step that the paper leaves open (its
 * examples are filtering and screening).  The
 * paper states no rule; the one read here: in depth units, with every comparison in
 * float32 (the same decision the GPU takes), bounds b_u = (float)(b_m / depth_scale);
 * a valid sample d (> 0, finite) is kept iff d >= min_u (bound set) and d <= max_u (bound
 * set); a kept sample is then screened out iff one of its 4-neighbours inside the image
 * is valid, within the bounds, and fabsf(d - d') > (float)screen_edge_rel * d.  Screened
 * and invalid samples are written as 0 in the input's format.  orc_fuse_frame applies it
 * to every camera first when any of the three settings is > 0, and uses D^r for both the
 * back-projection and the consistency gathers. */
int orc_screen_depth(const orc_params *p, int32_t w, int32_t h, const void *in, void *out);

int orc_fuse_frame(const orc_camera *cams, int32_t n_cams, const orc_params *p,
                   const void *const *depth, const float *const *conf,
                   const uint8_t *const *rgb, orc_points *pts, orc_cells *cells,
                   int64_t cell_capacity, orc_stats *st);

/* Eq. 12, the Multi-Camera Depth Consistency (MC) error of a point set rho = pts[n_pts][3]
 * (world frame, metres).  Reading of "visible": camera i is in gamma(P) when P lies in
 * front of it (z(T_i P) > 0), the nearest pixel floor(pi(T_i P) + 1/2) is inside the image,
 * D_i there is valid (> 0, finite) and P is not hidden behind the surface camera i
 * observes: z(T_i P) <= D_i + occlusion_m (INFINITY: no occlusion test).
 * Points visible in no camera are left out of the outer mean.  Per point (any pointer may
 * be NULL): err[k] = mean over gamma of |z(T_i P_k) - D_i(pixel)| in metres (NaN when gamma
 * is empty), nvis[k] = |gamma(P_k)|, tie_px[k] = smallest distance of u + 1/2 or v + 1/2
 * to an integer over the cameras in front of which P_k projects into the image or onto its
 * one-pixel border (where the rounding decides).  *mc_m = the mean of err over the points used and
 * *n_used their number.  Uses p->depth_format and p->depth_scale only. */
int orc_mc_error(const orc_camera *cams, int32_t n_cams, const orc_params *p,
                 const void *const *depth, const double *pts, int64_t n_pts,
                 double occlusion_m, double *err, int32_t *nvis, double *tie_px,
                 double *mc_m, int64_t *n_used);

/* Eq. 3 confidence of one depth image (w x h, depth format and scale of p), written to
 * out[h][w] (double).  Readings: depths in metres; G = |(g_x, g_y)|, g_x the central
 * difference (z(x+1) - z(x-1)) / 2 when both neighbours are valid, the one-sided
 * difference with the valid one otherwise, 0 with neither (same for g_y); sigma_local = the
 * population variance (m^2) of the valid depths of the 3x3 window; C = (alpha / (1 + beta G)
 * + gamma / (1 + delta sigma_local)) / (alpha + gamma), which keeps C in [0, 1] (Eq. 2);
 * C = 0 where the depth itself is invalid. */
int orc_confidence(const void *depth, int32_t w, int32_t h, const orc_params *p, double alpha,
                   double beta, double gamma, double delta, double *out);

#ifdef __cplusplus
}
#endif
#endif
