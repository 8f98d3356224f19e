/*
 * fuseflow.h - C ABI of the GB300 (sm_103a) FUSE-Flow per-frame fusion path.
 *
 * Method: "FUSE-Flow: Scalable Real-Time Multi-View Point Cloud Reconstruction Using
 * Confidence" (arXiv 2602.01035).  One call fuses the N RGB-D images of one time step
 * (problem statement, Sec. II.1, Eq. 1) into a point cloud with one fused point per
 * adaptive spatial-hash cell:
 *   (a) back-projection of every valid pixel and confidence gating (Eq. 8, Eq. 9),
 *   (b) joint weight = confidence x 3D distance consistency (Eq. 4-7, Eq. 10),
 *   (c) adaptive spatial hash: coarse density, level per coarse cell, cell keys
 *       (Sec. II.5(1) a-e),
 *   (d) one representative per cell (largest confidence, Sec. II.5(2)a) and the
 *       confidence-weighted fused position and colour of all members (Eq. 11).
 *
 * Conventions
 *   - Pixel (x, y) of camera i has its centre at integer coordinates; depth is z-depth.
 *   - Global pixel index g = off_i + y * W_i + x, off_i = sum_{k<i} W_k H_k.
 *   - Pose: x_cam = R x_world + t (camera-from-world T_i; Eq. 8 applies T_i^-1).
 *   - All image buffers are contiguous row-major, one buffer per camera.
 *   - Every entry point returns a fuseflow_status; nothing aborts or exits.
 *   - A context is not thread-safe: use one context per rig and per host thread.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 */
#ifndef FUSEFLOW_H
#define FUSEFLOW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FUSEFLOW_OK = 0,
    FUSEFLOW_ERR_INVALID_ARG = 1,   /* null pointer, bad size or parameter */
    FUSEFLOW_ERR_OUT_OF_MEMORY = 2, /* a device or host allocation failed */
    FUSEFLOW_ERR_CAPACITY = 3,      /* more cells than max_cells, or a hash table filled up */
    FUSEFLOW_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    FUSEFLOW_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    FUSEFLOW_ERR_INTERNAL = 6,      /* a device-side consistency check failed */
    FUSEFLOW_ERR_CANCELLED = 7      /* a served frame dropped before it started (rig removed) */
} fuseflow_status;

typedef enum {
    FUSEFLOW_DEPTH_U16 = 0,  /* uint16 depth units (e.g. millimetres), 0 = invalid */
    FUSEFLOW_DEPTH_F32 = 1   /* float32 depth units, invalid unless > 0 and finite */
} fuseflow_depth_format;

/* Pinhole intrinsics K_i (Sec. II.1; the paper names no distortion model). */
typedef struct {
    double fx, fy, cx, cy;
    int32_t width, height;
} fuseflow_intrinsics;

/* Extrinsic pose T_i, camera-from-world: x_cam = R x_world + t, R row-major, t metres. */
typedef struct {
    double R[9];
    double t[3];
} fuseflow_extrinsics;

/* Method parameters.  Start from fuseflow_default_params(). */
typedef struct {
    float tau;              /* Eq. 9 gate: a pixel is kept iff C > tau (float32 compare); 0.6 */
    int32_t k_views;        /* K of Eq. 7 counting camera i; effective K = min(k_views, N); 4 */
    double sigma_m;         /* sigma of Eq. 7 in metres (unspecified in the paper); 0.03 */
    double coarse_cell_m;   /* coarse grid edge s0 (Sec. II.5(1)c) in metres; 0.32 */
    int32_t max_level;      /* finest level Lmax, cell edge s0 / 2^Lmax; 4 (0 <= Lmax <= 14) */
    int32_t n_min;          /* level l needs n_c >= n_min * 4^l points in the coarse cell; 32 */
    int32_t depth_format;   /* fuseflow_depth_format */
    int32_t use_conf;       /* 0 = ablation "no measurement confidence": no gate, omega = V */
    double depth_scale;     /* metres per depth unit; 0.001 for millimetre uint16 */
    int32_t use_consistency;/* 0 = ablation "no distance consistency": V = 1 */
    int32_t top_k;          /* Sec. II.5(2)a: fuse only the top_k members of each cell by C
                               (ties to the lowest pixel index), with consistency computed
                               for those alone; 0 = every member (default); at most 7 */
    int64_t max_cells;      /* output capacity in cells; 0 = max(65536, pixels / 8) */
    /* Depth preprocessing D^r of Eq. 8 (the paper leaves the rule open, naming filtering and
     * screening as examples, so this one is stated here).  A screened-out pixel counts as
     * invalid everywhere: in the
     * back-projection and in the other views' consistency gathers of Eq. 5.  All three are
     * off by default (<= 0), and then D^r = D.  Decisions are taken in float32 on depth
     * units: bounds b_u = (float)(b_m / depth_scale); a valid depth d is kept iff
     * d >= min_u (when set) and d <= max_u (when set); then, with the edge screen on, d is
     * screened out iff one of its 4-neighbours inside the image, itself valid and within
     * the bounds, has fabsf(d - d') > (float)screen_edge_rel * d (flying pixels at depth
     * discontinuities).  Neighbours are judged on the range-screened image, once. */
    double screen_min_m;
    double screen_max_m;
    float screen_edge_rel;
    int32_t reserved1;      /* 0 */
} fuseflow_params;

/* Frame statistics; written on the device by fuseflow_fuse_frame. */
typedef struct {
    int64_t n_valid;        /* pixels with valid depth */
    int64_t n_gated;        /* pixels kept by the Eq. 9 gate */
    int64_t n_out_of_range; /* gated points whose finest cell index leaves [-2^19, 2^19) */
    int64_t n_cells;        /* cells of the fused cloud */
    float bbox[6];          /* min xyz, max xyz of the gated points (Sec. II.5(1)b), metres */
    int32_t error;          /* device error bits, 0 if none (see fuseflow_read_stats) */
    int32_t n_coarse;       /* occupied coarse cells */
} fuseflow_stats;

/* Fused cloud: device arrays owned by the context, valid until the next fuse call on the
 * same context or fuseflow_destroy.  Cells are ordered by representative pixel index,
 * ascending; only the first stats->n_cells entries are meaningful. */
typedef struct {
    fuseflow_stats *stats;  /* device pointer */
    float *pos;             /* [capacity][3] fused position (Eq. 11, normalised), metres */
    float *rgb;             /* [capacity][3] fused colour, 0..255 */
    float *weight;          /* [capacity] W = sum of the members' omega (Eq. 10) */
    uint32_t *count;        /* [capacity] members per cell */
    uint32_t *rep;          /* [capacity] representative's global pixel index */
    uint64_t *key;          /* [capacity] level << 60 | (kx+2^19) << 40 | (ky+2^19) << 20 | (kz+2^19) */
    int64_t capacity;       /* = max_cells */
} fuseflow_cloud;

/* Optional per-pixel trace of the last fused frame (caller-owned device arrays of
 * n_pixels entries; any pointer may be NULL).  Pixels that are not gated get
 * nview = -1, key = ~0 and NaN in the float arrays.  With top_k > 0 the weights of a
 * frame are computed for the cells' top-k members only, after the trace is written: gated
 * pixels get nview = -2 and omega, e are left untouched. */
typedef struct {
    float *pw;              /* [n][3] world point of Eq. 8, metres */
    float *omega;           /* Eq. 10 joint weight (may underflow to 0 in float32) */
    float *e;               /* exponent of Eq. 7, sum_j d_ij^2 / sigma^2 / (K-1) */
    int32_t *nview;         /* views that entered the sum of Eq. 7 */
    uint64_t *key;          /* cell key, ~0 if not gated or out of range */
} fuseflow_trace;

typedef struct fuseflow_ctx fuseflow_ctx;

/* Fills *p with the defaults listed above.  tau = 0.6 is Eq. 9's printed value. */
void fuseflow_default_params(fuseflow_params *p);

/* Creates a context for a rig of n_cams cameras (1 <= n_cams <= 64; K-1 <= 8).
 * Host arrays intr[n_cams], extr[n_cams] are copied; the context precomputes the
 * relative poses T_ji = T_j T_i^-1 of Eq. 4 in double precision, the static neighbour
 * table of Sec. II.5(2)b, and allocates its device tables on the current device.
 * Returns INVALID_ARG for bad sizes or parameters, OUT_OF_MEMORY, CUDA. */
int fuseflow_create(const fuseflow_intrinsics *intr, const fuseflow_extrinsics *extr,
                    int32_t n_cams, const fuseflow_params *params, fuseflow_ctx **out);

/* Releases every device and host resource of the context (NULL is a no-op). */
void fuseflow_destroy(fuseflow_ctx *ctx);

/* Fuses one frame (steps (a)-(d) above), asynchronously on `stream`.
 * depth[i], conf[i], rgb[i] are caller-owned DEVICE pointers to camera i's images
 * (depth: uint16 or float32 per params; conf: float32 in [0,1] (Eq. 2); rgb: uint8x3
 * interleaved), valid until the stream reaches the end of this call's work.
 * *out receives the context-owned output arrays.  Capacity overflows and device-side
 * failures are reported by the next fuseflow_read_stats.  Returns INVALID_ARG, CUDA. */
int fuseflow_fuse_frame(fuseflow_ctx *ctx, const void *const *depth, const float *const *conf,
                        const uint8_t *const *rgb, fuseflow_cloud *out, void *stream);

/* A fuse call recorded once as a CUDA graph, for callers whose input images live in the
 * same device buffers every frame (a capture loop that refills them): replaying it with
 * fuseflow_graph_launch is the same as calling fuseflow_fuse_frame with the pointers
 * given here, whose contents may change between launches, at one launch instead of seven
 * (eight with a depth screen set).
 * The graph keeps the context's launch geometry and trace registration as they were at
 * creation; results do not depend on the geometry.  It uses the context's tables, so
 * launches of graphs and fuse calls of one context must be ordered (one stream), and
 * every graph must be destroyed before its context.  create runs no GPU work (it records
 * on a private stream of its own); it returns INVALID_ARG or CUDA. */
typedef struct fuseflow_graph fuseflow_graph;
int fuseflow_graph_create(fuseflow_ctx *ctx, const void *const *depth, const float *const *conf,
                          const uint8_t *const *rgb, fuseflow_graph **out);
/* Enqueues the recorded frame on `stream`; *out (may be NULL) as for fuseflow_fuse_frame. */
int fuseflow_graph_launch(fuseflow_graph *graph, fuseflow_cloud *out, void *stream);
void fuseflow_graph_destroy(fuseflow_graph *graph);

/* The context's output arrays (device pointers, as fuseflow_fuse_frame returns them); they
 * hold the last frame fused on the context once the stream has reached that call. */
int fuseflow_get_cloud(const fuseflow_ctx *ctx, fuseflow_cloud *out);

/* Batched fusion (engineering entry points; frames are independent, Sec. I and II.1, so
 * fusing several at once changes no result).  A batch holds up to FUSEFLOW_MAX_BATCH
 * contexts (frames of one rig in several contexts, or of different rigs with any camera
 * counts and resolutions) that share the depth format and top_k and have no depth screen
 * set.  fuseflow_batch_fuse fuses one frame per context with every frame kernel launched
 * ONCE for all of them: the frames' blocks share each grid (count and assign grids
 * concatenate the frames' blocks; the others take the frame from the grid's second
 * dimension), so short kernels run once per batch and frames fill each other's tails.
 * depth[i], conf[i], rgb[i] are context i's per-camera device images (as for
 * fuseflow_fuse_frame); each context's cloud and statistics are then read with its usual
 * calls (fuseflow_get_cloud, fuseflow_read_stats) and are bitwise those of
 * fuseflow_fuse_frame on that context.  The contexts must not be used elsewhere while a
 * batch call runs; the batch holds pointers to them and does not own them.
 * fuseflow_batch_graph_create records one batch call on fixed input buffers as a CUDA
 * graph (replayed with fuseflow_graph_launch, whose cloud argument receives context 0's).
 * The contexts' tile heights (fuseflow_tuning.tile_h) must agree when a batch call is
 * made or recorded: one assign kernel serves the whole batch.
 * Returns INVALID_ARG (count, mixed formats or variants, a screen, a repeated context,
 * NULL pointers, tile heights that differ at call time), OUT_OF_MEMORY, CUDA. */
#define FUSEFLOW_MAX_BATCH 8
typedef struct fuseflow_batch fuseflow_batch;
int fuseflow_batch_create(fuseflow_ctx *const *ctxs, int32_t n, fuseflow_batch **out);
int fuseflow_batch_fuse(fuseflow_batch *batch, const void *const *const *depth,
                        const float *const *const *conf, const uint8_t *const *const *rgb,
                        void *stream);
int fuseflow_batch_graph_create(fuseflow_batch *batch, const void *const *const *depth,
                                const float *const *const *conf, const uint8_t *const *const *rgb,
                                fuseflow_graph **out);
void fuseflow_batch_destroy(fuseflow_batch *batch);

/* Point-wise fusion, the "No SA" ablation of Table II (fusion without the spatial hash,
 * Sec. IV ablations): every gated pixel of the frame is an output point with its own joint
 * weight omega = C V of Eq. 10, its consistency V computed over the camera's K-1 views
 * exactly as in fuseflow_fuse_frame (Eq. 4-8).  Outputs are caller-owned DEVICE arrays
 * indexed by the global pixel index g (n_pixels entries): pos[g][3] in metres (NaN when
 * the pixel is not gated), weight[g] (0 when not gated; may underflow to 0 in float32),
 * rgb_out[g][3] the pixel's 8-bit colour.  n_valid and n_gated (either may be NULL)
 * receive the frame's counts, which synchronizes `stream`; with both NULL the call is
 * asynchronous.  A context with a depth screen set is refused (INVALID_ARG). */
int fuseflow_fuse_points(fuseflow_ctx *ctx, const void *const *depth, const float *const *conf,
                         const uint8_t *const *rgb, float *pos, float *weight, uint8_t *rgb_out,
                         int64_t *n_valid, int64_t *n_gated, void *stream);

/* Waits for `stream`, copies the last frame's statistics to *host_stats and returns
 * CAPACITY if the frame overflowed max_cells or a hash table, INTERNAL if a device-side
 * check failed, OK otherwise. */
int fuseflow_read_stats(fuseflow_ctx *ctx, fuseflow_stats *host_stats, void *stream);

/* End-to-end variant on HOST buffers: copies the images host-to-device (pinned memory
 * gives asynchronous copies), fuses, waits, and copies the first n_cells cells into the
 * caller's host arrays (each sized for max_cells; any may be NULL).  Synchronous.
 * Returns the status of fuseflow_read_stats. */
int fuseflow_fuse_frame_host(fuseflow_ctx *ctx, const void *const *depth,
                             const float *const *conf, const uint8_t *const *rgb,
                             float *pos, float *rgb_out, float *weight, uint32_t *count,
                             uint32_t *rep, uint64_t *key, fuseflow_stats *host_stats,
                             void *stream);

/* Multi-Camera Depth Consistency error of Eq. 12 on a point set, against the rig's depth
 * maps of one frame: for each point P_k (pos: DEVICE float32 [n_points][3], world metres),
 * the cameras i that see it (z(T_i P_k) > 0, nearest pixel floor(pi(T_i P_k) + 1/2) inside
 * the image, valid D_i there, and not hidden behind the observed surface:
 * z(T_i P_k) <= D_i + occlusion_m; INFINITY disables that test) and the mean over them of
 * |z(T_i P_k) - D_i(pi(T_i P_k))|.  occlusion_m >= 0 (metres).  err_m (DEVICE float [n], metres, NaN where no camera
 * sees the point) and n_visible (DEVICE int32 [n]) may be NULL.  *mc_m receives E_MC, the
 * mean of the per-point errors over the points seen by at least one camera (metres), and
 * *n_used their number.  depth[i] are DEVICE pointers as for fuseflow_fuse_frame.  Waits
 * for `stream` before returning.  Returns INVALID_ARG, OUT_OF_MEMORY, CUDA. */
int fuseflow_mc_error(fuseflow_ctx *ctx, const float *pos, int64_t n_points,
                      const void *const *depth, double occlusion_m, float *err_m,
                      int32_t *n_visible, double *mc_m, int64_t *n_used, void *stream);

/* Weights of the confidence model of Eq. 3. */
typedef struct {
    double alpha, beta, gamma, delta;
} fuseflow_conf_params;

/* The screened depth D^r of Eq. 8 under the context's screen parameters (fuseflow_params),
 * for callers that want it outside a fuse call (e.g. to feed fuseflow_confidence): for every
 * camera i, reads depth_in[i] and writes depth_out[i] (DEVICE, the context's depth format,
 * [H_i][W_i]; the two must not overlap), screened-out and invalid samples as 0.  Every
 * fuse call of a context with a screen set applies the same step itself, into a scratch
 * buffer of the context.  Asynchronous on `stream`.  Returns INVALID_ARG, CUDA. */
int fuseflow_screen_depth(fuseflow_ctx *ctx, const void *const *depth_in, void *const *depth_out,
                          void *stream);

/* Eq. 3's printed constants: alpha = beta = 0.5, gamma = delta = 1. */
void fuseflow_default_conf_params(fuseflow_conf_params *cp);

/* Measurement confidence of Eq. 3 for callers without a confidence image: for every
 * camera i, reads depth[i] (DEVICE, the context's depth format) and writes conf_out[i]
 * (DEVICE float32 [H_i][W_i]).  Readings: depths in metres; G = |(g_x, g_y)| with g the
 * central difference (z(x+1) - z(x-1)) / 2 where both neighbours are valid, the one-sided
 * difference where one is, 0 where none is; sigma_local = the population variance (m^2)
 * of the valid depths in the 3x3 window; C = (alpha / (1 + beta G) + gamma / (1 + delta
 * sigma_local)) / (alpha + gamma), so that C stays in [0, 1] as Eq. 2 requires; C = 0 where
 * the depth is invalid.  cp NULL selects the printed constants.  Asynchronous on `stream`.
 * Returns INVALID_ARG, CUDA. */
int fuseflow_confidence(fuseflow_ctx *ctx, const void *const *depth, float *const *conf_out,
                        const fuseflow_conf_params *cp, void *stream);

/* Registers (or, with NULL, clears) a per-pixel trace written by later fuse calls. */
int fuseflow_set_trace(fuseflow_ctx *ctx, const fuseflow_trace *trace);

/* Copies the static neighbour table (n_cams rows of K-1 camera indices) to host `out`
 * (n_cams * (K-1) entries) and K-1 to *k_minus_1. */
int fuseflow_get_neighbours(const fuseflow_ctx *ctx, int32_t *out, int32_t *k_minus_1);

/* Per-stage device timing for profiling.  While enabled, every fuse call records CUDA
 * events between its stages on its own stream (a ring of the last 1024 frames).
 * fuseflow_read_stage_times waits for the last recorded event, writes the summed
 * milliseconds of each of the FUSEFLOW_N_STAGES stages to ms[] and the number of frames
 * to *n_frames, then resets the ring.  Stages: 0 clear (and the depth screen when one is
 * set), 1 count (a, c2), 2 assign (b, c, d per tile), 3 reduce (d per cell), 4 scan,
 * 5 emit. */
#define FUSEFLOW_N_STAGES 6
int fuseflow_enable_stage_timing(fuseflow_ctx *ctx, int enable);
int fuseflow_read_stage_times(fuseflow_ctx *ctx, double *ms, int64_t *n_frames);
const char *fuseflow_stage_name(int stage);

/* Launch geometry of a context: performance knobs only.  The fused cloud, its statistics
 * and any trace are bitwise the same for every admissible setting of the first four (the
 * path has no order-dependent arithmetic); tile_h changes how each cell's members are
 * grouped into per-tile fixed-point partial sums, so keys, counts, representatives, the
 * trace and the statistics stay bitwise the same while weights, positions and colours
 * may move in their last bits (far inside the 1e-5 relative tolerance: each partial is
 * exact at a scale of 2^-36 of the largest weight in its tile, and shifting it to the
 * cell's scale truncates below that).  A setting can be chosen by timing alone.
 *   count_chunks    2048-pixel chunks per block of the coarse-count step, 1..64
 *   emit_blocks     blocks of the level, reduce and emit steps, 1..65536
 *   prefetch_tiles  how many assign tiles ahead each assign block prefetches its
 *                   depth rows into L2; 0 turns the prefetch off
 *   programmatic    2: each kernel of a frame after the first is launched with
 *                   programmatic stream serialization, so that its blocks start while the
 *                   previous kernel's last blocks finish (they wait for its results on the
 *                   device); 1: the same except between the assign and reduce steps (early
 *                   reduce blocks slow the assign step's last wave on large frames); 0:
 *                   plain stream order.  Stage timing always uses plain order.
 *   tile_h          rows of the assign step's tiles of 32 columns: 8 (128 threads a
 *                   block), 16 (256) or 32 (512); 0 in fuseflow_set_tuning keeps the
 *                   current height
 * fuseflow_create picks count_chunks for one wave of four count blocks per SM (at most 6),
 * emit_blocks = 8 blocks per SM, prefetch_tiles = one wave of assign blocks,
 * programmatic = 2 for rigs of fewer than 2^21 pixels, 1 otherwise, and tile_h = 16. */
typedef struct fuseflow_tuning {
  int32_t count_chunks;
  int32_t emit_blocks;
  int32_t prefetch_tiles;
  int32_t programmatic;       /* 0, 1 or 2 */
  int32_t tile_h;             /* 8, 16 or 32 (0: keep, in set) */
} fuseflow_tuning;

/* Reads (get) or replaces (set) the context's launch geometry.  set returns INVALID_ARG,
 * leaving the context unchanged, for a value outside the ranges above.  Neither touches
 * the GPU; set must not race with a fuse call of the same context still being enqueued
 * from another host thread. */
int fuseflow_get_tuning(const fuseflow_ctx *ctx, fuseflow_tuning *out);
int fuseflow_set_tuning(fuseflow_ctx *ctx, const fuseflow_tuning *in);

/* Autotuner of the launch geometry.  Fuses the given frame (DEVICE inputs as for
 * fuseflow_fuse_frame) repeatedly on `stream` under candidate settings, one knob at a
 * time (tile_h, count_chunks, emit_blocks, prefetch_tiles, then programmatic; coordinate
 * descent from the context's current setting), and keeps a candidate only when the median of `reps`
 * timed frames (CUDA events on `stream`, L2 flushed before each frame by writing a
 * scratch buffer of twice the L2 size) is at least 1 % below the best so far.  The
 * chosen setting stays in the context and is copied to *chosen (may be NULL);
 * frame_us[0] and frame_us[1] (may be NULL) receive the median frame time, in
 * microseconds, of the starting and of the chosen setting, both measured at the end.
 * Any trace registered with fuseflow_set_trace is suspended while tuning.  Synchronous:
 * returns after `stream` is idle; the context's outputs then hold the frame's cloud.
 * reps in 3..101.  Returns INVALID_ARG, OUT_OF_MEMORY (scratch), CUDA. */
int fuseflow_autotune(fuseflow_ctx *ctx, const void *const *depth, const float *const *conf,
                      const uint8_t *const *rgb, int32_t reps, fuseflow_tuning *chosen,
                      double *frame_us, void *stream);

/* Number of pixels of the rig (sum of W_i H_i) and the output capacity. */
int64_t fuseflow_num_pixels(const fuseflow_ctx *ctx);
int64_t fuseflow_capacity(const fuseflow_ctx *ctx);

/* Device bytes held by the context (tables, scratch and outputs). */
int64_t fuseflow_device_bytes(const fuseflow_ctx *ctx);

/* Allocation-free variant of fuseflow_fuse_frame (the paper has no counterpart; it is
 * an engineering entry point).  Some callers cannot allocate device memory while they
 * run: a host application that hands the whole GPU memory budget to its own pool up
 * front, a real-time capture loop in which cudaMalloc's implicit device-wide
 * synchronisation and unbounded latency are not acceptable, or a plug-in that must not
 * change the process's memory footprint after start-up.  This call needs no context: it
 * takes the rig and parameters directly, calls no cudaMalloc, cudaFree or other
 * allocating routine (device or host), and keeps all of its scratch in one file-scope
 * device array of about 23 MiB that every GPU loading this library holds until exit.
 *
 * Limits: at most 524,288 pixels per frame over all cameras, at most 65,536 ray-table
 * entries (sum over cameras of width + height), 2 (K - 1) times that at most 393,216
 * (K = min(k_views, n_cams)), and max_cells <= 32,768 (0 selects 32,768); larger
 * requests return FUSEFLOW_ERR_CAPACITY before anything is sent to the GPU.  A
 * frame that produces more than 131,072 (tile, cell) partial records reports a capacity
 * error in stats->error.
 * Inputs are device pointers as for fuseflow_fuse_frame; pos[3*max_cells],
 * rgb_out[3*max_cells], weight, count, rep, key[max_cells] and *stats are caller-owned
 * DEVICE outputs with the layout of fuseflow_cloud and fuseflow_stats.  Asynchronous on
 * `stream`; errors found on the device appear in stats->error (bits as read by
 * fuseflow_read_stats).
 *
 * The first call on each device looks the array's device address up with
 * cudaGetSymbolAddress, empties its hash tables and synchronizes `stream`; make that
 * first call before any stream capture.  Every later call reuses the array as the last
 * call left it (each frame empties the tables it used again, also after a frame that
 * reported a capacity error).  Calls whose GPU work overlaps, on several streams or from
 * several host threads, race on the array: keep them ordered on one stream.  The call
 * stages the rig constants through host arrays that the next call overwrites, so it must
 * not be recorded into a CUDA graph: on a capturing stream it returns
 * FUSEFLOW_ERR_INVALID_ARG and does nothing. */
int fuseflow_fuse_frame_static(const fuseflow_intrinsics *intr, const fuseflow_extrinsics *extr,
                               int32_t n_cams, const fuseflow_params *params,
                               const void *const *depth, const float *const *conf,
                               const uint8_t *const *rgb, float *pos, float *rgb_out,
                               float *weight, uint32_t *count, uint32_t *rep, uint64_t *key,
                               fuseflow_stats *stats, void *stream);

/* ------------------------------------------------------------------------------------
 * Serving: several rigs, frames arriving from host memory, continuous batching.
 *
 * The paper fuses the frames of one rig as a real-time stream (Sec. I, Sec. II.1); a
 * server here keeps several rigs resident on one GPU and overlaps their frames.  Each
 * rig has up to n_slots frame slots, each with its own device tables, input staging
 * buffers and stream, allocated against an HBM budget as frames need them (see
 * fuseflow_server_add_rig).  A submitted frame starts at once when one of its rig's slots
 * is free or a new one fits in the budget, otherwise it waits and starts as soon as
 * fuseflow_server_poll finds a slot of its rig finished (among the waiting frames whose
 * rig can take one, the one submitted first starts first), so the copies and kernels of
 * frames of different rigs and slots overlap on the device.
 * Results do not depend on the mix: every frame runs the same kernels on its own tables.
 * Each slot has a stream of its own: with many slots, set CUDA_DEVICE_MAX_CONNECTIONS=32
 * in the environment before the process initialises CUDA, since streams that share one
 * of the default 8 hardware work queues run one after the other.
 * Not thread-safe: drive one server from one host thread.
 * ------------------------------------------------------------------------------------ */
typedef struct fuseflow_server fuseflow_server;

/* Caller-owned HOST output arrays for one frame (pinned memory, e.g. cudaHostAlloc;
 * each sized for `capacity` cells; any array pointer may be NULL).  The first n_cells
 * cells are written, in the order of fuseflow_cloud, before the frame completes. */
typedef struct {
    float *pos;             /* [capacity][3] */
    float *rgb;             /* [capacity][3] */
    float *weight;          /* [capacity] */
    uint32_t *count;        /* [capacity] */
    uint32_t *rep;          /* [capacity] */
    uint64_t *key;          /* [capacity] */
    int64_t capacity;
} fuseflow_host_cloud;

/* Counters of a server (fuseflow_server_get_stats). */
typedef struct {
    int64_t budget_bytes;           /* the HBM budget */
    int64_t used_bytes;             /* device bytes held by the slots */
    int32_t rigs;                   /* resident rigs */
    int32_t slots;                  /* frame slots allocated over all rigs */
    int32_t inflight;               /* frames on the device */
    int32_t waiting;                /* frames submitted and not started */
    int64_t frames_submitted;
    int64_t frames_completed;       /* reported by poll after running on a slot */
    int64_t frames_failed;          /* reported by poll with the status of a failed start */
    int64_t frames_cancelled;       /* reported by poll with CANCELLED (their rig was removed) */
    int64_t deferred_by_budget;     /* frames that found every slot of their rig busy while the
                                       rig held fewer slots than it asked for, and waited */
    int64_t slots_grown;            /* slots allocated (including each rig's first) */
} fuseflow_server_stats;

/* One finished frame, reported by fuseflow_server_poll. */
typedef struct {
    int64_t request;        /* id returned by fuseflow_server_submit */
    int32_t rig;            /* rig id */
    int32_t status;         /* as fuseflow_read_stats; CAPACITY also if n_cells > capacity */
    fuseflow_stats stats;
} fuseflow_completion;

/* Creates a server on the current device that may hold at most hbm_budget_bytes of
 * device memory for its rigs' slots (> 0).  Returns INVALID_ARG, OUT_OF_MEMORY. */
int fuseflow_server_create(int64_t hbm_budget_bytes, fuseflow_server **out);

/* Adds a rig (as fuseflow_create) that asks for up to n_slots >= 1 frames in flight;
 * *rig_id receives its id.  A slot is one frame's device working set (a context with its
 * tables and outputs, and a staging buffer for the frame's images).  The rig's first slot
 * is allocated now and kept while the rig is resident (its camera constants and hash
 * tables stay on the device); fuseflow_server_reserve allocates more, as far as the budget
 * allows, and a rig removal gives the freed memory to the rigs below their request, one
 * slot per rig in turn.  Slots are never allocated while frames are served (an allocation
 * synchronizes the device): a frame that finds every slot of its rig busy waits, and is
 * counted as deferred by the budget when the rig holds fewer slots than it asked for.
 * With n_slots > 1 the frames of the rig run with programmatic = 0 (fuseflow_tuning):
 * the slots' overlapping streams fill the kernel boundaries, and blocks waiting for an
 * earlier kernel would only hold back the other slots' work.
 * Returns CAPACITY, with nothing allocated, if one slot does not fit in the budget. */
int fuseflow_server_add_rig(fuseflow_server *srv, const fuseflow_intrinsics *intr,
                            const fuseflow_extrinsics *extr, int32_t n_cams,
                            const fuseflow_params *params, int32_t n_slots, int32_t *rig_id);

/* Allocates slots of rig `rig` until it holds min(n_slots, its request) or the next one
 * does not fit in the budget; *n_held (may be NULL) receives the slots it holds.  Calling
 * it for every rig with n_slots = 2, 3, ... in turn shares a binding budget evenly.
 * Returns INVALID_ARG (unknown or removed rig), OUT_OF_MEMORY, CUDA; a budget that stops
 * the growth is not an error. */
int fuseflow_server_reserve(fuseflow_server *srv, int32_t rig, int32_t n_slots, int32_t *n_held);

/* Removes rig `rig`: its frames on the device are waited for and reported by the next
 * fuseflow_server_poll with their own status, its waiting frames are reported there with
 * FUSEFLOW_ERR_CANCELLED (their host buffers are free at once), its slots are released
 * and the memory returns to the budget, where the rigs holding fewer slots than they asked
 * for take it one slot per rig in turn (their waiting frames may then start).  The id is
 * not reused; later calls naming it return INVALID_ARG.  Synchronous for that rig's frames. */
int fuseflow_server_remove_rig(fuseflow_server *srv, int32_t rig);

/* Submits one frame of rig `rig`: depth[i], conf[i], rgb[i] are HOST pointers (pinned
 * for asynchronous copies) and *out the host output arrays (pinned: the copy-out kernel
 * writes them through their mapped addresses); all stay valid and untouched until the
 * frame is reported complete.  On systems where the GPU reaches pageable host memory
 * directly (Grace-based nodes) the server cannot tell pinned memory from any other host
 * address, so the arrays must be valid host memory of the stated size: an invalid address
 * is written by the device there.  Never blocks on the device.  *request receives the frame's
 * id; every accepted frame is reported exactly once by fuseflow_server_poll.  Returns
 * INVALID_ARG (the frame is then not accepted). */
int fuseflow_server_submit(fuseflow_server *srv, int32_t rig, const void *const *depth,
                           const float *const *conf, const uint8_t *const *rgb,
                           const fuseflow_host_cloud *out, int64_t *request);

/* Non-blocking: reports up to max_done finished frames in done[], their number in
 * *n_done, and starts waiting frames on the slots that became free.  A frame whose start
 * failed (host output arrays that are not pinned, a CUDA error) is reported with that
 * status, and only once every copy already queued from its host buffers has finished, so
 * that the caller may reuse them; frames of a removed rig are reported as described for
 * fuseflow_server_remove_rig.  Returns INVALID_ARG for bad arguments, else OK. */
int fuseflow_server_poll(fuseflow_server *srv, fuseflow_completion *done, int32_t max_done,
                         int32_t *n_done);

/* Caps the frames on the device at once over all rigs (0, the default: every free slot
 * takes a frame).  Waiting frames start in submission order across rigs, each as soon as
 * a slot of its rig is free and the cap allows; a lower cap gives each frame more of the
 * GPU and shortens the latency tail when many frames arrive together, at some loss of
 * overlap.  Returns INVALID_ARG for a negative cap, else OK. */
int fuseflow_server_set_max_inflight(fuseflow_server *srv, int32_t max_inflight);

/* Testing hook for the server's error paths (made on the host; no GPU fault is involved):
 * the next n frame starts fail with `status` (not OK), either before anything is queued
 * (after_copies = 0) or after the frame's image copies were queued (after_copies = 1; the
 * frame is then reported once those copies have finished).  n = 0 clears it.  Returns
 * INVALID_ARG for bad arguments. */
int fuseflow_server_inject_start_failure(fuseflow_server *srv, int32_t n, int32_t status,
                                         int32_t after_copies);

/* The server's counters (memory, slots, frames and deferrals). */
int fuseflow_server_get_stats(const fuseflow_server *srv, fuseflow_server_stats *out);

/* Frames submitted but not yet reported by fuseflow_server_poll. */
int64_t fuseflow_server_pending(const fuseflow_server *srv);

/* Autotunes the launch geometry of rig `rig` (fuseflow_autotune on the context of its
 * first slot, with one sample frame given as HOST pointers as for submit) and applies the
 * chosen setting to all of the rig's slots (programmatic = 0 with several slots, as in
 * fuseflow_server_add_rig).  The rig must be idle: INVALID_ARG while any
 * of its frames is in flight or waiting.  Synchronous.  *chosen and frame_us as for
 * fuseflow_autotune (either may be NULL). */
int fuseflow_server_autotune(fuseflow_server *srv, int32_t rig, const void *const *depth,
                             const float *const *conf, const uint8_t *const *rgb,
                             int32_t reps, fuseflow_tuning *chosen, double *frame_us);

/* Device bytes held by the server's slots (<= the budget). */
int64_t fuseflow_server_device_bytes(const fuseflow_server *srv);

/* Waits for every slot's stream and releases all resources (NULL is a no-op). */
void fuseflow_server_destroy(fuseflow_server *srv);

/* Static description of a status code. */
const char *fuseflow_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* FUSEFLOW_H */
