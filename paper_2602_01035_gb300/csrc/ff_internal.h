// ff_internal.h - host <-> kernel interface of the fusion path (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fuseflow.h"
#include "ff_device.cuh"

namespace ffl {

struct FramePtrs {               // one frame's caller-owned device images, per camera
  const void* depth[kMaxCams];
  const float* conf[kMaxCams];
  const uint8_t* rgb[kMaxCams];
};

struct Tables {                  // context-owned device scratch
  // cells: dense slots, coarse cell c owns [cbase(c), cbase(c) + 8^level(c))
  SlotRec* frec;                 // key, list head and smallest exponent per slot
  unsigned* fused;               // used slots, in claim order
  unsigned max_slots;
  // coarse hash table (open addressing), ccap entries
  CoarseEntry* coarse;
  unsigned* cused;
  unsigned cmask;
  FrameCounters* cnt;
  BlockStats* bstats;            // one per block of the coarse-count step
  int n_bstats;
  Partial* part;                 // (tile, cell) partials, max_partials entries
  unsigned max_partials;
  CellOut* staged;               // fused cells by claim order, max_cells entries
  unsigned* bitmap;              // representative bitmap, one bit per pixel
  unsigned* wprefix;             // per-word exclusive prefix within its 1024-word block
  unsigned* bsum;                // per 1024-word block: exclusive prefix after the scan
  long long n_words;
  int n_wblocks;
  int n_min, max_level;          // level rule (Sec. II.5(1)d)
  const BlockConst* bconst;      // per-camera block constants
  const float4* pray;            // separable pair rays (PairDev::ga, gb)
  int n_tiles;
};

struct TraceDev {
  float* pw;
  float* omega;
  float* e;
  int* nview;
  unsigned long long* key;
};

struct OutDev {
  fuseflow_stats* stats;
  float* pos;
  float* rgb;
  float* weight;
  uint32_t* count;
  uint32_t* rep;
  unsigned long long* key;
  long long max_cells;
  float s0_m;                    // coarse edge, metres
  float unit_f;                  // metres per depth unit, float32
  double unit_m;                 // metres per depth unit
};

// Assign-step prefetch distance (tiles) that turns the L2 prefetch off.
constexpr int kNoPrefetch = 1 << 30;

// Everything the frame kernels need about one frame: the rig constants, its images, its
// tables and outputs, its tile index and count-step geometry.
struct FrameArgs {
  const RigDev* rig;
  const float2* rays;
  FramePtrs fp;
  Tables t;
  TraceDev tr;
  OutDev out;
  TileIndex ti;
  int count_blocks_x, count_chunks;
  float unit_m;
  int pad;
};

// Frames of one launch of the frame kernels, passed as one __grid_constant__ kernel
// parameter (kernel parameter space holds up to 32,764 bytes).  One-dimensional grids
// (count, assign) concatenate the frames' blocks: frame f owns blocks
// [count_first[f], count_first[f + 1]) of the count grid and [tile_first[f],
// tile_first[f + 1]) of the assign grid; the other kernels take the frame from blockIdx.y.
// NB = 1 is the plain one-frame launch (frame index 0, a compile-time constant).
constexpr int kMaxBatch = FUSEFLOW_MAX_BATCH;
template <int NB>
struct BatchArgs {
  int n;
  int count_first[NB + 1];
  int tile_first[NB + 1];
  FrameArgs f[NB];
};
static_assert(sizeof(BatchArgs<kMaxBatch>) <= 32764, "a batch fits in kernel parameter space");

// Depth preprocessing D^r of Eq. 8: range screen in depth units, then the edge screen
// against valid in-range 4-neighbours (bounds and ratio <= 0 are off).
struct ScreenArgs {
  const void* in[kMaxCams];
  void* out[kMaxCams];
  int W[kMaxCams], H[kMaxCams];
  int n_cams;
  float min_u, max_u;
  float edge_rel;
};
cudaError_t launch_screen(const ScreenArgs& a, bool depth_f32, long long max_px, cudaStream_t s);

struct Geometry {
  int n_cams;
  int depth_f32;
  int screen;                    // a screen is set: fuse calls write D^r into screen_buf first
  ScreenArgs scr;                // bounds, sizes and the context's D^r buffers (out)
  long long max_px;
  int count_blocks_x;            // blocks per camera of the coarse-count step (max over cams)
  int count_chunks;              // 2048-pixel chunks per block of the coarse-count step
  int emit_blocks;
  int top_k;                     // Sec. II.5(2)a variant (0: every member is fused)
  int pdl;                       // programmatic launches: 0 none, 1 all but assign -> reduce, 2 all
  TileIndex tiles;               // assign-step tiles
};

cudaError_t launch_init_tables(const Tables& t, unsigned fcap, unsigned ccap, cudaStream_t s);

// Host-side construction of the assign step's tile index and per-camera block constants
// (caller-sized array of rig.n_cams entries) from the rig constants.
// Host-mapped output arrays of one served frame (device-accessible addresses of pinned
// host memory) and the pinned statistics record the copy-out kernel fills.
struct HostOutDev {
  float* pos;
  float* rgb;
  float* weight;
  uint32_t* count;
  uint32_t* rep;
  unsigned long long* key;
  long long capacity;
  fuseflow_stats* stats;
};

// Copies the first min(n_cells, capacity) cells of a fused cloud and its statistics into
// host-mapped memory, asynchronously on s (one kernel, coalesced 4-byte stores).
cudaError_t launch_copyout(const fuseflow_cloud& src, const HostOutDev& dst, cudaStream_t s);

// Status of a frame from its device error bits: capacity overflows first, then internal
// consistency failures.
inline int status_of_error(unsigned err) {
  if (err & (kErrSlots | kErrCoarseFull | kErrCells | kErrPartials)) return FUSEFLOW_ERR_CAPACITY;
  if (err & (kErrCoarseMiss | kErrList)) return FUSEFLOW_ERR_INTERNAL;
  return FUSEFLOW_OK;
}

// Eq. 12 over n points (world metres): per-point error (metres) and visible-camera count
// (either may be NULL), per-block sums and counts in bsum/bcnt (mc_blocks(n) entries).
int mc_blocks(long long n);
cudaError_t launch_mc(const RigDev* rig, const FramePtrs& fp, bool depth_f32, const float* pos,
                      long long n, double unit_m, double occlusion_m, float* err, int* nvis,
                      double* bsum, long long* bcnt, cudaStream_t s);

// Point-wise fusion (Table II "No SA"): per global pixel index, the position (metres), the
// joint weight and the colour; counts[0..1] = valid and gated pixels of the frame.
struct PointsDev {
  float* pos;
  float* weight;
  uint8_t* rgb;
  unsigned long long* counts;
  float unit_f;
};
cudaError_t launch_points(const RigDev* rig, const float2* rays, const FramePtrs& fp, const Tables& t,
                          const PointsDev& out, bool depth_f32, int n_cams, long long max_px,
                          cudaStream_t s);

// Eq. 3 confidence producer: per camera, depth in, float32 confidence out.
struct ConfArgs {
  const void* depth[kMaxCams];
  float* out[kMaxCams];
  int W[kMaxCams], H[kMaxCams];
  int n_cams;
  float scale;                   // metres per depth unit
  float alpha, beta, gamma, delta;
  float inv_ag;                  // 1 / (alpha + gamma)
};
cudaError_t launch_confidence(const ConfArgs& a, bool depth_f32, int max_w, int max_h,
                              cudaStream_t s);

// assign-step blocks resident per SM for tiles of th rows and k1 neighbour views
int assign_resident_blocks(int th, int k1);
// tiles of th rows (8, 16 or 32) of the rig's cameras; returns their number
int fill_tile_index(const RigDev& rig, TileIndex* out, int th);
// the same index re-cut into tiles of th rows; returns their number
int retile(TileIndex* ti, int th);
void fill_block_consts(const RigDev& rig, BlockConst* out);
// Kernel attributes a frame's launches need (called by context creation, so that a later
// stream capture of launch_frame makes no attribute call).
cudaError_t prepare_launch(bool depth_f32);
// One frame of a launch (host side): rig constants, images, tables, trace, outputs and the
// launch geometry of its context.
struct FrameLaunch {
  const RigDev* rig;
  const float2* rays;
  FramePtrs fp;
  Tables t;
  TraceDev tr;
  OutDev out;
  const Geometry* geo;
};
// n <= kMaxBatch frames (one depth type, one fusion variant) with every frame kernel
// launched once for all of them: the frames' blocks share each grid.
cudaError_t launch_batch(const FrameLaunch* frames, int n, cudaStream_t s);
// ev: NULL, or FUSEFLOW_N_STAGES + 1 events recorded before, between and after the stages
cudaError_t launch_frame(const RigDev* rig, const float2* rays, const FramePtrs& fp,
                         const Tables& t, const TraceDev& tr, const OutDev& out,
                         const Geometry& geo, cudaStream_t s, cudaEvent_t* ev);

}  // namespace ffl
