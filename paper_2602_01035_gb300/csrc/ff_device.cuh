// ff_device.cuh - device data layout and per-pixel arithmetic of the sm_103a fusion path.
//
// Geometry is carried in "depth units" (metres per unit = depth_scale), so that the depth
// sample z of a pixel is exact in float32 (uint16 codes and float32 samples both are).
// World points, cell keys and the projection that selects a pixel are float32; the 3D
// residual of Eq. 6 is evaluated in double-float ("ff", an unevaluated hi + lo pair of
// float32) so that the joint weight of Eq. 10 keeps ~1e-7 relative accuracy although the
// residual is a difference of two metre-scale vectors.  The error-free transformations are
// Knuth's TwoSum, Dekker's Fast2Sum and the FMA TwoProduct, combined as in the compensated
// dot product of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26(6), 2005).
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace ffl {

constexpr int kMaxCams = 64;
constexpr int kMaxK1 = 8;
constexpr int kMaxTopK = 7;              // top-k keys travel in a partial record (rep + 6)
constexpr unsigned long long kKeyEmpty = ~0ull;
constexpr uint32_t kSlotNone = 0xffffffffu;
constexpr int kFixShift = 36;            // per-cell fixed point: largest member weight ~ 2^36
constexpr int kKeyBias = 1 << 19;        // cell index range [-2^19, 2^19) per axis
constexpr float kTieBandPx = 4e-3f;      // float32 projection error bound (pixels), generous

// error bits of FrameCounters::error
constexpr unsigned kErrSlots = 1u;       // the cells' dense slot ranges exceed the slot capacity
constexpr unsigned kErrCoarseFull = 2u;  // coarse hash table could not take a key
constexpr unsigned kErrCells = 4u;       // more cells than the output capacity
constexpr unsigned kErrCoarseMiss = 8u;  // a point's coarse cell was not found (internal)
constexpr unsigned kErrPartials = 16u;   // more (tile, cell) partials than the buffer holds
constexpr unsigned kErrList = 32u;       // a cell list was longer than the partials written

struct CamDev {
  int W, H;
  long long off;                 // global index of pixel (0, 0)
  float fx, fy, cx, cy;          // float32 intrinsics (projection into this camera)
  float fxh, fxl, fyh, fyl;      // ff intrinsics for exact half-pixel decisions
  float cxh, cxl, cyh, cyl;
  float Rwc[9];                  // world-from-camera rotation R^T, row-major
  float cwc[3];                  // camera centre (depth units)
  int ray_x, ray_y;              // offsets of this camera's ray tables
  int pair0;                     // first neighbour pair of this camera
  int pad;
};

struct PairDev {                 // camera i -> neighbour j: a = R_ji p_c + t_ji
  float Rh[9], Rl[9];            // R_ji = R_j R_i^T as ff
  float th[3], tl[3];            // t_ji = t_j - R_ji t_i as ff (depth units)
  int j;
  // separable pair rays: with p_c = z (rx(x), ry(y), 1), R_ji p_c = z (A(x) + B(y)),
  // A_k(x) = R_ji[k][0] rx(x) + R_ji[k][2] and B_k(y) = R_ji[k][1] ry(y), each stored as
  // ff in two float4 per column / row: (A0h, A0l, A1h, A1l), (A2h, A2l, 0, 0)
  int ga, gb;                    // float4 index of column 0's A and row 0's B
  int pad;
};

struct RigDev {
  int n_cams, k1;                // k1 = K - 1 neighbours per camera
  float tau;                     // Eq. 9 gate
  int use_conf, use_cons;
  int max_level, n_min;
  float inv_s0u;                 // 1 / s0 in 1 / depth units
  float einv_h, einv_l;          // 1 / (sigma_u^2 (K-1)) as ff
  int depth_f32;
  int top_k;                     // Sec. II.5(2)a variant: fuse the top_k members only (0: all)
  long long n_px;
  CamDev cam[kMaxCams];
  PairDev pair[kMaxCams * kMaxK1];
};

// Constants of one camera's tiles: the camera, its K-1 neighbour pairs and the neighbour
// cameras, contiguous so that a block copies them to shared memory in one round trip.
struct BlockConst {
  CamDev cam;
  PairDev pair[kMaxK1];
  CamDev nb[kMaxK1];
};

// Where the assign step's tiles are: camera i owns tiles [first[i], first[i+1]), row-major
// over its ceil(W/32) x ceil(H/th) grid.  Passed by value (constant bank) to the kernel.
struct TileIndex {
  int n_cams, k1;
  int th;                        // tile height (8, 16 or 32 rows of 32 columns)
  int first[kMaxCams + 1];
  int W[kMaxCams], H[kMaxCams];
  long long off[kMaxCams];       // global index of each camera's pixel (0, 0)
  int pray[kMaxCams];            // float4 index of the camera's first pair ray: pair q's A
                                 // starts at pray + 2 q (W + H), its B 2 W further
  int per_cam;                   // tiles per camera when all cameras share W and H, else 0
  int ahead;                     // tiles resident at once: block b prefetches tile b + ahead
};

// Per (tile, cell) partial result of the assign step, pushed onto its cell's list when it
// is written.  Sums are exact integers in units of 2^-(kFixShift + mmin) of the tile's own
// smallest weight exponent mmin; the reduce step shifts them to the cell's smallest one.
// Each sum is below 2^46 (at most 512 terms below 2^37), so 48 bits hold it: the record is
// 64 bytes, two aligned 32-byte sectors.
struct __align__(64) Partial {
  unsigned long long rep;        // max of ordered(C) << 32 | ~g (top-k: the tile's first key)
  unsigned next;                 // next partial of the same cell, kSlotNone at the end
  unsigned count;                // members in the tile
  union {
    struct {
      int mmin;                  // smallest weight exponent m in the tile
      unsigned lo[7];            // bits 0..31 of the sums of w, w frac_x, w frac_y, w frac_z,
      unsigned short hi[7];      //   w r, w g, w b; bits 32..47
      unsigned short pad;
    } sum;
    unsigned long long top[kMaxTopK - 1];   // top-k variant: the tile's keys 2..k
  };
  __device__ __forceinline__ void set_sum(int a, unsigned long long v) {
    sum.lo[a] = (unsigned)v;
    sum.hi[a] = (unsigned short)(v >> 32);
  }
  __device__ __forceinline__ unsigned long long get_sum(int a) const {
    return ((unsigned long long)sum.hi[a] << 32) | sum.lo[a];
  }
};
static_assert(sizeof(Partial) == 64, "partial record layout");

// Per dense cell slot: the cell's key, its list head and its smallest weight exponent, in
// one 16-byte record so that the reduce step reads a single sector per cell.
struct __align__(16) SlotRec {
  unsigned long long key;
  unsigned head;                 // last partial pushed, kSlotNone if none
  int mmin;                      // smallest weight exponent over the cell's partials
};

// Coarse hash-table record: key, density count (Sec. II.5(1)c) and, once every count is
// in, the level and first dense cell slot packed as level << 27 | base.
struct __align__(16) CoarseEntry {
  unsigned long long key;
  unsigned count;
  unsigned lvbase;
};
constexpr unsigned kBaseNone = (1u << 27) - 1u;    // base field of a coarse cell without slots

// Fused cell staged by the reduce step (indexed by insertion order) for the emit step.
struct __align__(16) CellOut {
  float pos[3];
  float rgb[3];
  float weight;
  unsigned count;
  unsigned rep;
  unsigned pad;
  unsigned long long key;
};
static_assert(sizeof(CellOut) == 48, "staged cell layout");

struct FrameCounters {           // zeroed before every frame
  unsigned n_cells, n_coarse;
  unsigned error;
  unsigned n_partials;
  unsigned long long n_valid, n_gated, n_oor;
  unsigned bmin_inv[3];          // ~ordered(min): max-reduced so that zero is neutral
  unsigned bmax[3];              // ordered(max)
  unsigned scan_done;            // blocks of the scan step that have finished
  unsigned pad;
  unsigned long long n_slots;    // dense cell slots claimed (sum over coarse cells of 8^l)
};

struct BlockStats {              // per block of the coarse-count step
  unsigned n_valid, n_gated, n_oor, pad;
  unsigned bmin[3], bmax[3];     // ordered-integer encodings
  unsigned pad2[2];
};

// ----------------------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned ordered(float f) {
  unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float from_ordered(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
#else
  unsigned v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  float f;
  memcpy(&f, &v, 4);
  return f;
#endif
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
  k ^= k >> 31;
  k *= 0x7fb5d329728ea185ull;
  k ^= k >> 27;
  k *= 0x81dadef4bc2dd44dull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ unsigned long long pack_key(int l, int kx, int ky, int kz) {
  return ((unsigned long long)l << 60) | ((unsigned long long)(kx + kKeyBias) << 40) |
         ((unsigned long long)(ky + kKeyBias) << 20) | (unsigned long long)(kz + kKeyBias);
}

// --------------------------------------------------------------------------- double-float
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// Row k of an affine map in ff: o = R[k,:] . (px, py, z) + t[k], with px, py ff and z exact.
__device__ __forceinline__ void ff_affine_row(const float* Rh, const float* Rl, float th, float tl,
                                              float pxh, float pxl, float pyh, float pyl, float z,
                                              float& oh, float& ol) {
  float p1, e1, p2, e2, p3, e3;
  two_prod(Rh[0], pxh, p1, e1);
  e1 = __fmaf_rn(Rh[0], pxl, e1);
  e1 = __fmaf_rn(Rl[0], pxh, e1);
  two_prod(Rh[1], pyh, p2, e2);
  e2 = __fmaf_rn(Rh[1], pyl, e2);
  e2 = __fmaf_rn(Rl[1], pyh, e2);
  two_prod(Rh[2], z, p3, e3);
  e3 = __fmaf_rn(Rl[2], z, e3);
  float s, q1, q2, q3;
  two_sum(p1, p2, s, q1);
  two_sum(s, p3, s, q2);
  two_sum(s, th, s, q3);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, q1)),
                             __fadd_rn(__fadd_rn(q2, q3), tl));
  fast_two_sum(s, lo, oh, ol);
}

// One component of a = z (A + B) + t in ff (A, B, t as ff, z exact); the result (oh, ol)
// is not renormalised (|ol| stays within a few ulp of oh, unless z(A + B) and t cancel).
__device__ __forceinline__ void ff_ray_affine(float Ah, float Al, float Bh, float Bl, float z,
                                              float th, float tl, float& oh, float& ol) {
  float gh, ge, p, pe, e;
  two_sum(Ah, Bh, gh, ge);
  ge = __fadd_rn(ge, __fadd_rn(Al, Bl));
  two_prod(z, gh, p, pe);
  pe = __fmaf_rn(z, ge, pe);
  two_sum(p, th, oh, e);
  ol = __fadd_rn(e, __fadd_rn(pe, tl));
}

// --------------------------------------------------------------------------- depth decode
template <typename DT> struct Depth;
template <> struct Depth<uint16_t> {
  static __device__ __forceinline__ bool valid(uint16_t d) { return d != 0; }
  static __device__ __forceinline__ float z(uint16_t d) { return (float)d; }
};
template <> struct Depth<float> {
  static __device__ __forceinline__ bool valid(float d) { return d > 0.0f && d < __int_as_float(0x7f800000); }
  static __device__ __forceinline__ float z(float d) { return d; }
};

// Eq. 8 in float32: world point (depth units) of pixel ray (rx, ry, 1) at z-depth z.
// Every step uses the same rounding-explicit sequence so all kernels agree bit for bit.
__device__ __forceinline__ void world_point(const CamDev& c, float z, float rx, float ry,
                                            float P[3]) {
  const float px = __fmul_rn(z, rx), py = __fmul_rn(z, ry);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    P[k] = __fmaf_rn(c.Rwc[3 * k + 0], px,
                     __fmaf_rn(c.Rwc[3 * k + 1], py, __fmaf_rn(c.Rwc[3 * k + 2], z, c.cwc[k])));
}

// 2^e as a float for -126 <= e <= 127, built from its bits (exact scaling by a product).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// Sec. II.5(1): coarse-grid coordinate r = P / s0 and the range test at the finest level:
// floor(r 2^Lmax) in [-2^19, 2^19)  <=>  r 2^Lmax in [-2^19, 2^19).
__device__ __forceinline__ bool grid_coords(const RigDev& rig, const float P[3], float r[3]) {
  bool ok = true;
  const float lim = (float)kKeyBias;
  const float sL = pow2f(rig.max_level);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r[k] = __fmul_rn(P[k], rig.inv_s0u);
    const float v = __fmul_rn(r[k], sL);
    ok = ok && (v >= -lim) && (v < lim);
  }
  return ok;
}

__device__ __forceinline__ unsigned long long coarse_key(const float r[3]) {
  return pack_key(0, (int)floorf(r[0]), (int)floorf(r[1]), (int)floorf(r[2]));
}

// Sec. II.5(1)d: level of a coarse cell holding n_c points: largest l <= Lmax with
// n_c >= n_min 4^l, else 0.
__device__ __forceinline__ int level_for(unsigned n_c, int n_min, int max_level) {
  int l = 0;
  for (int c = 1; c <= max_level; ++c)
    if ((unsigned long long)n_c >= ((unsigned long long)n_min << (2 * c))) l = c;
  return l;
}

__device__ __forceinline__ unsigned long long fine_key(const float r[3], int l) {
  const float sl = pow2f(l);
  return pack_key(l, (int)floorf(__fmul_rn(r[0], sl)), (int)floorf(__fmul_rn(r[1], sl)),
                  (int)floorf(__fmul_rn(r[2], sl)));
}

}  // namespace ffl
