// ff_kernels.cu - sm_103a kernels of the FUSE-Flow per-frame fusion path.
//
// Launch sequence of one frame (all on the caller's stream):
//   memset   frame counters + representative bitmap
//   count    (a) decode + gate + back-project (Eq. 8, 9), coarse density n_c (Sec. II.5(1)c),
//            per-block pixel counts and extent (Sec. II.5(1)b)
//   assign   (b) consistency V (Eq. 4-7), omega = C V (Eq. 10) as mantissa/exponent;
//            (c) level per coarse cell (Sec. II.5(1)d), cell key (Sec. II.5(1)e), fine
//            hash insertion; (d) per (tile, cell): member count, representative
//            (Sec. II.5(2)a), smallest weight exponent and exact fixed-point sums of
//            omega, omega P, omega RGB (Eq. 11), written as one partial record linked
//            into the cell's list
//   reduce   per cell: walk its partials, combine them, stage the fused cell, mark its
//            representative; the used hash slots are cleared for the next frame
//   scan     ranks of the representatives (output order), frame statistics
//   emit     fused cells in representative order
//
// Every reduction is order-independent (integer counts, max, min and fixed-point sums,
// warp-level first, then shared memory, then one record per tile and cell), so the output
// is bitwise reproducible.
#include <climits>
#include <cstdint>

#include "ff_internal.h"

namespace ffl {

namespace {

constexpr int kThreads = 256;
constexpr int kCountPx = 4;                       // pixels per thread in the count step
constexpr int kCountBlockPx = kThreads * kCountPx;
constexpr int kTileW = 32, kTileH = 16;           // assign/accum tile: 8 warps x 2 rows
constexpr int kTilePx = kTileW * kTileH;
constexpr int kMaxProbe = 1 << 14;
constexpr float kLn2H = 0.693147182464599609375f;         // float(ln 2)
constexpr float kLn2L = -1.904654299957768e-09f;          // ln 2 - kLn2H
constexpr float kInvLn2 = 1.44269504088896340736f;

// ------------------------------------------------------------------ global hash tables
__device__ __forceinline__ unsigned fine_insert(const Tables& t, unsigned long long key) {
  unsigned h = (unsigned)mix64(key) & t.fmask;
  for (int probe = 0; probe < kMaxProbe; ++probe) {
    unsigned long long cur = __ldcg(&t.fkey[h]);
    if (cur == key) return h;
    if (cur == kKeyEmpty) {
      cur = atomicCAS(&t.fkey[h], kKeyEmpty, key);
      if (cur == kKeyEmpty) {
        const unsigned n = atomicAdd(&t.cnt->n_cells, 1u);
        if (n <= t.fmask) t.fused[n] = h;
        return h;
      }
      if (cur == key) return h;
    }
    h = (h + 1) & t.fmask;
  }
  atomicOr(&t.cnt->error, kErrFineFull);
  return kSlotNone;
}

__device__ __forceinline__ unsigned coarse_insert(const Tables& t, unsigned long long key) {
  unsigned h = (unsigned)mix64(key) & t.cmask;
  for (int probe = 0; probe < kMaxProbe; ++probe) {
    unsigned long long cur = __ldcg(&t.ckey[h]);
    if (cur == key) return h;
    if (cur == kKeyEmpty) {
      cur = atomicCAS(&t.ckey[h], kKeyEmpty, key);
      if (cur == kKeyEmpty) {
        const unsigned n = atomicAdd(&t.cnt->n_coarse, 1u);
        if (n <= t.cmask) t.cused[n] = h;
        return h;
      }
      if (cur == key) return h;
    }
    h = (h + 1) & t.cmask;
  }
  atomicOr(&t.cnt->error, kErrCoarseFull);
  return kSlotNone;
}

__device__ __forceinline__ unsigned coarse_count_of(const Tables& t, unsigned long long key) {
  unsigned h = (unsigned)mix64(key) & t.cmask;
  for (int probe = 0; probe < kMaxProbe; ++probe) {
    const unsigned long long cur = __ldcg(&t.ckey[h]);
    if (cur == key) return __ldcg(&t.ccount[h]);
    if (cur == kKeyEmpty) break;
    h = (h + 1) & t.cmask;
  }
  atomicOr(&t.cnt->error, kErrCoarseMiss);
  return 0;
}

// Block-local open addressing (shared memory); returns the table position or -1.
template <int TS, typename K>
__device__ __forceinline__ int local_pos(K* tab, K empty, K key) {
  unsigned h = (unsigned)mix64((unsigned long long)key) & (TS - 1);
  for (int probe = 0; probe < TS; ++probe) {
    const K cur = *static_cast<volatile K*>(&tab[h]);
    if (cur == key) return (int)h;
    if (cur == empty) {
      const K prev = atomicCAS(&tab[h], empty, key);
      if (prev == empty || prev == key) return (int)h;
    }
    h = (h + 1) & (TS - 1);
  }
  return -1;
}

// ------------------------------------------------------------------ block constants
// The tile's camera, its K-1 neighbour pairs and the neighbour cameras, staged in shared
// memory once per block (every pixel of a tile belongs to the same camera).
struct BlockConst {
  CamDev cam;
  PairDev pair[kMaxK1];
  CamDev nb[kMaxK1];
};

__device__ __forceinline__ void copy_words(void* dst, const void* src, int bytes) {
  int* d = static_cast<int*>(dst);
  const int* s = static_cast<const int*>(src);
  for (int i = threadIdx.x; i < bytes / 4; i += blockDim.x) d[i] = s[i];
}

// ------------------------------------------------------------------ Eq. 4-7 per point
// Exact floor(u + 1/2) for u = fx a_x / a_z + cx near a tie at integer r (a_z > 0):
// u + 1/2 >= r  <=>  fx a_x + (cx + 1/2 - r) a_z >= 0, evaluated in double-float.
__device__ __forceinline__ int exact_round(float fh, float fl, float ch, float cl, float axh,
                                           float axl, float azh, float azl, float r) {
  float p1, e1, c0, ce, p2, e2, s, q;
  two_prod(fh, axh, p1, e1);
  e1 = __fmaf_rn(fh, axl, __fmaf_rn(fl, axh, e1));
  two_sum(ch, __fsub_rn(0.5f, r), c0, ce);
  ce = __fadd_rn(ce, cl);
  two_prod(c0, azh, p2, e2);
  e2 = __fmaf_rn(c0, azl, __fmaf_rn(ce, azh, e2));
  two_sum(p1, p2, s, q);
  const float f = __fadd_rn(s, __fadd_rn(__fadd_rn(e1, e2), q));
  return (f >= 0.0f) ? (int)r : (int)r - 1;
}

// Sum over the K-1 neighbour views of d_ij^2 (Eq. 6) in depth units^2, as ff (sh, sl).
template <typename DT>
__device__ __forceinline__ void residual_sum(const BlockConst& bc, int k1,
                                             const float2* __restrict__ rays,
                                             const FramePtrs& fp, float z, float2 rx, float2 ry,
                                             float& sh, float& sl, int& nview) {
  float pxh, pxl, pyh, pyl;
  two_prod(z, rx.x, pxh, pxl);
  pxl = __fmaf_rn(z, rx.y, pxl);
  two_prod(z, ry.x, pyh, pyl);
  pyl = __fmaf_rn(z, ry.y, pyl);
  sh = 0.0f;
  sl = 0.0f;
  nview = 0;
  for (int q = 0; q < k1; ++q) {
    const PairDev& P = bc.pair[q];
    const CamDev& J = bc.nb[q];
    float a[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      a[k] = __fmaf_rn(P.Rh[3 * k], pxh, __fmaf_rn(P.Rh[3 * k + 1], pyh,
                                                   __fmaf_rn(P.Rh[3 * k + 2], z, P.th[k])));
    float ah[3], al[3];
    bool have = false;
    if (a[2] < kZGuard) {       // close to camera j's image plane: decide the sign exactly
#pragma unroll
      for (int k = 0; k < 3; ++k)
        ff_affine_row(P.Rh + 3 * k, P.Rl + 3 * k, P.th[k], P.tl[k], pxh, pxl, pyh, pyl, z,
                      ah[k], al[k]);
      have = true;
      if (!(ah[2] > 0.0f)) continue;                    // behind camera j (Eq. 4 FoV check)
      a[0] = ah[0];
      a[1] = ah[1];
      a[2] = ah[2];
    }
    const float inv = __frcp_rn(a[2]);
    const float fu = __fadd_rn(__fmaf_rn(J.fx, __fmul_rn(a[0], inv), J.cx), 0.5f);
    const float fv = __fadd_rn(__fmaf_rn(J.fy, __fmul_rn(a[1], inv), J.cy), 0.5f);
    if (!(fu > -1.0f && fu < (float)J.W + 1.0f && fv > -1.0f && fv < (float)J.H + 1.0f))
      continue;
    const float ru = rintf(fu), rv = rintf(fv);
    const bool tie_u = fabsf(fu - ru) < kTieBandPx, tie_v = fabsf(fv - rv) < kTieBandPx;
    if ((tie_u || tie_v) && !have) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
        ff_affine_row(P.Rh + 3 * k, P.Rl + 3 * k, P.th[k], P.tl[k], pxh, pxl, pyh, pyl, z,
                      ah[k], al[k]);
      have = true;
    }
    const int px = tie_u ? exact_round(J.fxh, J.fxl, J.cxh, J.cxl, ah[0], al[0], ah[2], al[2], ru)
                         : (int)floorf(fu);
    const int py = tie_v ? exact_round(J.fyh, J.fyl, J.cyh, J.cyl, ah[1], al[1], ah[2], al[2], rv)
                         : (int)floorf(fv);
    if (px < 0 || px >= J.W || py < 0 || py >= J.H) continue;   // field-of-view check
    const DT Dj = __ldg(static_cast<const DT*>(fp.depth[P.j]) + (long long)py * J.W + px);
    if (!Depth<DT>::valid(Dj)) continue;
    if (!have) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
        ff_affine_row(P.Rh + 3 * k, P.Rl + 3 * k, P.th[k], P.tl[k], pxh, pxl, pyh, pyl, z,
                      ah[k], al[k]);
    }
    // Eq. 5: Q = D_j(u_j) (rx_j, ry_j, 1) in camera-j coordinates (rigid motion keeps d).
    const float zj = Depth<DT>::z(Dj);
    const float2 qx = __ldg(rays + J.ray_x + px), qy = __ldg(rays + J.ray_y + py);
    float qh[3], ql[3];
    two_prod(zj, qx.x, qh[0], ql[0]);
    ql[0] = __fmaf_rn(zj, qx.y, ql[0]);
    two_prod(zj, qy.x, qh[1], ql[1]);
    ql[1] = __fmaf_rn(zj, qy.y, ql[1]);
    qh[2] = zj;
    ql[2] = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {                      // Eq. 6: d^2 = |a - Q|^2 in ff
      float s, e, dh, dl, p, pe, t;
      two_sum(ah[k], -qh[k], s, e);
      e = __fadd_rn(e, __fsub_rn(al[k], ql[k]));
      fast_two_sum(s, e, dh, dl);
      two_prod(dh, dh, p, pe);
      pe = __fmaf_rn(__fmul_rn(2.0f, dh), dl, pe);
      two_sum(sh, p, sh, t);
      sl = __fadd_rn(sl, __fadd_rn(t, pe));
    }
    ++nview;
  }
}

// ------------------------------------------------------------------ count step
template <typename DT>
__device__ __forceinline__ void load4(const DT* __restrict__ d, const float* __restrict__ c,
                                      long long p0, long long npx, DT dv[4], float cv[4]) {
  const bool full = p0 + 3 < npx;
  if constexpr (sizeof(DT) == 2) {
    if (full && ((reinterpret_cast<uintptr_t>(d + p0) & 7) == 0)) {
      const uint2 u = __ldcs(reinterpret_cast<const uint2*>(d + p0));
      dv[0] = (DT)(u.x & 0xffff); dv[1] = (DT)(u.x >> 16);
      dv[2] = (DT)(u.y & 0xffff); dv[3] = (DT)(u.y >> 16);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) dv[k] = (p0 + k < npx) ? d[p0 + k] : (DT)0;
    }
  } else {
    if (full && ((reinterpret_cast<uintptr_t>(d + p0) & 15) == 0)) {
      const float4 f = __ldcs(reinterpret_cast<const float4*>(d + p0));
      dv[0] = f.x; dv[1] = f.y; dv[2] = f.z; dv[3] = f.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) dv[k] = (p0 + k < npx) ? d[p0 + k] : (DT)0;
    }
  }
  if (full && ((reinterpret_cast<uintptr_t>(c + p0) & 15) == 0)) {
    const float4 f = __ldcs(reinterpret_cast<const float4*>(c + p0));
    cv[0] = f.x; cv[1] = f.y; cv[2] = f.z; cv[3] = f.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) cv[k] = (p0 + k < npx) ? c[p0 + k] : 0.0f;
  }
}

template <typename DT>
__global__ void __launch_bounds__(kThreads, 4)
k_count(const RigDev* __restrict__ rigp, const float2* __restrict__ rays, FramePtrs fp, Tables t,
        int blocks_x) {
  constexpr int TS = 2 * kCountBlockPx;
  __shared__ unsigned long long s_key[TS];
  __shared__ unsigned s_cnt[TS];
  __shared__ unsigned s_red[kThreads / 32][9];
  const RigDev& rig = *rigp;
  const int cam = blockIdx.y;
  const CamDev& C = rig.cam[cam];
  const long long npx = (long long)C.W * C.H;
  const int bid = cam * blocks_x + blockIdx.x;
  if ((long long)blockIdx.x * kCountBlockPx >= npx) {
    if (threadIdx.x == 0) {
      BlockStats b = {};
      for (int k = 0; k < 3; ++k) { b.bmin[k] = 0xffffffffu; b.bmax[k] = 0u; }
      t.bstats[bid] = b;
    }
    return;
  }
  for (int i = threadIdx.x; i < TS; i += kThreads) { s_key[i] = kKeyEmpty; s_cnt[i] = 0; }
  __syncthreads();

  const DT* __restrict__ dep = static_cast<const DT*>(fp.depth[cam]);
  const float* __restrict__ cf = fp.conf[cam];
  const long long p0 = ((long long)blockIdx.x * kThreads + threadIdx.x) * kCountPx;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  DT dv[4];
  float cv[4];
  unsigned nv = 0, ng = 0, noor = 0;
  unsigned bmin[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, bmax[3] = {0u, 0u, 0u};
  unsigned long long rk[kCountPx] = {kKeyEmpty, kKeyEmpty, kKeyEmpty, kKeyEmpty};
  unsigned rn[kCountPx] = {1u, 1u, 1u, 1u};
  if (p0 < npx) {
    load4<DT>(dep, cf, p0, npx, dv, cv);
    int y = (int)(p0 / C.W);
    int x = (int)(p0 - (long long)y * C.W);
#pragma unroll
    for (int k = 0; k < kCountPx; ++k) {
      if (p0 + k < npx && Depth<DT>::valid(dv[k])) {
        ++nv;
        if (!rig.use_conf || cv[k] > rig.tau) {       // Eq. 9
          ++ng;
          float P[3], r[3];
          world_point(C, Depth<DT>::z(dv[k]), __ldg(&rays[C.ray_x + x].x), __ldg(&rays[C.ray_y + y].x), P);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const unsigned o = ordered(P[a]);
            bmin[a] = min(bmin[a], o);
            bmax[a] = max(bmax[a], o);
          }
          if (grid_coords(rig, P, r)) rk[k] = coarse_key(r);
          else ++noor;
        }
      }
      if (++x == C.W) { x = 0; ++y; }
    }
  }
  // Sec. II.5(1)c density estimate: merge the thread's equal neighbours, then one
  // shared-memory update per distinct key and thread
#pragma unroll
  for (int k = 1; k < kCountPx; ++k)
    if (rk[k] != kKeyEmpty && rk[k] == rk[k - 1]) {
      rn[k] += rn[k - 1];
      rk[k - 1] = kKeyEmpty;
    }
#pragma unroll
  for (int j = 0; j < kCountPx; ++j) {
    if (rk[j] == kKeyEmpty) continue;
    const int h = local_pos<TS>(s_key, kKeyEmpty, rk[j]);
    if (h >= 0) atomicAdd(&s_cnt[h], rn[j]);
    else atomicOr(&t.cnt->error, kErrCoarseFull);
  }
  // per-block pixel counts and extent
  unsigned vals[9] = {nv, ng, noor, bmin[0], bmin[1], bmin[2], bmax[0], bmax[1], bmax[2]};
  vals[0] = __reduce_add_sync(0xffffffffu, vals[0]);
  vals[1] = __reduce_add_sync(0xffffffffu, vals[1]);
  vals[2] = __reduce_add_sync(0xffffffffu, vals[2]);
  for (int a = 0; a < 3; ++a) {
    vals[3 + a] = __reduce_min_sync(0xffffffffu, vals[3 + a]);
    vals[6 + a] = __reduce_max_sync(0xffffffffu, vals[6 + a]);
  }
  if (lane == 0)
    for (int a = 0; a < 9; ++a) s_red[warp][a] = vals[a];
  __syncthreads();
  if (threadIdx.x == 0) {
    BlockStats b = {};
    for (int k = 0; k < 3; ++k) { b.bmin[k] = 0xffffffffu; b.bmax[k] = 0u; }
    for (int w = 0; w < kThreads / 32; ++w) {
      b.n_valid += s_red[w][0];
      b.n_gated += s_red[w][1];
      b.n_oor += s_red[w][2];
      for (int k = 0; k < 3; ++k) {
        b.bmin[k] = min(b.bmin[k], s_red[w][3 + k]);
        b.bmax[k] = max(b.bmax[k], s_red[w][6 + k]);
      }
    }
    t.bstats[bid] = b;
  }
  for (int i = threadIdx.x; i < TS; i += kThreads) {
    const unsigned long long key = s_key[i];
    if (key == kKeyEmpty) continue;
    const unsigned slot = coarse_insert(t, key);
    if (slot != kSlotNone) atomicAdd(&t.ccount[slot], s_cnt[i]);
  }
}

// ------------------------------------------------------------------ assign step
constexpr int kAssignTS = 2 * kTilePx;     // shared hash positions (keys <= pixels of a tile)
constexpr int kAssignNL = kTilePx;         // distinct fine cells of a tile, at most
constexpr size_t align16(size_t v) { return (v + 15) / 16 * 16; }
constexpr size_t kSmBC = 0;
constexpr size_t kSmCK = align16(kSmBC + sizeof(BlockConst));      // u64[TS] coarse keys
constexpr size_t kSmCL = align16(kSmCK + 8 * kAssignTS);           // u8[TS] coarse levels
constexpr size_t kSmFK = align16(kSmCL + kAssignTS);               // u64[TS] fine keys
constexpr size_t kSmFI = align16(kSmFK + 8 * kAssignTS);           // int[TS] entry of a position
constexpr size_t kSmEK = align16(kSmFI + 4 * kAssignTS);           // u64[NL] key of an entry
constexpr size_t kSmAcc = align16(kSmEK + 8 * kAssignNL);          // u32[14][NL] split sums
constexpr size_t kSmCnt = align16(kSmAcc + 14 * 4 * kAssignNL);    // u32[NL] members
constexpr size_t kSmCmax = align16(kSmCnt + 4 * kAssignNL);        // u32[NL] largest ordered C
constexpr size_t kSmGmin = align16(kSmCmax + 4 * kAssignNL);       // u32[NL] lowest index at it
constexpr size_t kSmMin = align16(kSmGmin + 4 * kAssignNL);        // int[NL] smallest exponent
constexpr size_t kSmPid = align16(kSmMin + 4 * kAssignNL);         // u16[tile] gated pixels
constexpr size_t kAssignSmem = align16(kSmPid + 2 * kTilePx);
constexpr unsigned kLoBits = 22;           // split of a <= 2^37 sum term: 512 lows fit in u32

template <typename DT>
__global__ void __launch_bounds__(kThreads, 3)
k_assign(const RigDev* __restrict__ rigp, const float2* __restrict__ rays, FramePtrs fp, Tables t,
         TraceDev tr, float unit_m) {
  extern __shared__ __align__(16) unsigned char smem[];
  BlockConst& bc = *reinterpret_cast<BlockConst*>(smem + kSmBC);
  unsigned long long* s_ck = reinterpret_cast<unsigned long long*>(smem + kSmCK);
  unsigned char* s_cl = smem + kSmCL;
  unsigned long long* s_fk = reinterpret_cast<unsigned long long*>(smem + kSmFK);
  int* s_fi = reinterpret_cast<int*>(smem + kSmFI);
  unsigned long long* s_ek = reinterpret_cast<unsigned long long*>(smem + kSmEK);
  unsigned* s_acc = reinterpret_cast<unsigned*>(smem + kSmAcc);
  unsigned* s_cnt = reinterpret_cast<unsigned*>(smem + kSmCnt);
  unsigned* s_cmax = reinterpret_cast<unsigned*>(smem + kSmCmax);
  unsigned* s_gmin = reinterpret_cast<unsigned*>(smem + kSmGmin);
  int* s_min = reinterpret_cast<int*>(smem + kSmMin);
  unsigned short* s_pid = reinterpret_cast<unsigned short*>(smem + kSmPid);
  __shared__ unsigned s_n, s_base, s_ng;
  __shared__ unsigned s_wc[2 * (kThreads / 32)];

  const RigDev& rig = *rigp;
  const int cam = blockIdx.y;
  const int W = rig.cam[cam].W, H = rig.cam[cam].H;
  const int tiles_x = (W + kTileW - 1) / kTileW;
  const int tiles_y = (H + kTileH - 1) / kTileH;
  if ((int)blockIdx.x >= tiles_x * tiles_y) return;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k1 = rig.k1;
  copy_words(&bc.cam, &rig.cam[cam], sizeof(CamDev));
  for (int q = 0; q < k1; ++q) {
    const PairDev& src = rig.pair[rig.cam[cam].pair0 + q];
    copy_words(&bc.pair[q], &src, sizeof(PairDev));
    copy_words(&bc.nb[q], &rig.cam[src.j], sizeof(CamDev));
  }
  for (int i = threadIdx.x; i < kAssignTS; i += kThreads) {
    s_ck[i] = kKeyEmpty;
    s_fk[i] = kKeyEmpty;
  }
  if (threadIdx.x == 0) s_n = 0;

  const DT* __restrict__ dep = static_cast<const DT*>(fp.depth[cam]);
  const float* __restrict__ cf = fp.conf[cam];
  const uint8_t* __restrict__ col = fp.rgb[cam];
  const bool trace = tr.pw || tr.omega || tr.e || tr.nview || tr.key;
  const float qnan = __int_as_float(0x7fc00000);

  // (a) Eq. 9 gate, then compaction of the tile's gated pixels so that the per-point work
  // below runs on full warps
  unsigned gmask[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int row = warp + 8 * k;
    const int x = tx * kTileW + lane, y = ty * kTileH + row;
    bool gated = false;
    if (x < W && y < H) {
      const long long li = (long long)y * W + x;
      const DT D = dep[li];
      gated = Depth<DT>::valid(D) && (!rig.use_conf || cf[li] > rig.tau);
      if (!gated && trace) {
        const long long g = rig.cam[cam].off + li;
        if (tr.pw) { tr.pw[3 * g] = qnan; tr.pw[3 * g + 1] = qnan; tr.pw[3 * g + 2] = qnan; }
        if (tr.e) tr.e[g] = qnan;
        if (tr.omega) tr.omega[g] = qnan;
        if (tr.nview) tr.nview[g] = -1;
        if (tr.key) tr.key[g] = kKeyEmpty;
      }
    }
    gmask[k] = __ballot_sync(0xffffffffu, gated);
    if (lane == 0) s_wc[row] = __popc(gmask[k]);
  }
  __syncthreads();
  if (threadIdx.x < 32) {            // exclusive scan of the 16 row counts
    const unsigned v = threadIdx.x < 16 ? s_wc[threadIdx.x] : 0u;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (threadIdx.x < 16) s_wc[threadIdx.x] = x - v;
    if (threadIdx.x == 15) s_ng = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int row = warp + 8 * k;
    if ((gmask[k] >> lane) & 1u)
      s_pid[s_wc[row] + __popc(gmask[k] & ((1u << lane) - 1u))] = (unsigned short)(row * kTileW + lane);
  }
  __syncthreads();
  const int n_g = (int)s_ng;
  const CamDev& C = bc.cam;

  // (a) + (b): back-project, consistency, weight; coarse cell of each gated point
  float r[2][3];
  bool has[2] = {false, false};
  float mu[2] = {0.0f, 0.0f};
  int mexp[2] = {0, 0};
  unsigned cord[2] = {0u, 0u};
  int hpos[2] = {0, 0};
  long long gi[2] = {0, 0}, li[2] = {0, 0};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int i = threadIdx.x + j * kThreads;
    if (i >= n_g) continue;
    const int pid = s_pid[i];
    const int x = tx * kTileW + (pid & (kTileW - 1)), y = ty * kTileH + pid / kTileW;
    li[j] = (long long)y * W + x;
    gi[j] = C.off + li[j];
    const float z = Depth<DT>::z(dep[li[j]]);
    const float c = cf[li[j]];
    const float2 rx = __ldg(rays + C.ray_x + x), ry = __ldg(rays + C.ray_y + y);
    float P[3];
    world_point(C, z, rx.x, ry.x, P);                                 // Eq. 8
    float sh = 0.0f, sl = 0.0f, eh = 0.0f, el = 0.0f;
    int nview = 0;
    if (rig.use_cons && k1 > 0) {
      residual_sum<DT>(bc, k1, rays, fp, z, rx, ry, sh, sl, nview);
      fast_two_sum(sh, sl, sh, sl);
      two_prod(sh, rig.einv_h, eh, el);                               // Eq. 7 exponent
      el = __fmaf_rn(sh, rig.einv_l, __fmaf_rn(sl, rig.einv_h, el));
      fast_two_sum(eh, el, eh, el);
    }
    // omega = C exp(-e) = mu 2^-m, e = m ln2 + f, f in [0, ln2): mu never underflows
    int m = 0;
    float fh = eh, fl = el;
    if (eh > 0.0f) {
      m = (int)floorf(__fmul_rn(fminf(eh, 1.0e9f), kInvLn2));
      const float mf = (float)m;
      float p, pe;
      two_prod(mf, kLn2H, p, pe);
      fh = __fsub_rn(eh, p);
      fl = __fsub_rn(__fsub_rn(el, pe), __fmul_rn(mf, kLn2L));
    }
    const float base = rig.use_conf ? c : 1.0f;                       // Eq. 10
    mu[j] = __fmul_rn(__fmul_rn(base, expf(-fh)), __fsub_rn(1.0f, fl));
    mexp[j] = m;
    cord[j] = ordered(c);
    has[j] = grid_coords(rig, P, r[j]);
    if (trace) {
      if (tr.pw) {
        tr.pw[3 * gi[j] + 0] = P[0] * unit_m;
        tr.pw[3 * gi[j] + 1] = P[1] * unit_m;
        tr.pw[3 * gi[j] + 2] = P[2] * unit_m;
      }
      if (tr.e) tr.e[gi[j]] = eh;
      if (tr.omega) tr.omega[gi[j]] = ldexpf(mu[j], -m);
      if (tr.nview) tr.nview[gi[j]] = nview;
      if (tr.key && !has[j]) tr.key[gi[j]] = kKeyEmpty;
    }
    if (has[j]) {
      hpos[j] = local_pos<kAssignTS>(s_ck, kKeyEmpty, coarse_key(r[j]));
      if (hpos[j] < 0) { has[j] = false; atomicOr(&t.cnt->error, kErrCoarseFull); }
    }
  }
  __syncthreads();
  // (c) Sec. II.5(1)d: level of each coarse cell present in the tile
  for (int i = threadIdx.x; i < kAssignTS; i += kThreads) {
    const unsigned long long ck = s_ck[i];
    if (ck != kKeyEmpty)
      s_cl[i] = (unsigned char)level_for(coarse_count_of(t, ck), rig.n_min, rig.max_level);
  }
  __syncthreads();
  // (c) Sec. II.5(1)e: cell key and the point's offset inside its cell
  float frac[2][3];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (!has[j]) continue;
    const int l = s_cl[hpos[j]];
    const unsigned long long fk = fine_key(r[j], l);
    const int kk[3] = {(int)((fk >> 40) & 0xfffff) - kKeyBias, (int)((fk >> 20) & 0xfffff) - kKeyBias,
                       (int)(fk & 0xfffff) - kKeyBias};
#pragma unroll
    for (int a = 0; a < 3; ++a) frac[j][a] = __fsub_rn(ldexpf(r[j][a], l), (float)kk[a]);
    hpos[j] = local_pos<kAssignTS>(s_fk, kKeyEmpty, fk);
    if (hpos[j] < 0) { has[j] = false; atomicOr(&t.cnt->error, kErrFineFull); }
    if (trace && tr.key) tr.key[gi[j]] = has[j] ? fk : kKeyEmpty;
  }
  __syncthreads();
  // compact the tile's cells: entry index per hash position
  for (int i = threadIdx.x; i < kAssignTS; i += kThreads) {
    const unsigned long long fk = s_fk[i];
    if (fk == kKeyEmpty) continue;
    const int e = (int)atomicAdd(&s_n, 1u);
    s_fi[i] = e;
    s_ek[e] = fk;
    s_cnt[e] = 0u;
    s_cmax[e] = 0u;
    s_gmin[e] = 0xffffffffu;
    s_min[e] = INT_MAX;
#pragma unroll
    for (int a = 0; a < 14; ++a) s_acc[a * kAssignNL + e] = 0u;
  }
  __syncthreads();
  // (d) Sec. II.5(2)a: members, largest C, smallest weight exponent
  int ent[2] = {0, 0};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (!has[j]) continue;
    ent[j] = s_fi[hpos[j]];
    atomicAdd(&s_cnt[ent[j]], 1u);
    atomicMax(&s_cmax[ent[j]], cord[j]);
    atomicMin(&s_min[ent[j]], mexp[j]);
  }
  __syncthreads();
  // representative: lowest pixel index among the largest C; Eq. 11 sums at the tile's
  // scale 2^-(36 + mmin_tile), each 64-bit term split in two native 32-bit atomics
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (!has[j]) continue;
    const int e = ent[j];
    if (cord[j] == s_cmax[e]) atomicMin(&s_gmin[e], (unsigned)gi[j]);
    const int sh = mexp[j] - s_min[e];
    const float w = sh > 62 ? 0.0f : ldexpf(mu[j], kFixShift - sh);
    const uint8_t* px = col + 3 * li[j];
    unsigned long long q[7];
    q[0] = __float2ull_rn(w);
#pragma unroll
    for (int a = 0; a < 3; ++a) q[1 + a] = __float2ull_rn(__fmul_rn(w, frac[j][a]));
#pragma unroll
    for (int a = 0; a < 3; ++a) q[4 + a] = __float2ull_rn(__fmul_rn(w, (float)px[a] * 0.00390625f));
#pragma unroll
    for (int a = 0; a < 7; ++a) {
      atomicAdd(&s_acc[(2 * a) * kAssignNL + e], (unsigned)(q[a] & ((1ull << kLoBits) - 1ull)));
      atomicAdd(&s_acc[(2 * a + 1) * kAssignNL + e], (unsigned)(q[a] >> kLoBits));
    }
  }
  __syncthreads();
  // one partial record per (tile, cell), pushed onto the cell's list
  const unsigned n_local = s_n;
  if (threadIdx.x == 0) s_base = atomicAdd(&t.cnt->n_partials, n_local);
  __syncthreads();
  for (int e = threadIdx.x; e < (int)n_local; e += kThreads) {
    const unsigned slot = fine_insert(t, s_ek[e]);
    const unsigned pi = s_base + (unsigned)e;
    if (slot == kSlotNone) continue;
    if (pi >= t.max_partials) { atomicOr(&t.cnt->error, kErrPartials); continue; }
    Partial p;
    p.count = s_cnt[e];
    p.mmin = s_min[e];
    p.pad = 0u;
    p.rep = ((unsigned long long)s_cmax[e] << 32) | (unsigned)(~s_gmin[e]);
#pragma unroll
    for (int a = 0; a < 7; ++a)
      p.s[a] = ((unsigned long long)s_acc[(2 * a + 1) * kAssignNL + e] << kLoBits) +
               s_acc[(2 * a) * kAssignNL + e];
    p.next = atomicExch(&t.fhead[slot], pi);
    t.part[pi] = p;
  }
}

// ------------------------------------------------------------------ reduce step
__global__ void __launch_bounds__(kThreads) k_reduce(Tables t, OutDev out) {
  const unsigned n_cells = min(t.cnt->n_cells, t.fmask + 1u);
  const unsigned n_coarse = min(t.cnt->n_coarse, t.cmask + 1u);
  const unsigned n_part = min(t.cnt->n_partials, t.max_partials);
  const unsigned n = max(n_cells, n_coarse);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < n_cells) {
      const unsigned slot = t.fused[i];
      const unsigned long long key = t.fkey[slot];
      const unsigned head = t.fhead[slot];
      unsigned count = 0u, steps = 0u;
      unsigned long long rep = 0ull;
      int mmin = INT_MAX;
      for (unsigned p = head; p != kSlotNone && steps <= n_part; p = t.part[p].next, ++steps) {
        const Partial& P = t.part[p];
        count += P.count;
        rep = max(rep, P.rep);
        mmin = min(mmin, P.mmin);
      }
      unsigned long long S[7] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
      steps = 0u;
      for (unsigned p = head; p != kSlotNone && steps <= n_part; p = t.part[p].next, ++steps) {
        const Partial& P = t.part[p];
        const int sh = P.mmin - mmin;
#pragma unroll
        for (int a = 0; a < 7; ++a) S[a] += sh < 64 ? (P.s[a] >> sh) : 0ull;
      }
      if (steps > n_part) atomicOr(&t.cnt->error, kErrList);
      const unsigned g = head != kSlotNone ? ~(unsigned)(rep & 0xffffffffull) : 0xffffffffu;
      CellOut c;
      const int l = (int)(key >> 60);
      const double edge = ldexp(out.s0_m, -l);
      const double kx = (double)((int)((key >> 40) & 0xfffff) - kKeyBias);
      const double ky = (double)((int)((key >> 20) & 0xfffff) - kKeyBias);
      const double kz = (double)((int)(key & 0xfffff) - kKeyBias);
      const double Wq = (double)S[0];
      const double inv = S[0] ? 1.0 / Wq : __longlong_as_double(0x7ff8000000000000ll);
      c.pos[0] = (float)(edge * (kx + (double)S[1] * inv));
      c.pos[1] = (float)(edge * (ky + (double)S[2] * inv));
      c.pos[2] = (float)(edge * (kz + (double)S[3] * inv));
      c.rgb[0] = (float)(256.0 * (double)S[4] * inv);
      c.rgb[1] = (float)(256.0 * (double)S[5] * inv);
      c.rgb[2] = (float)(256.0 * (double)S[6] * inv);
      c.weight = (float)ldexp(Wq, -kFixShift - mmin);
      c.count = count;
      c.rep = g;
      c.pad = 0u;
      c.key = key;
      t.staged[i] = c;
      if (head != kSlotNone) atomicOr(&t.bitmap[g >> 5], 1u << (g & 31));
      t.fkey[slot] = kKeyEmpty;                 // ready for the next frame
      t.fhead[slot] = kSlotNone;
    }
    if (i < n_coarse) {
      const unsigned cs = t.cused[i];
      t.ckey[cs] = kKeyEmpty;
      t.ccount[cs] = 0u;
    }
  }
}

// ------------------------------------------------------------------ scan + stats
__device__ __forceinline__ unsigned block_excl_scan_1024(unsigned v, unsigned* s_w, unsigned& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned w = s_w[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_w[lane] = w;
  }
  __syncthreads();
  total = s_w[31];
  const unsigned before = warp ? s_w[warp - 1] : 0u;
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(1024) k_scan_words(Tables t) {
  __shared__ unsigned s_w[32];
  const long long w = (long long)blockIdx.x * 1024 + threadIdx.x;
  const unsigned v = (w < t.n_words) ? __popc(t.bitmap[w]) : 0u;
  unsigned total;
  const unsigned ex = block_excl_scan_1024(v, s_w, total);
  if (w < t.n_words) t.wprefix[w] = ex;
  if (threadIdx.x == 0) t.bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_blocks(Tables t, OutDev out) {
  __shared__ unsigned s_w[32];
  unsigned carry = 0;
  for (int base = 0; base < t.n_wblocks; base += 1024) {
    const int i = base + threadIdx.x;
    const unsigned v = (i < t.n_wblocks) ? t.bsum[i] : 0u;
    unsigned total;
    const unsigned ex = block_excl_scan_1024(v, s_w, total);
    if (i < t.n_wblocks) t.bsum[i] = carry + ex;
    carry += total;
  }
  // frame statistics from the per-block partials of the count step
  unsigned long long nv = 0, ng = 0, noor = 0;
  unsigned bmin[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, bmax[3] = {0u, 0u, 0u};
  for (int i = threadIdx.x; i < t.n_bstats; i += 1024) {
    const BlockStats b = t.bstats[i];
    nv += b.n_valid;
    ng += b.n_gated;
    noor += b.n_oor;
    for (int k = 0; k < 3; ++k) { bmin[k] = min(bmin[k], b.bmin[k]); bmax[k] = max(bmax[k], b.bmax[k]); }
  }
  __shared__ unsigned long long s_l[3][32];
  __shared__ unsigned s_b[6][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    nv += __shfl_xor_sync(0xffffffffu, nv, o);
    ng += __shfl_xor_sync(0xffffffffu, ng, o);
    noor += __shfl_xor_sync(0xffffffffu, noor, o);
  }
  for (int k = 0; k < 3; ++k) {
    bmin[k] = __reduce_min_sync(0xffffffffu, bmin[k]);
    bmax[k] = __reduce_max_sync(0xffffffffu, bmax[k]);
  }
  if (lane == 0) {
    s_l[0][warp] = nv; s_l[1][warp] = ng; s_l[2][warp] = noor;
    for (int k = 0; k < 3; ++k) { s_b[k][warp] = bmin[k]; s_b[3 + k][warp] = bmax[k]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    fuseflow_stats st = {};
    unsigned mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
    for (int w = 0; w < 32; ++w) {
      st.n_valid += (int64_t)s_l[0][w];
      st.n_gated += (int64_t)s_l[1][w];
      st.n_out_of_range += (int64_t)s_l[2][w];
      for (int k = 0; k < 3; ++k) { mn[k] = min(mn[k], s_b[k][w]); mx[k] = max(mx[k], s_b[3 + k][w]); }
    }
    const unsigned nc = t.cnt->n_cells;
    unsigned err = t.cnt->error;
    if ((long long)nc > out.max_cells) err |= kErrCells;
    if (t.cnt->n_partials > t.max_partials) err |= kErrPartials;
    st.n_cells = (int64_t)(nc < out.max_cells ? nc : out.max_cells);
    for (int k = 0; k < 3; ++k) {
      st.bbox[k] = st.n_gated ? (float)((double)from_ordered(mn[k]) * out.unit_m) : __int_as_float(0x7f800000);
      st.bbox[3 + k] = st.n_gated ? (float)((double)from_ordered(mx[k]) * out.unit_m) : __int_as_float(0xff800000);
    }
    st.error = (int32_t)err;
    st.n_coarse = (int32_t)t.cnt->n_coarse;
    *out.stats = st;
  }
}

// ------------------------------------------------------------------ emit
__global__ void __launch_bounds__(kThreads) k_emit(Tables t, OutDev out) {
  const unsigned n_cells = min(t.cnt->n_cells, t.fmask + 1u);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n_cells; i += gridDim.x * blockDim.x) {
    const CellOut c = t.staged[i];
    const unsigned g = c.rep;
    if ((long long)g >= t.n_words * 32) continue;          // cell without partials (overflow)
    const unsigned w = g >> 5;
    if (!((t.bitmap[w] >> (g & 31)) & 1u)) continue;
    const unsigned long long rnk = (unsigned long long)t.bsum[w >> 10] + t.wprefix[w] +
                                   __popc(t.bitmap[w] & ((1u << (g & 31)) - 1u));
    if (rnk >= (unsigned long long)out.max_cells) continue;
    out.pos[3 * rnk + 0] = c.pos[0];
    out.pos[3 * rnk + 1] = c.pos[1];
    out.pos[3 * rnk + 2] = c.pos[2];
    out.rgb[3 * rnk + 0] = c.rgb[0];
    out.rgb[3 * rnk + 1] = c.rgb[1];
    out.rgb[3 * rnk + 2] = c.rgb[2];
    out.weight[rnk] = c.weight;
    out.count[rnk] = c.count;
    out.rep[rnk] = g;
    out.key[rnk] = c.key;
  }
}

__global__ void k_init_tables(Tables t, unsigned fcap, unsigned ccap) {
  const unsigned n = max(fcap, ccap);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < fcap) {
      t.fkey[i] = kKeyEmpty;
      t.fhead[i] = kSlotNone;
    }
    if (i < ccap) {
      t.ckey[i] = kKeyEmpty;
      t.ccount[i] = 0u;
    }
  }
}

template <typename DT>
cudaError_t launch_typed(const RigDev* rig, const float2* rays, const FramePtrs& fp, const Tables& t,
                         const TraceDev& tr, const OutDev& out, const Geometry& geo, cudaStream_t s,
                         cudaEvent_t* ev) {
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(k_assign<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kAssignSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], s); };
  mark(0);
  cudaError_t err = cudaMemsetAsync(t.cnt, 0, sizeof(FrameCounters) + sizeof(unsigned) * (size_t)t.n_words, s);
  if (err != cudaSuccess) return err;
  mark(1);
  k_count<DT><<<dim3(geo.count_blocks_x, geo.n_cams), kThreads, 0, s>>>(rig, rays, fp, t, geo.count_blocks_x);
  mark(2);
  k_assign<DT><<<dim3(geo.tiles_max, geo.n_cams), kThreads, kAssignSmem, s>>>(rig, rays, fp, t, tr,
                                                                                (float)out.unit_m);
  mark(3);
  k_reduce<<<geo.emit_blocks, kThreads, 0, s>>>(t, out);
  mark(4);
  k_scan_words<<<t.n_wblocks, 1024, 0, s>>>(t);
  k_scan_blocks<<<1, 1024, 0, s>>>(t, out);
  mark(5);
  k_emit<<<geo.emit_blocks, kThreads, 0, s>>>(t, out);
  mark(6);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init_tables(const Tables& t, unsigned fcap, unsigned ccap, cudaStream_t s) {
  k_init_tables<<<1024, 256, 0, s>>>(t, fcap, ccap);
  return cudaGetLastError();
}

cudaError_t launch_frame(const RigDev* rig, const float2* rays, const FramePtrs& fp, const Tables& t,
                         const TraceDev& tr, const OutDev& out, const Geometry& geo, cudaStream_t s,
                         cudaEvent_t* ev) {
  if (geo.depth_f32) return launch_typed<float>(rig, rays, fp, t, tr, out, geo, s, ev);
  return launch_typed<uint16_t>(rig, rays, fp, t, tr, out, geo, s, ev);
}

}  // namespace ffl
