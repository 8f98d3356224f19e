// ff_kernels.cu - sm_103a kernels of the FUSE-Flow per-frame fusion path.
//
// Launch sequence of one frame (all on the caller's stream; from the level step on,
// optionally as programmatic dependent launches, see pdl_release / pdl_wait):
//   memset   frame counters + representative bitmap
//   screen   (only with a depth screen set) D^r of Eq. 8 into the context's buffers
//   count    (a) decode + gate + back-project (Eq. 8, 9), coarse density n_c (Sec. II.5(1)c)
//            from equal-cell runs merged across each warp, per-block pixel counts and
//            extent (Sec. II.5(1)b)
//   levels   level of each coarse cell (Sec. II.5(1)d) and its range of 8^level dense
//            cell slots
//   assign   per 32x16 tile: (b) consistency V (Eq. 4-7) in double-float, omega = C V
//            (Eq. 10) as mantissa/exponent; (c) cell key (Sec. II.5(1)e) and dense slot;
//            (d) per (tile, cell): member count, representative (Sec. II.5(2)a), smallest
//            weight exponent and exact fixed-point sums of omega, omega P, omega RGB
//            (Eq. 11), written as one partial record pushed onto its cell's list
//   reduce   per cell: walk its partials, combine them, stage the fused cell, mark its
//            representative; the used slots and coarse entries are cleared for the next frame
//            (top-k variant: k_reduce_topk weighs and fuses each cell's k most confident
//            members here instead)
//   scan     ranks of the representatives (output order) and frame statistics
//   emit     fused cells in representative order
// Outside the frame sequence: k_copyout (served frames: cloud into pinned host memory),
// k_mc (the multi-camera depth consistency error of Eq. 12 on a point set), k_confidence
// (Eq. 3 confidence from depth) and the stand-alone depth screen.
//
// Every reduction of the frame is order-independent (integer counts, max, min and
// fixed-point sums), so its output is bitwise reproducible.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdint>

#include "ff_internal.h"

namespace ffl {

namespace {

constexpr int kThreads = 256;
constexpr int kCountPx = 8;                       // pixels per thread in the count step
constexpr int kCountBlockPx = kThreads * kCountPx;
constexpr int kTileW = 32;                        // assign tile: 32 columns by TH rows
constexpr int kMaxProbe = 1 << 14;
constexpr float kLn2H = 0.693147182464599609375f;         // float(ln 2)
constexpr float kLn2L = -1.904654299957768e-09f;          // ln 2 - kLn2H
constexpr float kInvLn2 = 1.44269504088896340736f;

// ------------------------------------------------------------------ global hash tables
__device__ __forceinline__ unsigned coarse_insert(const Tables& t, unsigned long long key) {
  unsigned h = (unsigned)mix64(key) & t.cmask;
  for (int probe = 0; probe < kMaxProbe; ++probe) {
    // one round trip per probe: the swap either claims an empty slot or reports its key
    const unsigned long long cur = atomicCAS(&t.coarse[h].key, kKeyEmpty, key);
    if (cur == kKeyEmpty) {
      const unsigned n = atomicAdd(&t.cnt->n_coarse, 1u);
      if (n <= t.cmask) t.cused[n] = h;
      return h;
    }
    if (cur == key) return h;
    h = (h + 1) & t.cmask;
  }
  atomicOr(&t.cnt->error, kErrCoarseFull);
  return kSlotNone;
}

// Level and slot base (packed level << 27 | base) of an existing coarse key, continuing a
// probe whose first record `e` (at position h) was loaded earlier.
__device__ __forceinline__ unsigned coarse_lvbase(const Tables& t, unsigned long long key,
                                                  unsigned h, ulonglong2 e) {
  for (int probe = 0; probe < kMaxProbe; ++probe) {
    if (e.x == key) return (unsigned)(e.y >> 32);
    if (e.x == kKeyEmpty) break;
    h = (h + 1) & t.cmask;
    e = __ldcg(reinterpret_cast<const ulonglong2*>(&t.coarse[h]));
  }
  atomicOr(&t.cnt->error, kErrCoarseMiss);
  return kBaseNone;
}

// Sec. II.5(1)d for every coarse cell once all counts are in: its level l and a range of
// 8^l dense cell slots.  Ranges are claimed with one atomic per warp (an inclusive scan of
// the sizes inside the warp), so their placement depends on scheduling; no result does.
// Programmatic dependent launch between the kernels of one frame: each kernel lets the next
// one start launching as soon as all of its own blocks are running (pdl_release), and a
// kernel waits for the previous one to complete, its memory visible, before it touches
// anything that one (or any earlier kernel of the frame) wrote (pdl_wait).  Outside such a
// launch both are no-ops.
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Frame of a block of a one-dimensional grid that concatenates the frames' blocks
// (first[f] = the frame's first block), and the block's index within its frame.
template <int NB>
__device__ __forceinline__ int batch_frame(const int (&first)[NB + 1], int n, int b, int& local) {
  int f = 0;
#pragma unroll
  for (int k = 1; k < NB; ++k)
    if (k < n && b >= first[k]) f = k;
  local = b - first[f];
  return f;
}
// Frame of a block of a grid whose y dimension runs over the frames.
template <int NB>
__device__ __forceinline__ int batch_frame_y() { return NB == 1 ? 0 : (int)blockIdx.y; }

template <int NB>
__global__ void __launch_bounds__(kThreads) k_levels(const __grid_constant__ BatchArgs<NB> args) {
  const Tables& t = args.f[batch_frame_y<NB>()].t;
  pdl_release();
  pdl_wait();
  const unsigned n_coarse = min(t.cnt->n_coarse, t.cmask + 1u);
  const int lane = threadIdx.x & 31;
  const unsigned long long cap = t.max_slots;
  for (unsigned base = blockIdx.x * blockDim.x; base < n_coarse; base += gridDim.x * blockDim.x) {
    const unsigned i = base + threadIdx.x;
    unsigned cs = 0, l = 0;
    unsigned long long size = 0;
    if (i < n_coarse) {
      cs = t.cused[i];
      l = (unsigned)level_for(t.coarse[cs].count, t.n_min, t.max_level);
      size = min(1ull << (3 * l), cap + 1ull);           // 8^l, clamped: never fits then
    }
    unsigned long long x = size;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    unsigned long long wbase = 0;
    if (lane == 31 && x) wbase = atomicAdd(&t.cnt->n_slots, x);
    wbase = __shfl_sync(0xffffffffu, wbase, 31);
    if (i < n_coarse) {
      const unsigned long long b = wbase + x - size;
      const bool fits = b + size <= cap;
      t.coarse[cs].lvbase = (l << 27) | (fits ? (unsigned)b : kBaseNone);
      if (!fits) atomicOr(&t.cnt->error, kErrSlots);
    }
  }
}

// Block-local open addressing (shared memory); returns the table position or -1, and sets
// `fresh` when this call inserted the key.  32-bit keys (dense cell slots) take a
// multiplicative (Fibonacci) hash, 64-bit keys (packed coarse keys) the 64-bit mixer.
template <int TS, typename K>
__device__ __forceinline__ int local_pos(K* tab, K empty, K key, int max_probe, bool& fresh) {
  unsigned h;
  if constexpr (sizeof(K) == 4) {
    constexpr int kBits = TS == 512 ? 9 : TS == 1024 ? 10 : TS == 2048 ? 11 : TS == 4096 ? 12 : 0;
    static_assert(kBits > 0, "block table size");
    h = ((unsigned)key * 0x9E3779B1u) >> (32 - kBits);
  } else {
    h = (unsigned)mix64((unsigned long long)key) & (TS - 1);
  }
  fresh = false;
  for (int probe = 0; probe < max_probe; ++probe) {
    const K cur = *static_cast<volatile K*>(&tab[h]);
    if (cur == key) return (int)h;
    if (cur == empty) {
      const K prev = atomicCAS(&tab[h], empty, key);
      fresh = prev == empty;
      if (fresh || prev == key) return (int)h;
    }
    h = (h + 1) & (TS - 1);
  }
  return -1;
}
template <int TS, typename K>
__device__ __forceinline__ int local_pos(K* tab, K empty, K key, int max_probe = TS) {
  bool fresh;
  return local_pos<TS>(tab, empty, key, max_probe, fresh);
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
// A pixel at z-depth z; the transform into view j (Eq. 4) uses the pixel's separable pair
// rays (from the tile's shared-memory copy or the global tables), so that
// a = z (A(x) + B(y)) + t_ji costs one ff sum, one ff product and one ff sum per component.
// Views go in groups of kViewGroup: every view of a group is projected and its depth gather
// issued before any residual is formed.  Groups of one measure fastest on GB300 (larger
// groups spill at four blocks per SM and grow the code past the instruction cache).
constexpr int kViewGroup = 1;

// Pair rays of a tile of TH rows staged in shared memory (pixel (lx, ly) of the tile): per
// view, A of the 32 columns and B of the TH rows, each as two float4 planes.
template <int TH>
struct TilePairRays {
  const float4* s_pr;
  int lx, ly;
  __device__ __forceinline__ void operator()(int q, const PairDev&, float4& a01, float4& a2,
                                             float4& b01, float4& b2) const {
    const float4* pr = s_pr + q * (2 * kTileW + 2 * TH);
    a01 = pr[lx];
    a2 = pr[kTileW + lx];
    b01 = pr[2 * kTileW + ly];
    b2 = pr[2 * kTileW + TH + ly];
  }
};

// Pair rays read from the global tables (pixel (x, y) of the camera).
struct GlobalPairRays {
  const float4* pray;
  int x, y;
  __device__ __forceinline__ void operator()(int, const PairDev& P, float4& a01, float4& a2,
                                             float4& b01, float4& b2) const {
    a01 = __ldg(pray + P.ga + 2 * x);
    a2 = __ldg(pray + P.ga + 2 * x + 1);
    b01 = __ldg(pray + P.gb + 2 * y);
    b2 = __ldg(pray + P.gb + 2 * y + 1);
  }
};

template <typename DT, typename PR>
__device__ __forceinline__ void residual_sum(const BlockConst& bc, int k1, const PR& prays,
                                             const float2* __restrict__ rays,
                                             const FramePtrs& fp, float z,
                                             float& sh, float& sl, int& nview) {
  sh = 0.0f;
  sl = 0.0f;
  nview = 0;
  for (int q0 = 0; q0 < k1; q0 += kViewGroup) {
    float ah[kViewGroup][3], al[kViewGroup][3];
    int px[kViewGroup], py[kViewGroup];
    DT Dj[kViewGroup];
    bool ok[kViewGroup];
    // Eq. 4: transform, projection, nearest pixel and field-of-view test of each view
#pragma unroll
    for (int g = 0; g < kViewGroup; ++g) {
      ok[g] = false;
      px[g] = 0;
      py[g] = 0;
      Dj[g] = (DT)0;
      const int q = q0 + g;
      if (q >= k1) continue;
      const PairDev& P = bc.pair[q];
      const CamDev& J = bc.nb[q];
      float4 a01, a2, b01, b2;
      prays(q, P, a01, a2, b01, b2);
      ff_ray_affine(a01.x, a01.y, b01.x, b01.y, z, P.th[0], P.tl[0], ah[g][0], al[g][0]);
      ff_ray_affine(a01.z, a01.w, b01.z, b01.w, z, P.th[1], P.tl[1], ah[g][1], al[g][1]);
      ff_ray_affine(a2.x, a2.y, b2.x, b2.y, z, P.th[2], P.tl[2], ah[g][2], al[g][2]);
      fast_two_sum(ah[g][2], al[g][2], ah[g][2], al[g][2]);   // sign of a_z is that of ah
      if (!(ah[g][2] > 0.0f)) continue;                        // behind camera j
      // float32 estimate of u + 1/2 from the ff high parts (relative error ~1e-7, so a
      // few 1e-4 px); within kTieBandPx of a tie the pixel is decided exactly
      const float fu = __fadd_rn(__fmaf_rn(J.fx, __fdividef(ah[g][0], ah[g][2]), J.cx), 0.5f);
      const float fv = __fadd_rn(__fmaf_rn(J.fy, __fdividef(ah[g][1], ah[g][2]), J.cy), 0.5f);
      if (!(fu > -1.0f && fu < (float)J.W + 1.0f && fv > -1.0f && fv < (float)J.H + 1.0f))
        continue;
      const float ru = rintf(fu), rv = rintf(fv);
      px[g] = fabsf(fu - ru) < kTieBandPx
                  ? exact_round(J.fxh, J.fxl, J.cxh, J.cxl, ah[g][0], al[g][0], ah[g][2], al[g][2], ru)
                  : (int)floorf(fu);
      py[g] = fabsf(fv - rv) < kTieBandPx
                  ? exact_round(J.fyh, J.fyl, J.cyh, J.cyl, ah[g][1], al[g][1], ah[g][2], al[g][2], rv)
                  : (int)floorf(fv);
      if (px[g] < 0 || px[g] >= J.W || py[g] < 0 || py[g] >= J.H) continue;
      Dj[g] = __ldg(static_cast<const DT*>(fp.depth[P.j]) + (long long)py[g] * J.W + px[g]);
      ok[g] = true;
    }
    // Eq. 5-6 for the views whose gathered depth is valid
#pragma unroll
    for (int g = 0; g < kViewGroup; ++g) {
      if (!ok[g] || !Depth<DT>::valid(Dj[g])) continue;
      const CamDev& J = bc.nb[q0 + g];
      // Q = D_j(u_j) (rx_j, ry_j, 1) in camera-j coordinates (rigid motion keeps d)
      const float zj = Depth<DT>::z(Dj[g]);
      const float2 qx = __ldg(rays + J.ray_x + px[g]), qy = __ldg(rays + J.ray_y + py[g]);
      float qh[3], ql[3];
      two_prod(zj, qx.x, qh[0], ql[0]);
      ql[0] = __fmaf_rn(zj, qx.y, ql[0]);
      two_prod(zj, qy.x, qh[1], ql[1]);
      ql[1] = __fmaf_rn(zj, qy.y, ql[1]);
      qh[2] = zj;
      ql[2] = 0.0f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {                    // d^2 = |a - Q|^2 in ff
        float s, e, p, pe, tt;
        two_sum(ah[g][k], -qh[k], s, e);
        e = __fadd_rn(e, __fsub_rn(al[g][k], ql[k]));
        // (s + e)^2 = s^2 + 2 s e + e^2; e^2 is below the ff rounding of the sum
        two_prod(s, s, p, pe);
        pe = __fmaf_rn(__fmul_rn(2.0f, s), e, pe);
        two_sum(sh, p, sh, tt);
        sl = __fadd_rn(sl, __fadd_rn(tt, pe));
      }
      ++nview;
    }
  }
}

// Eq. 7 and 10 from the residual sum (sh, sl): omega = C' exp(-e) = mu 2^-m with
// e = m ln 2 + f, f in [0, ln 2), so that mu never underflows (C' = C, or 1 without the
// confidence term).  Returns e (high part) for traces.
__device__ __forceinline__ float joint_weight(const RigDev& rig, int k1, float sh, float sl,
                                              float c, float& mu, int& m) {
  float eh = 0.0f, el = 0.0f;
  if (rig.use_cons && k1 > 0) {
    fast_two_sum(sh, sl, sh, sl);
    two_prod(sh, rig.einv_h, eh, el);                                  // Eq. 7 exponent
    el = __fmaf_rn(sh, rig.einv_l, __fmaf_rn(sl, rig.einv_h, el));
    fast_two_sum(eh, el, eh, el);
  }
  m = 0;
  float fh = eh, fl = el;
  if (eh > 0.0f) {
    m = (int)floorf(__fmul_rn(fminf(eh, 1.0e9f), kInvLn2));
    const float mf = (float)m;
    float p, pe;
    two_prod(mf, kLn2H, p, pe);
    fh = __fsub_rn(eh, p);
    fl = __fsub_rn(__fsub_rn(el, pe), __fmul_rn(mf, kLn2L));
  }
  const float base = rig.use_conf ? c : 1.0f;                          // Eq. 10
  mu = __fmul_rn(__fmul_rn(base, expf(-fh)), __fsub_rn(1.0f, fl));
  return eh;
}

// ------------------------------------------------------------------ count step
template <typename DT>
__device__ __forceinline__ void load8(const DT* __restrict__ d, const float* __restrict__ c,
                                      long long p0, long long npx, DT dv[8], float cv[8]) {
  const bool full = p0 + 7 < npx;
  if constexpr (sizeof(DT) == 2) {
    if (full && ((reinterpret_cast<uintptr_t>(d + p0) & 15) == 0)) {
      const uint4 u = __ldg(reinterpret_cast<const uint4*>(d + p0));
      const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) { dv[2 * k] = (DT)(w[k] & 0xffff); dv[2 * k + 1] = (DT)(w[k] >> 16); }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) dv[k] = (p0 + k < npx) ? d[p0 + k] : (DT)0;
    }
  } else {
    if (full && ((reinterpret_cast<uintptr_t>(d + p0) & 15) == 0)) {
      const float4 f0 = __ldg(reinterpret_cast<const float4*>(d + p0));
      const float4 f1 = __ldg(reinterpret_cast<const float4*>(d + p0) + 1);
      dv[0] = f0.x; dv[1] = f0.y; dv[2] = f0.z; dv[3] = f0.w;
      dv[4] = f1.x; dv[5] = f1.y; dv[6] = f1.z; dv[7] = f1.w;
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) dv[k] = (p0 + k < npx) ? d[p0 + k] : (DT)0;
    }
  }
  if (full && ((reinterpret_cast<uintptr_t>(c + p0) & 15) == 0)) {
    const float4 f0 = __ldg(reinterpret_cast<const float4*>(c + p0));
    const float4 f1 = __ldg(reinterpret_cast<const float4*>(c + p0) + 1);
    cv[0] = f0.x; cv[1] = f0.y; cv[2] = f0.z; cv[3] = f0.w;
    cv[4] = f1.x; cv[5] = f1.y; cv[6] = f1.z; cv[7] = f1.w;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) cv[k] = (p0 + k < npx) ? c[p0 + k] : 0.0f;
  }
}

// Adds n points to coarse key k: the block table while it is at most 3/4 full (so that
// probe runs stay short), else, or after 32 probes, the global table directly.
template <int TS>
__device__ __forceinline__ void count_add(const Tables& t, unsigned long long* s_key,
                                          unsigned* s_cnt, unsigned* s_fill,
                                          unsigned long long k, unsigned n) {
  int h = -1;
  if (*static_cast<volatile unsigned*>(s_fill) < 3u * TS / 4u) {
    bool fresh;
    h = local_pos<TS>(s_key, kKeyEmpty, k, 32, fresh);
    if (fresh) atomicAdd(s_fill, 1u);
  }
  if (h >= 0) {
    atomicAdd(&s_cnt[h], n);
  } else {
    const unsigned slot = coarse_insert(t, k);
    if (slot != kSlotNone) atomicAdd(&t.coarse[slot].count, n);
  }
}

template <typename DT, int NB>
__global__ void __launch_bounds__(kThreads, 4) k_count(const __grid_constant__ BatchArgs<NB> args) {
  int local;
  const FrameArgs& fa = args.f[batch_frame<NB>(args.count_first, args.n, (int)blockIdx.x, local)];
  const RigDev* __restrict__ rigp = fa.rig;
  const float2* __restrict__ rays = fa.rays;
  const FramePtrs& fp = fa.fp;
  const Tables& t = fa.t;
  const int blocks_x = fa.count_blocks_x, chunks = fa.count_chunks;
  const int cam = local / blocks_x, bx = local - cam * blocks_x;
  pdl_release();
  constexpr int TS = 2048;                                      // block table of coarse keys
  __shared__ unsigned long long s_key[TS];
  __shared__ unsigned s_cnt[TS];
  __shared__ unsigned s_fill;                                    // keys in the block table
  __shared__ unsigned short s_occ[TS];                           // occupied positions, packed
  // the packing loop below walks the table in whole warps (every lane reaches the ballot)
  // and stores positions as 16-bit values
  static_assert(TS % kThreads == 0 && kThreads % 32 == 0 && TS <= 65536, "block table shape");
  __shared__ unsigned s_nocc;
  __shared__ unsigned s_red[kThreads / 32][9];
  // per warp, the runs its lanes send to the block table in a chunk (at most one per run,
  // kCountPx a lane), inserted by the whole warp at once; the counts share the storage of
  // s_occ, which only the final flush uses
  constexpr int kRunCap = 32 * kCountPx;
  static_assert((kThreads / 32) * kRunCap <= TS, "run counts fit in s_occ");
  __shared__ unsigned long long s_mk[kThreads / 32][kRunCap];
  unsigned short* const s_mn = s_occ + (threadIdx.x >> 5) * kRunCap;
  __shared__ unsigned s_mcount[kThreads / 32];
  const RigDev& rig = *rigp;
  // the camera's constants and the rig's scalars in registers (they would otherwise be
  // re-read for every pixel, as the atomics below may alias memory for the compiler)
  const CamDev C = rig.cam[cam];
  const float tau = rig.tau, inv_s0u = rig.inv_s0u;
  const int use_conf = rig.use_conf, lim = kKeyBias >> rig.max_level;
  const long long npx = (long long)C.W * C.H;
  const int bid = cam * blocks_x + bx;
  const long long c0 = (long long)bx * chunks;                  // first chunk of 2048 pixels
  const bool idle = c0 * kCountBlockPx >= npx;                  // uniform over the block
  for (int i = threadIdx.x; i < TS; i += kThreads) { s_key[i] = kKeyEmpty; s_cnt[i] = 0; }
  if (threadIdx.x == 0) { s_fill = 0u; s_nocc = 0u; }
  if (threadIdx.x < kThreads / 32) s_mcount[threadIdx.x] = 0u;
  __syncthreads();

  const DT* __restrict__ dep = static_cast<const DT*>(fp.depth[cam]);
  const float* __restrict__ cf = fp.conf[cam];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned nv = 0, ng = 0, noor = 0;
  float fmn[3] = {__int_as_float(0x7f800000), __int_as_float(0x7f800000), __int_as_float(0x7f800000)};
  float fmx[3] = {__int_as_float(0xff800000), __int_as_float(0xff800000), __int_as_float(0xff800000)};
  long long pn = (c0 * kThreads + threadIdx.x) * kCountPx;
  int y = (int)((unsigned)pn / (unsigned)C.W);                  // W H <= 2^30
  int x = (int)((unsigned)pn - (unsigned)y * (unsigned)C.W);
  // no prefetch of the next chunk: registers stay under 64, and four resident blocks per
  // SM hide the load latency better than a second set of eight samples per thread did
  for (int ch = 0; ch < (idle ? 0 : chunks); ++ch) {
    const long long pc = pn;
    if ((c0 + ch) * kCountBlockPx >= npx) break;                 // uniform over the block
    DT dcur[kCountPx];
    float ccur[kCountPx];
    if (pc < npx) load8<DT>(dep, cf, pc, npx, dcur, ccur);
    pn = pc + kCountBlockPx;
    // Sec. II.5(1)c density estimate. Runs of equal coarse cells along the thread's
    // pixels: the first run (if the thread has several) and the last run are kept for the
    // merge along the warp, the ones between are staged for the warp's insertion pass (a
    // block-table insertion in the unrolled loop itself would run once per unrolled pixel
    // for the whole warp whenever any lane ends a run there).
    unsigned long long khead = kKeyEmpty, ktail = kKeyEmpty;
    unsigned nhead = 0u, run = 0u, nruns = 0u;
    int cx = 0, cy = 0, cz = 0;
    if (pc < npx) {
      // the pixels' ray components: one row and 16-byte aligned rays (every rig whose
      // widths are multiples of 8) take four vector loads, other groups one load per pixel
      float rxk[kCountPx], ryk[kCountPx];
      if (x + kCountPx <= C.W && ((C.ray_x + x) & 1) == 0) {
        const float4* r4 = reinterpret_cast<const float4*>(rays + C.ray_x + x);
#pragma unroll
        for (int k = 0; k < kCountPx / 2; ++k) {
          const float4 v = __ldg(r4 + k);
          rxk[2 * k] = v.x;
          rxk[2 * k + 1] = v.z;
        }
        const float ry = __ldg(&rays[C.ray_y + y].x);
#pragma unroll
        for (int k = 0; k < kCountPx; ++k) ryk[k] = ry;
      } else {
        int xx = x, yy = y;
#pragma unroll
        for (int k = 0; k < kCountPx; ++k) {
          rxk[k] = __ldg(&rays[C.ray_x + xx].x);
          ryk[k] = __ldg(&rays[C.ray_y + min(yy, C.H - 1)].x);
          if (++xx == C.W) { xx = 0; ++yy; }
        }
      }
      // branch-free per pixel: every lane evaluates every pixel, predicates select
#pragma unroll
      for (int k = 0; k < kCountPx; ++k) {
        const bool valid = pc + k < npx && Depth<DT>::valid(dcur[k]);
        const bool gated = valid && (!use_conf || ccur[k] > tau);  // Eq. 9
        nv += valid ? 1u : 0u;
        ng += gated ? 1u : 0u;
        float P[3];
        world_point(C, valid ? Depth<DT>::z(dcur[k]) : 0.0f, rxk[k], ryk[k], P);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          fmn[a] = gated ? fminf(fmn[a], P[a]) : fmn[a];
          fmx[a] = gated ? fmaxf(fmx[a], P[a]) : fmx[a];
        }
        // coarse coordinates floor(P / s0); the finest index floor(r 2^Lmax) is in
        // [-2^19, 2^19) exactly when floor(r) is in [-2^(19-Lmax), 2^(19-Lmax))
        const int ix = (int)floorf(__fmul_rn(P[0], inv_s0u));
        const int iy = (int)floorf(__fmul_rn(P[1], inv_s0u));
        const int iz = (int)floorf(__fmul_rn(P[2], inv_s0u));
        const bool inr = (unsigned)(ix + lim) < (unsigned)(2 * lim) &&
                         (unsigned)(iy + lim) < (unsigned)(2 * lim) &&
                         (unsigned)(iz + lim) < (unsigned)(2 * lim);
        noor += (gated && !inr) ? 1u : 0u;
        const bool counted = gated && inr;
        const bool same = run && ix == cx && iy == cy && iz == cz;
        if (counted && !same && run) {                            // a run ends
          if (nruns == 1u) {
            khead = pack_key(0, cx, cy, cz);
            nhead = run;
          } else {
            const unsigned q = atomicAdd(&s_mcount[warp], 1u);
            s_mk[warp][q] = pack_key(0, cx, cy, cz);
            s_mn[q] = (unsigned short)run;
          }
        }
        if (counted) {
          run = same ? run + 1u : 1u;
          nruns += same ? 0u : 1u;
          cx = ix;
          cy = iy;
          cz = iz;
        }
      }
    }
    {
      if (run) ktail = pack_key(0, cx, cy, cz);
      // merge the lanes' runs along the warp (consecutive lanes hold consecutive pixels):
      // a lane's first run continues the previous lane's last run when the keys agree
      const unsigned long long kfirst = nruns >= 2u ? khead : ktail;
      const unsigned long long kprev = __shfl_up_sync(0xffffffffu, ktail, 1);
      const bool cont = lane > 0 && ktail != kKeyEmpty && kfirst == kprev;
      // a continuing head run is credited to the previous lane's chain
      const unsigned give = (cont && nruns >= 2u) ? nhead : 0u;
      unsigned v = run + __shfl_down_sync(0xffffffffu, give, 1) * (lane < 31 ? 1u : 0u);
      bool start = !(cont && nruns == 1u);
      const bool nstart = __shfl_down_sync(0xffffffffu, (unsigned)start, 1) != 0u;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {                          // segmented inclusive scan
        const unsigned v2 = __shfl_up_sync(0xffffffffu, v, d);
        const bool f2 = __shfl_up_sync(0xffffffffu, (unsigned)start, d) != 0u;
        if (lane >= d) {
          if (!start) v += v2;
          start = start || f2;
        }
      }
      // the lane's first run unless it continues the previous lane's chain, and its last
      // run where a chain ends, join the middle runs; then every run of the warp goes to
      // the block table, one lane each
      if (nruns >= 2u && !cont) {
        const unsigned q = atomicAdd(&s_mcount[warp], 1u);
        s_mk[warp][q] = khead;
        s_mn[q] = (unsigned short)nhead;
      }
      if (ktail != kKeyEmpty && (lane == 31 || nstart)) {
        const unsigned q = atomicAdd(&s_mcount[warp], 1u);
        s_mk[warp][q] = ktail;
        s_mn[q] = (unsigned short)v;
      }
      __syncwarp();
      const unsigned nm = s_mcount[warp];
      for (unsigned q = lane; q < nm; q += 32u) count_add<TS>(t, s_key, s_cnt, &s_fill, s_mk[warp][q], s_mn[q]);
      __syncwarp();
      if (lane == 0) s_mcount[warp] = 0u;
      __syncwarp();
    }
    x += kCountBlockPx;                                           // next chunk's first pixel
    while (x >= C.W) { x -= C.W; ++y; }
  }
  // per-block pixel counts and extent
  unsigned vals[9] = {nv, ng, noor, ordered(fmn[0]), ordered(fmn[1]), ordered(fmn[2]),
                      ordered(fmx[0]), ordered(fmx[1]), ordered(fmx[2])};
  if (ng == 0) {
    for (int a = 0; a < 3; ++a) { vals[3 + a] = 0xffffffffu; vals[6 + a] = 0u; }
  }
  vals[0] = __reduce_add_sync(0xffffffffu, vals[0]);
  vals[1] = __reduce_add_sync(0xffffffffu, vals[1]);
  vals[2] = __reduce_add_sync(0xffffffffu, vals[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    vals[3 + a] = __reduce_min_sync(0xffffffffu, vals[3 + a]);
    vals[6 + a] = __reduce_max_sync(0xffffffffu, vals[6 + a]);
  }
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < 9; ++a) s_red[warp][a] = vals[a];
  }
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
  // the block table into the global one: the occupied positions are packed first, so that a
  // thread sends at most a few of them and the global round trips of all of them overlap
  // (walking the table in strides left up to eight dependent round trips per thread)
  for (int i = threadIdx.x; i < TS; i += kThreads) {
    const bool occ = s_key[i] != kKeyEmpty;
    const unsigned m = __ballot_sync(0xffffffffu, occ);
    unsigned base = 0u;
    if (lane == 0 && m) base = atomicAdd(&s_nocc, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (occ) s_occ[base + __popc(m & ((1u << lane) - 1u))] = (unsigned short)i;
  }
  __syncthreads();
  const int n_occ = (int)s_nocc;
  for (int j = threadIdx.x; j < n_occ; j += kThreads) {
    const int i = s_occ[j];
    const unsigned slot = coarse_insert(t, s_key[i]);
    if (slot != kSlotNone) atomicAdd(&t.coarse[slot].count, s_cnt[i]);
  }
}

// ------------------------------------------------------------------ assign step
constexpr size_t align16(size_t v) { return (v + 15) / 16 * 16; }
static_assert(kMaxTopK * 8 <= 14 * 4, "a cell's top-k keys fit in its 14 split-sum words");

// The assign step's tile: 32 columns by TH rows (TH = 8, 16 or 32: a launch-geometry
// choice), one warp per two rows, two pixels a thread, and its shared-memory layout.
// Distinct cells of a tile with shared-memory accumulators: NL.  In a tile with more
// distinct cells (sparse, noisy tiles only) the cells with two or more members in the tile
// take the accumulators and every other member files a single-member partial, which is the
// record the accumulator would have produced for it; if even the multi-member cells are too
// many, every member files alone.  Both rules depend on the tile's cells alone, never on
// the order of the insertions, so that every cell's sums, and the fused cloud, are bitwise
// reproducible for a given tile shape.
template <int TH>
struct AssignTile {
  static_assert(TH == 8 || TH == 16 || TH == 32, "tile heights");
  static constexpr int Px = kTileW * TH;
  static constexpr int Threads = 16 * TH;
  static constexpr int Warps = Threads / 32;
  // registers (64 a thread) allow this many blocks per SM (shared memory may allow fewer)
  static constexpr int BlocksPerSM = 4 * 256 / Threads;
  static constexpr int PrayPerView = 2 * kTileW + 2 * TH;  // staged pair-ray float4 per view
  static constexpr int TS = 2 * Px;                         // shared hash positions
  static constexpr int NL = Px / 2;                         // accumulator entries
  static constexpr int ConstWords =
      (int)((sizeof(CamDev) + kMaxK1 * (sizeof(PairDev) + sizeof(CamDev))) / 4 + Threads - 1) / Threads;
  static_assert(ConstWords <= 4, "a few words per thread copy a block's constants");
  static constexpr size_t BC = 0;
  // per hash position (TS): cell slot, entry index, smallest weight exponent, largest
  // ordered C, member count; the last four are contiguous so that one loop clears them
  static constexpr size_t FK = align16(BC + sizeof(BlockConst));   // u32 cell slot
  static constexpr size_t MinP = FK + 4 * TS;                      // int smallest exponent
  static constexpr size_t CmaxP = MinP + 4 * TS;                   // u32 largest ordered C
  static constexpr size_t CntP = CmaxP + 4 * TS;                   // u32 members
  static constexpr size_t FI = align16(CntP + 4 * TS);             // int entry of a position
  // per entry (NL): key, hash position, lowest index at the largest C, split sums
  static constexpr size_t EK = align16(FI + 4 * TS);               // u64 key
  static constexpr size_t EP = align16(EK + 8 * NL);               // u32 hash position
  static constexpr size_t Gmin = align16(EP + 4 * NL);             // u32 lowest index
  static constexpr size_t Acc = align16(Gmin + 4 * NL);            // u32[14][NL] split sums
  static constexpr size_t Pid = align16(Acc + 14 * 4 * NL);        // u16[tile] gated pixels
  static constexpr size_t Z = align16(Pid + 2 * Px);               // f32[tile] their depth
  static constexpr size_t C = align16(Z + 4 * Px);                 // f32[tile] confidence
  static constexpr size_t RGB = align16(C + 4 * Px);               // u32[tile] colour
  static constexpr size_t PR = align16(RGB + 4 * Px);              // float4[K1][PrayPerView]
  // dynamic shared memory of a launch with k1 neighbour views
  static constexpr size_t smem(int k1) { return PR + 16 * (size_t)k1 * PrayPerView; }
};
constexpr unsigned kLoBits = 22;           // split of a <= 2^37 sum term: 512 lows fit in u32

// Writes partial p as record pi and pushes it onto its cell's list; true when it is the
// cell's first partial of the frame (the caller then lists the cell).
// mmin: the record's smallest weight exponent, INT_MAX for top-k records (no sums).
__device__ __forceinline__ bool file_partial(const Tables& t, Partial& p, unsigned slot,
                                             unsigned long long key, int mmin, unsigned pi) {
  SlotRec& rec = t.frec[slot];
  rec.key = key;                                // the same value from every tile of the cell
  if (mmin != INT_MAX) atomicMin(&rec.mmin, mmin);
  p.next = atomicExch(&rec.head, pi);           // list push
  t.part[pi] = p;
  return p.next == kSlotNone;
}

// rint(v) for 0 <= v < 2^37 as hi 2^22 + lo with lo in [0, 2^22], using 32-bit conversions
// only: v - floor(v 2^-22) 2^22 is exact (both are multiples of ulp(v)), and adding the even
// integer hi 2^22 does not change a round-half-even decision.
__device__ __forceinline__ void split_round(float v, unsigned& lo, unsigned& hi) {
  const float hf = floorf(__fmul_rn(v, 1.0f / (float)(1u << kLoBits)));
  hi = (unsigned)hf;
  lo = __float2uint_rn(__fmaf_rn(-hf, (float)(1u << kLoBits), v));
}

// First probe of a point's coarse record (read-only during the assign step, L1-cached);
// coarse_lvbase() finishes the probe once the value is needed.
__device__ __forceinline__ ulonglong2 coarse_probe(const Tables& t, unsigned long long key, unsigned& h) {
  h = (unsigned)mix64(key) & t.cmask;
  return __ldg(reinterpret_cast<const ulonglong2*>(&t.coarse[h]));
}

// Camera and first pixel of tile T (tiles of TH rows): a division when every camera has the
// same size, else a binary search of the per-camera tile ranges (constant bank).
template <int TH>
__device__ __forceinline__ void tile_of(const TileIndex& ti, int T, int& cam, int& x0, int& y0) {
  if (ti.per_cam) {
    cam = T / ti.per_cam;
  } else {
    cam = 0;
    for (int lo = 0, hi = ti.n_cams - 1; lo <= hi;) {
      const int mid = (lo + hi) >> 1;
      if (ti.first[mid] <= T) { cam = mid; lo = mid + 1; } else { hi = mid - 1; }
    }
  }
  const int local = T - ti.first[cam], tiles_x = (ti.W[cam] + kTileW - 1) / kTileW;
  x0 = (local % tiles_x) * kTileW;
  y0 = (local / tiles_x) * TH;
}

// TOPK: the Sec. II.5(2)a variant; members are keyed and counted as usual, but a tile keeps
// each cell's top-k members by C (packed (ordered(C) << 32) | ~g keys) instead of weights;
// the consistency and weights of those members are computed per cell by k_reduce_topk.
template <typename DT, bool TOPK, bool TRACE, int NB, int TH>
__global__ void __launch_bounds__(AssignTile<TH>::Threads, AssignTile<TH>::BlocksPerSM)
k_assign(const __grid_constant__ BatchArgs<NB> args) {
  using AT = AssignTile<TH>;
  constexpr int kTileH = TH, kTilePx = AT::Px, kAssignThreads = AT::Threads, kAssignWarps = AT::Warps;
  constexpr int kAssignTS = AT::TS, kAssignNL = AT::NL, kPrayPerView = AT::PrayPerView;
  constexpr int kConstWords = AT::ConstWords;
  constexpr size_t kSmBC = AT::BC, kSmFK = AT::FK, kSmMinP = AT::MinP, kSmCmaxP = AT::CmaxP,
                   kSmCntP = AT::CntP, kSmFI = AT::FI, kSmEK = AT::EK, kSmEP = AT::EP,
                   kSmGmin = AT::Gmin, kSmAcc = AT::Acc, kSmPid = AT::Pid, kSmZ = AT::Z, kSmC = AT::C,
                   kSmRGB = AT::RGB, kSmPR = AT::PR;
  int T;
  const FrameArgs& fa = args.f[batch_frame<NB>(args.tile_first, args.n, (int)blockIdx.x, T)];
  const RigDev* __restrict__ rigp = fa.rig;
  const float2* __restrict__ rays = fa.rays;
  const FramePtrs& fp = fa.fp;
  const Tables& t = fa.t;
  const TraceDev& tr = fa.tr;
  const float unit_m = (float)fa.unit_m;
  const TileIndex& ti = fa.ti;
  pdl_release();
  extern __shared__ __align__(16) unsigned char smem[];
  BlockConst& bc = *reinterpret_cast<BlockConst*>(smem + kSmBC);
  unsigned* s_fk = reinterpret_cast<unsigned*>(smem + kSmFK);
  int* s_minp = reinterpret_cast<int*>(smem + kSmMinP);
  unsigned* s_cmaxp = reinterpret_cast<unsigned*>(smem + kSmCmaxP);
  unsigned* s_cntp = reinterpret_cast<unsigned*>(smem + kSmCntP);
  int* s_fi = reinterpret_cast<int*>(smem + kSmFI);
  unsigned long long* s_ek = reinterpret_cast<unsigned long long*>(smem + kSmEK);
  unsigned* s_ep = reinterpret_cast<unsigned*>(smem + kSmEP);
  unsigned* s_gmin = reinterpret_cast<unsigned*>(smem + kSmGmin);
  unsigned* s_acc = reinterpret_cast<unsigned*>(smem + kSmAcc);
  unsigned short* s_pid = reinterpret_cast<unsigned short*>(smem + kSmPid);
  float* s_z = reinterpret_cast<float*>(smem + kSmZ);
  float* s_c = reinterpret_cast<float*>(smem + kSmC);
  unsigned* s_rgb = reinterpret_cast<unsigned*>(smem + kSmRGB);
  __shared__ unsigned s_n, s_base, s_ng, s_nm;

  const RigDev& rig = *rigp;
  int cam, x0, y0;
  tile_of<TH>(ti, T, cam, x0, y0);
  const int W = ti.W[cam], H = ti.H[cam], k1 = ti.k1;
  struct { int x0, y0; long long off; } td;
  td.x0 = x0;
  td.y0 = y0;
  td.off = ti.off[cam];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // warm L2 with the images of the tile that starts when this wave of blocks has finished
  if (threadIdx.x < 4 * kTileH && T + ti.ahead < t.n_tiles) {
    int pc, px0, py0;
    tile_of<TH>(ti, T + ti.ahead, pc, px0, py0);
    const int row = py0 + (threadIdx.x & (kTileH - 1)), kind = threadIdx.x / kTileH;
    if (row < ti.H[pc]) {                     // every address lies inside its image
      const long long li = (long long)row * ti.W[pc] + px0;
      const long long last = (long long)row * ti.W[pc] + min(px0 + kTileW, ti.W[pc]) - 1;
      const char* a = kind == 0 ? static_cast<const char*>(fp.depth[pc]) + li * sizeof(DT)
                    : kind == 1 ? reinterpret_cast<const char*>(fp.conf[pc] + li)
                    : reinterpret_cast<const char*>(fp.rgb[pc]) + 3 * (kind == 3 ? last : li);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
  }
  const DT* __restrict__ dep = static_cast<const DT*>(fp.depth[cam]);
  const float* __restrict__ cf = fp.conf[cam];
  const uint8_t* __restrict__ col = fp.rgb[cam];
  // issue the constant-block loads (L2) and the tile's image loads (HBM) before waiting
  // on either: the words of cam, pair[0, k1) and nb[0, k1) of this camera's BlockConst
  constexpr int kCamW = sizeof(CamDev) / 4, kPairW = sizeof(PairDev) / 4;
  constexpr int kNbAt = (int)(offsetof(BlockConst, nb) / 4), kPairAt = (int)(offsetof(BlockConst, pair) / 4);
  const int n_cw = kCamW + k1 * (kPairW + kCamW);
  const int* gsrc = reinterpret_cast<const int*>(&t.bconst[cam]);
  int cwv[kConstWords], cwi[kConstWords];
#pragma unroll
  for (int r = 0; r < kConstWords; ++r) {
    const int w = threadIdx.x + r * kAssignThreads;
    cwi[r] = w < kCamW ? w
           : w < kCamW + k1 * kPairW ? kPairAt + (w - kCamW)
           : w < n_cw ? kNbAt + (w - kCamW - k1 * kPairW) : -1;
    cwv[r] = cwi[r] >= 0 ? __ldg(gsrc + cwi[r]) : 0;
  }
  // the tile's pair rays (Eq. 4): per view, A of its 32 columns and B of its 16 rows, each
  // as two float4 planes: [A first halves | A second halves | B first | B second]
  constexpr int kPrayLoads = (kMaxK1 * kPrayPerView + kAssignThreads - 1) / kAssignThreads;
  float4 prv[kPrayLoads];
  int pri[kPrayLoads];
  {
    const int Wp = W, Hp = H;
#pragma unroll
    for (int r = 0; r < kPrayLoads; ++r) {
      const int idx = threadIdx.x + r * kAssignThreads;
      pri[r] = -1;
      prv[r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (TOPK || idx >= k1 * kPrayPerView) continue;
      const int q = idx / kPrayPerView, o = idx - q * kPrayPerView;
      const int base = ti.pray[cam] + 2 * q * (Wp + Hp);
      int src = -1;
      if (o < 2 * kTileW) {                                        // A: plane o / 32
        const int c = td.x0 + (o & (kTileW - 1));
        if (c < Wp) src = base + 2 * c + o / kTileW;
      } else {                                                     // B: plane (o - 64) / 16
        const int rr = o - 2 * kTileW, row = td.y0 + (rr & (kTileH - 1));
        if (row < Hp) src = base + 2 * Wp + 2 * row + rr / kTileH;
      }
      if (src >= 0) {
        prv[r] = __ldg(t.pray + src);
        pri[r] = idx;
      }
    }
  }
  DT Dk[2];
  float ckv[2];
  uint8_t cb[2][3];
  bool inimg[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int x = td.x0 + lane, y = td.y0 + warp + kAssignWarps * k;
    inimg[k] = x < W && y < H;
    Dk[k] = (DT)0;
    ckv[k] = 0.0f;
    cb[k][0] = cb[k][1] = cb[k][2] = 0;
    if (inimg[k]) {
      const long long li = (long long)y * W + x;
      Dk[k] = dep[li];
      ckv[k] = cf[li];
      const uint8_t* px = col + 3 * li;
      cb[k][0] = px[0];
      cb[k][1] = px[1];
      cb[k][2] = px[2];
    }
  }
  int* sdst = reinterpret_cast<int*>(&bc);
#pragma unroll
  for (int r = 0; r < kConstWords; ++r)
    if (cwi[r] >= 0) sdst[cwi[r]] = cwv[r];
  float4* s_pr = reinterpret_cast<float4*>(smem + kSmPR);
#pragma unroll
  for (int r = 0; r < kPrayLoads; ++r)
    if (pri[r] >= 0) s_pr[pri[r]] = prv[r];
  // clear the per-position arrays: slot none, exponent INT_MAX, largest C 0, count 0
  for (int i = threadIdx.x; i < kAssignTS; i += kAssignThreads) {
    const unsigned v = i < kAssignTS / 4 ? kSlotNone : i < kAssignTS / 2 ? (unsigned)INT_MAX : 0u;
    reinterpret_cast<uint4*>(smem + kSmFK)[i] = make_uint4(v, v, v, v);
  }
  if (threadIdx.x == 0) { s_n = 0; s_ng = 0; }
  __syncthreads();

  constexpr bool trace = TRACE;             // per-pixel trace (tests) in its own instantiation
  const float qnan = __int_as_float(0x7fc00000);

  // (a) Eq. 9 gate and compaction of the tile's gated pixels (any order: every reduction
  // below is order-independent), so that the per-point work runs on full warps
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int row = warp + kAssignWarps * k;
    bool gated = false;
    if (inimg[k]) {
      gated = Depth<DT>::valid(Dk[k]) && (!rig.use_conf || ckv[k] > rig.tau);
      if (!gated && trace) {
        const long long g = td.off + (long long)(td.y0 + row) * W + td.x0 + lane;
        if (tr.pw) { tr.pw[3 * g] = qnan; tr.pw[3 * g + 1] = qnan; tr.pw[3 * g + 2] = qnan; }
        if (tr.e) tr.e[g] = qnan;
        if (tr.omega) tr.omega[g] = qnan;
        if (tr.nview) tr.nview[g] = -1;
        if (tr.key) tr.key[g] = kKeyEmpty;
      }
    }
    const unsigned gmask = __ballot_sync(0xffffffffu, gated);
    unsigned wbase = 0u;
    if (lane == 0 && gmask) wbase = atomicAdd(&s_ng, (unsigned)__popc(gmask));
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    if (gated) {
      const int pos = (int)wbase + __popc(gmask & ((1u << lane) - 1u));
      s_pid[pos] = (unsigned short)(row * kTileW + lane);
      s_z[pos] = Depth<DT>::z(Dk[k]);
      s_c[pos] = ckv[k];
      s_rgb[pos] = (unsigned)cb[k][0] | ((unsigned)cb[k][1] << 8) | ((unsigned)cb[k][2] << 16);
    }
  }
  __syncthreads();
  const int n_g = (int)s_ng;
  const CamDev& C = bc.cam;
  // everything above read only the frame's inputs and the context's constants; the coarse
  // table (count and level steps) and every table written below need the earlier kernels
  pdl_wait();

  // (a) Eq. 8, (b) Eq. 4-7 and 10, (c) Sec. II.5(1)d-e for each gated point
  bool has[2] = {false, false};
  float mu[2] = {0.0f, 0.0f};
  int mexp[2] = {0, 0};
  unsigned cord[2] = {0u, 0u};
  int hpos[2] = {0, 0};
  long long gi[2] = {0, 0};
  float frac[2][3];
  unsigned long long fkey[2] = {kKeyEmpty, kKeyEmpty};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int i = threadIdx.x + j * kAssignThreads;
    if (i >= n_g) continue;
    const int pid = s_pid[i];
    const int x = td.x0 + (pid & (kTileW - 1)), y = td.y0 + pid / kTileW;
    gi[j] = td.off + (long long)y * W + x;
    const float z = s_z[i];
    const float c = s_c[i];
    const float rx = __ldg(&rays[C.ray_x + x].x), ry = __ldg(&rays[C.ray_y + y].x);
    float P[3], r[3];
    world_point(C, z, rx, ry, P);                                     // Eq. 8
    has[j] = grid_coords(rig, P, r);
    // start the lookup of the coarse cell's level and slot range (Sec. II.5(1)d)
    const unsigned long long ck = has[j] ? coarse_key(r) : kKeyEmpty;
    unsigned ch = 0u;
    ulonglong2 ce = make_ulonglong2(kKeyEmpty, 0ull);
    if (has[j]) ce = coarse_probe(t, ck, ch);
    float sh = 0.0f, sl = 0.0f, eh = 0.0f;
    int nview = 0, m = 0;
    if constexpr (!TOPK) {
      if (rig.use_cons && k1 > 0)
        residual_sum<DT>(bc, k1, TilePairRays<TH>{reinterpret_cast<const float4*>(smem + kSmPR),
                                                  x - td.x0, y - td.y0},
                         rays, fp, z, sh, sl, nview);
      eh = joint_weight(rig, k1, sh, sl, c, mu[j], m);
    }
    mexp[j] = m;
    cord[j] = ordered(c);
    if (trace) {
      if (tr.pw) {
        tr.pw[3 * gi[j] + 0] = P[0] * unit_m;
        tr.pw[3 * gi[j] + 1] = P[1] * unit_m;
        tr.pw[3 * gi[j] + 2] = P[2] * unit_m;
      }
      if (!TOPK) {
        if (tr.e) tr.e[gi[j]] = eh;
        if (tr.omega) tr.omega[gi[j]] = ldexpf(mu[j], -m);
        if (tr.nview) tr.nview[gi[j]] = nview;
      } else if (tr.nview) {                    // the top-k variant weighs cells' top-k only:
        tr.nview[gi[j]] = -2;                   // gated, weight not evaluated here
      }
    }
    if (has[j]) {
      // Sec. II.5(1)e: cell key, its dense slot, and the point's offset inside the cell
      const unsigned lb = coarse_lvbase(t, ck, ch, ce);
      const int l = (int)(lb >> 27);
      const unsigned cbase = lb & kBaseNone;
      const unsigned long long fk = fine_key(r, l);
      const int kk[3] = {(int)((fk >> 40) & 0xfffff) - kKeyBias, (int)((fk >> 20) & 0xfffff) - kKeyBias,
                         (int)(fk & 0xfffff) - kKeyBias};
      const float sl2 = pow2f(l);
#pragma unroll
      for (int a = 0; a < 3; ++a) frac[j][a] = __fsub_rn(__fmul_rn(r[a], sl2), (float)kk[a]);
      // sub-cell of the coarse cell: k - (coarse << l) = k & (2^l - 1)
      const unsigned mask = (1u << l) - 1u;
      const unsigned local = ((((unsigned)kk[0] & mask) << l | ((unsigned)kk[1] & mask)) << l) |
                             ((unsigned)kk[2] & mask);
      if (cbase == kBaseNone) {                 // slot capacity exceeded (reported)
        has[j] = false;
      } else {
        fkey[j] = fk;
        bool fresh;
        const int h = local_pos<kAssignTS>(s_fk, kSlotNone, cbase + local, kAssignTS, fresh);
        hpos[j] = h;
        if (h < 0) {
          has[j] = false;
          atomicOr(&t.cnt->error, kErrSlots);
        } else {
          if (fresh) {                          // the cell's entry: index and accumulators
            const int e = (int)atomicAdd(&s_n, 1u);
            s_fi[h] = e;
            if (e < kAssignNL) {
              s_ek[e] = fk;
              s_ep[e] = (unsigned)h;
              s_gmin[e] = 0xffffffffu;
              if constexpr (TOPK) {             // the entry's top-k list (u64 view of s_acc)
                unsigned long long* top = reinterpret_cast<unsigned long long*>(s_acc) + e * kMaxTopK;
#pragma unroll
                for (int q = 0; q < kMaxTopK; ++q) top[q] = 0ull;
              } else {
#pragma unroll
                for (int a = 0; a < 14; ++a) s_acc[a * kAssignNL + e] = 0u;
              }
            }
          }
          // Sec. II.5(2)a: members, largest C, smallest weight exponent
          atomicAdd(&s_cntp[h], 1u);
          if (!TOPK) {
            atomicMax(&s_cmaxp[h], cord[j]);
            atomicMin(&s_minp[h], mexp[j]);
          }
        }
      }
    }
    if (trace && tr.key) tr.key[gi[j]] = has[j] ? fkey[j] : kKeyEmpty;
  }
  __syncthreads();
  // more cells than accumulators: the multi-member cells take them (see kAssignNL)
  const bool renumber = s_n > (unsigned)kAssignNL;         // the same in every thread
  bool all_alone = false;
  unsigned n_local = s_n;
  if (renumber) {
    if (threadIdx.x == 0) s_nm = 0u;
    __syncthreads();
    for (int h = threadIdx.x; h < kAssignTS; h += kAssignThreads) {
      if (s_fk[h] == kSlotNone) continue;
      int e = kAssignNL;
      if (s_cntp[h] >= 2u) {
        e = (int)atomicAdd(&s_nm, 1u);
        if (e < kAssignNL) {
          s_ep[e] = (unsigned)h;
          s_gmin[e] = 0xffffffffu;
          if constexpr (TOPK) {
            unsigned long long* top = reinterpret_cast<unsigned long long*>(s_acc) + e * kMaxTopK;
#pragma unroll
            for (int q = 0; q < kMaxTopK; ++q) top[q] = 0ull;
          } else {
#pragma unroll
            for (int a = 0; a < 14; ++a) s_acc[a * kAssignNL + e] = 0u;
          }
        } else {
          e = kAssignNL;
        }
      }
      s_fi[h] = e;
    }
    __syncthreads();
    all_alone = s_nm > (unsigned)kAssignNL;
    n_local = all_alone ? 0u : s_nm;
  }
  // reserve the tile's partial records now; the index is needed only at the end
  unsigned base_pi = 0u;
  if (threadIdx.x == 0) base_pi = atomicAdd(&t.cnt->n_partials, n_local);
  // representative: lowest pixel index among the largest C; Eq. 11 sums at the tile's
  // scale 2^-(36 + mmin_tile), each 64-bit term split in two native 32-bit atomics
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (!has[j]) continue;
    const int h = hpos[j], e = s_fi[h];
    const bool alone = all_alone || e >= kAssignNL;
    if (renumber && !alone) s_ek[e] = fkey[j];  // every member writes the cell's key
    if constexpr (TOPK) {
      // Sec. II.5(2)a: insert the member into its cell's sorted top-k list; each slot keeps
      // the largest key that reaches it and passes the smaller one down, so the list ends
      // as the k largest keys whatever the order of the atomics
      unsigned long long key = ((unsigned long long)cord[j] << 32) | (unsigned)(~(unsigned)gi[j]);
      if (!alone) {
        unsigned long long* top = reinterpret_cast<unsigned long long*>(s_acc) + e * kMaxTopK;
        for (int q = 0; q < rig.top_k && key; ++q) {
          const unsigned long long old = atomicMax(&top[q], key);
          key = old < key ? old : key;
        }
      } else {                                  // a single-member partial of its own
        Partial p;
        const unsigned slot = s_fk[h];
        p.count = 1u;
        p.rep = key;
#pragma unroll
        for (int a = 0; a < kMaxTopK - 1; ++a) p.top[a] = 0ull;
        const unsigned pi = atomicAdd(&t.cnt->n_partials, 1u);
        if (pi >= t.max_partials) {
          atomicOr(&t.cnt->error, kErrPartials);
        } else if (file_partial(t, p, slot, fkey[j], INT_MAX, pi)) {
          const unsigned n = atomicAdd(&t.cnt->n_cells, 1u);
          if (n < t.max_slots) t.fused[n] = slot;
        }
      }
      continue;
    }
    if (!alone && cord[j] == s_cmaxp[h]) atomicMin(&s_gmin[e], (unsigned)gi[j]);
    const int sh = alone ? 0 : mexp[j] - s_minp[h];
    const float w = sh > 62 ? 0.0f : __fmul_rn(mu[j], pow2f(kFixShift - sh));
    const unsigned rgb = s_rgb[threadIdx.x + j * kAssignThreads];
    float v[7];
    v[0] = w;
#pragma unroll
    for (int a = 0; a < 3; ++a) v[1 + a] = __fmul_rn(w, frac[j][a]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
      v[4 + a] = __fmul_rn(w, (float)((rgb >> (8 * a)) & 0xffu) * 0.00390625f);
    if (!alone) {
#pragma unroll
      for (int a = 0; a < 7; ++a) {
        unsigned lo, hi;
        split_round(v[a], lo, hi);
        atomicAdd(&s_acc[(2 * a) * kAssignNL + e], lo);
        atomicAdd(&s_acc[(2 * a + 1) * kAssignNL + e], hi);
      }
    } else {                                    // a single-member partial of its own
      Partial p;
      const unsigned slot = s_fk[hpos[j]];
      p.count = 1u;
      p.sum.mmin = mexp[j];
      p.sum.pad = 0;
      p.rep = ((unsigned long long)cord[j] << 32) | (unsigned)(~(unsigned)gi[j]);
#pragma unroll
      for (int a = 0; a < 7; ++a) {
        unsigned lo, hi;
        split_round(v[a], lo, hi);
        p.set_sum(a, ((unsigned long long)hi << kLoBits) + lo);
      }
      const unsigned pi = atomicAdd(&t.cnt->n_partials, 1u);
      if (pi >= t.max_partials) {
        atomicOr(&t.cnt->error, kErrPartials);
      } else if (file_partial(t, p, slot, fkey[j], mexp[j], pi)) {
        const unsigned n = atomicAdd(&t.cnt->n_cells, 1u);
        if (n < t.max_slots) t.fused[n] = slot;
      }
    }
  }
  if (threadIdx.x == 0) s_base = base_pi;
  __syncthreads();
  // one partial record per (tile, cell), pushed onto its cell's list
  for (int e0 = 0; e0 < (int)n_local; e0 += kAssignThreads) {
    const int e = e0 + threadIdx.x;
    bool first = false;
    unsigned slot = 0u;
    if (e < (int)n_local) {
      const unsigned pi = s_base + (unsigned)e;
      if (pi >= t.max_partials) {
        atomicOr(&t.cnt->error, kErrPartials);
      } else {
        const unsigned h = s_ep[e];
        Partial p;
        slot = s_fk[h];
        p.count = s_cntp[h];
        if constexpr (TOPK) {
          const unsigned long long* top = reinterpret_cast<const unsigned long long*>(s_acc) + e * kMaxTopK;
          p.rep = top[0];
#pragma unroll
          for (int a = 0; a < kMaxTopK - 1; ++a) p.top[a] = top[a + 1];
        } else {
          p.sum.mmin = s_minp[h];
          p.sum.pad = 0;
          p.rep = ((unsigned long long)s_cmaxp[h] << 32) | (unsigned)(~s_gmin[e]);
#pragma unroll
          for (int a = 0; a < 7; ++a)
            p.set_sum(a, ((unsigned long long)s_acc[(2 * a + 1) * kAssignNL + e] << kLoBits) +
                             s_acc[(2 * a) * kAssignNL + e]);
        }
        first = file_partial(t, p, slot, s_ek[e], TOPK ? INT_MAX : s_minp[h], pi);
      }
    }
    // one counter update per warp for the cells claimed in it
    const unsigned claim = __ballot_sync(0xffffffffu, first);
    unsigned nb = 0u;
    if (lane == 0 && claim) nb = atomicAdd(&t.cnt->n_cells, (unsigned)__popc(claim));
    nb = __shfl_sync(0xffffffffu, nb, 0);
    if (first) {
      const unsigned n = nb + __popc(claim & ((1u << lane) - 1u));
      if (n < t.max_slots) t.fused[n] = slot;
    }
  }
}

// ------------------------------------------------------------------ reduce step
// u64 -> float32 through two 32-bit conversions (at most two roundings)
__device__ __forceinline__ float u64_to_f32(unsigned long long x) {
  return __fmaf_rn(__uint2float_rn((unsigned)(x >> 32)), 4294967296.0f, __uint2float_rn((unsigned)x));
}

template <int NB>
__global__ void __launch_bounds__(kThreads) k_reduce(const __grid_constant__ BatchArgs<NB> args) {
  const Tables& t = args.f[batch_frame_y<NB>()].t;
  const OutDev& out = args.f[batch_frame_y<NB>()].out;
  pdl_release();
  pdl_wait();
  const unsigned n_cells = min(t.cnt->n_cells, t.max_slots);
  const unsigned n_coarse = min(t.cnt->n_coarse, t.cmask + 1u);
  const unsigned n_part = min(t.cnt->n_partials, t.max_partials);
  const unsigned n = max(n_cells, n_coarse);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < n_cells) {
      const unsigned slot = t.fused[i];
      const SlotRec rec = t.frec[slot];
      const unsigned long long key = rec.key;
      const unsigned head = rec.head;
      const int mmin = rec.mmin;
      unsigned count = 0u, steps = 0u;
      unsigned long long rep = 0ull;
      unsigned long long S[7] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
      for (unsigned p = head; p != kSlotNone && steps <= n_part; ++steps) {
        const Partial P = t.part[p];
        count += P.count;
        rep = max(rep, P.rep);
        const int sh = P.sum.mmin - mmin;      // shift to the cell's smallest exponent
#pragma unroll
        for (int a = 0; a < 7; ++a) S[a] += sh < 64 ? (P.get_sum(a) >> sh) : 0ull;
        p = P.next;
      }
      if (steps > n_part) atomicOr(&t.cnt->error, kErrList);
      const unsigned g = head != kSlotNone ? ~(unsigned)(rep & 0xffffffffull) : 0xffffffffu;
      CellOut c;
      // Eq. 11 in float32: position = edge (k + S_k / S_0), colour = 256 S_c / S_0,
      // weight = S_0 2^-(36 + mmin); each result is within a few float32 roundings
      const int l = (int)(key >> 60);
      const float edge = __fmul_rn(out.s0_m, pow2f(-l));
      const float Wf = u64_to_f32(S[0]);
      const float inv = S[0] ? __frcp_rn(Wf) : __int_as_float(0x7fc00000);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int ka = (int)((key >> (40 - 20 * a)) & 0xfffff) - kKeyBias;
        c.pos[a] = __fmaf_rn(edge, (float)ka, __fmul_rn(edge, __fmul_rn(u64_to_f32(S[1 + a]), inv)));
        c.rgb[a] = __fmul_rn(256.0f, __fmul_rn(u64_to_f32(S[4 + a]), inv));
      }
      c.weight = ldexpf(Wf, -kFixShift - min(mmin, 1 << 30));
      c.count = count;
      c.rep = g;
      c.pad = 0u;
      c.key = key;
      if ((long long)i < out.max_cells) {
        t.staged[i] = c;
        if (head != kSlotNone) atomicOr(&t.bitmap[g >> 5], 1u << (g & 31));
      }
      // ready for the next frame: head = none, mmin = INT_MAX (one 8-byte store)
      reinterpret_cast<unsigned long long*>(&t.frec[slot])[1] =
          ((unsigned long long)(unsigned)INT_MAX << 32) | kSlotNone;
    }
    if (i < n_coarse) {
      const unsigned cs = t.cused[i];
      t.coarse[cs].key = kKeyEmpty;
      t.coarse[cs].count = 0u;
    }
  }
}

// ------------------------------------------------------------------ top-k reduce
// Sec. II.5(2) variant, per cell: merge the tiles' top-k lists (the k largest packed
// (ordered(C) << 32) | ~g keys of the union: order-independent), then for each of the
// cell's k representatives recompute the world point (Eq. 8, the same float32 sequence as
// the other steps), its consistency over its camera's K-1 views (Eq. 4-7, double-float,
// global pair rays) and omega = C V (Eq. 10), and fuse them (Eq. 11, normalised, weights
// scaled by the largest).  Members are counted over the whole cell; the representative is
// the cell's top member.
template <typename DT, int NB>
__global__ void __launch_bounds__(kThreads, 3) k_reduce_topk(const __grid_constant__ BatchArgs<NB> args) {
  const FrameArgs& fa = args.f[batch_frame_y<NB>()];
  const RigDev* __restrict__ rigp = fa.rig;
  const float2* __restrict__ rays = fa.rays;
  const FramePtrs& fp = fa.fp;
  const Tables& t = fa.t;
  const OutDev& out = fa.out;
  pdl_release();
  pdl_wait();
  const RigDev& rig = *rigp;
  const unsigned n_cells = min(t.cnt->n_cells, t.max_slots);
  const unsigned n_coarse = min(t.cnt->n_coarse, t.cmask + 1u);
  const unsigned n_part = min(t.cnt->n_partials, t.max_partials);
  const unsigned n = max(n_cells, n_coarse);
  const int K = rig.top_k;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < n_cells) {
      const unsigned slot = t.fused[i];
      const SlotRec rec = t.frec[slot];
      unsigned long long top[kMaxTopK];
#pragma unroll
      for (int q = 0; q < kMaxTopK; ++q) top[q] = 0ull;
      unsigned count = 0u, steps = 0u;
      for (unsigned p = rec.head; p != kSlotNone && steps <= n_part; ++steps) {
        const Partial P = t.part[p];
        count += P.count;
        for (int a = 0; a < K; ++a) {           // insert the tile's key a into the sorted list
          unsigned long long key = a == 0 ? P.rep : P.top[a - 1];
#pragma unroll
          for (int q = 0; q < kMaxTopK; ++q) {
            if (q < K && key > top[q]) {
              const unsigned long long tmp = top[q];
              top[q] = key;
              key = tmp;
            }
          }
        }
        p = P.next;
      }
      if (steps > n_part) atomicOr(&t.cnt->error, kErrList);
      // weights and world points of the representatives
      float mu[kMaxTopK], P3[kMaxTopK][3], col[kMaxTopK][3];
      int mx[kMaxTopK];
      int mmin = INT_MAX, nr = 0;
#pragma unroll
      for (int q = 0; q < kMaxTopK; ++q) {      // sorted: the filled entries come first
        mu[q] = 0.0f;
        mx[q] = 0;
        if (q >= K || !top[q]) continue;
        const unsigned g = ~(unsigned)(top[q] & 0xffffffffull);
        if ((long long)g >= rig.n_px) {         // not a pixel: a corrupted list (reported)
          atomicOr(&t.cnt->error, kErrList);
          top[q] = 0ull;
          continue;
        }
        int cam = 0;
        for (int c = 1; c < rig.n_cams; ++c)
          if ((long long)g >= rig.cam[c].off) cam = c;
        const CamDev& C = rig.cam[cam];
        const long long li = (long long)g - C.off;
        const int y = (int)(li / C.W), x = (int)(li - (long long)y * C.W);
        const float z = Depth<DT>::z(static_cast<const DT*>(fp.depth[cam])[li]);
        const float c = fp.conf[cam][li];
        const uint8_t* px = fp.rgb[cam] + 3 * li;
        world_point(C, z, __ldg(&rays[C.ray_x + x].x), __ldg(&rays[C.ray_y + y].x), P3[q]);
        float sh = 0.0f, sl = 0.0f;
        int nview = 0;
        if (rig.use_cons && rig.k1 > 0)
          residual_sum<DT>(t.bconst[cam], rig.k1, GlobalPairRays{t.pray, x, y}, rays, fp, z, sh,
                           sl, nview);
        joint_weight(rig, rig.k1, sh, sl, c, mu[q], mx[q]);
        mmin = min(mmin, mx[q]);
        col[q][0] = px[0];
        col[q][1] = px[1];
        col[q][2] = px[2];
        ++nr;
      }
      CellOut cell;
      float sw = 0.0f, sp[3] = {0.0f, 0.0f, 0.0f}, sc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int q = 0; q < kMaxTopK; ++q) {      // Eq. 11, weights relative to the largest
        if (q >= nr) continue;
        const int sh = mx[q] - mmin;
        const float w = sh > 126 ? 0.0f : __fmul_rn(mu[q], pow2f(-sh));
        sw = __fadd_rn(sw, w);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          sp[a] = __fmaf_rn(w, P3[q][a], sp[a]);
          sc[a] = __fmaf_rn(w, col[q][a], sc[a]);
        }
      }
      const float inv = nr ? __frcp_rn(sw) : __int_as_float(0x7fc00000);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        cell.pos[a] = __fmul_rn(__fmul_rn(sp[a], inv), out.unit_f);
        cell.rgb[a] = __fmul_rn(sc[a], inv);
      }
      cell.weight = nr ? ldexpf(sw, -min(mmin, 1 << 30)) : 0.0f;
      cell.count = count;
      const bool have = nr > 0 && top[0] != 0ull;
      const unsigned g = have ? ~(unsigned)(top[0] & 0xffffffffull) : 0xffffffffu;
      cell.rep = g;
      cell.pad = 0u;
      cell.key = rec.key;
      if ((long long)i < out.max_cells) {
        t.staged[i] = cell;
        if (have) atomicOr(&t.bitmap[g >> 5], 1u << (g & 31));   // g < n_px (checked above)
      }
      reinterpret_cast<unsigned long long*>(&t.frec[slot])[1] =
          ((unsigned long long)(unsigned)INT_MAX << 32) | kSlotNone;
    }
    if (i < n_coarse) {
      const unsigned cs = t.cused[i];
      t.coarse[cs].key = kKeyEmpty;
      t.coarse[cs].count = 0u;
    }
  }
}

// ------------------------------------------------------------------ point-wise (No SA)
// Table II's "No SA" ablation: fusion without the spatial hash, every gated pixel an output
// point with its own joint weight.  Per pixel: Eq. 8-9 (gate, back-projection), Eq. 4-7 over
// the camera's K-1 views (the same double-float evaluation and global pair rays as the
// top-k reduce step) and Eq. 10; outputs are indexed by the global pixel index (position in
// metres and weight; NaN position and weight 0 for pixels that are not gated, 8-bit colour
// copied), so the cloud is in pixel order without a compaction pass.  One thread a pixel,
// cameras along the grid's second dimension.
template <typename DT>
__global__ void __launch_bounds__(kThreads) k_points(const RigDev* __restrict__ rigp,
                                                     const float2* __restrict__ rays, FramePtrs fp,
                                                     Tables t, PointsDev out) {
  const RigDev& rig = *rigp;
  const int cam = blockIdx.y;
  const CamDev& C = rig.cam[cam];
  const long long npx = (long long)C.W * C.H;
  const DT* __restrict__ dep = static_cast<const DT*>(fp.depth[cam]);
  const float* __restrict__ cf = fp.conf[cam];
  const uint8_t* __restrict__ col = fp.rgb[cam];
  const float qnan = __int_as_float(0x7fc00000);
  unsigned nv = 0u, ng = 0u;
  for (long long li = (long long)blockIdx.x * blockDim.x + threadIdx.x; li < npx;
       li += (long long)gridDim.x * blockDim.x) {
    const long long g = C.off + li;
    const DT D = dep[li];
    const float c = cf[li];
    const bool valid = Depth<DT>::valid(D);
    const bool gated = valid && (!rig.use_conf || c > rig.tau);          // Eq. 9
    nv += valid ? 1u : 0u;
    ng += gated ? 1u : 0u;
    out.rgb[3 * g] = col[3 * li];
    out.rgb[3 * g + 1] = col[3 * li + 1];
    out.rgb[3 * g + 2] = col[3 * li + 2];
    if (!gated) {
      out.pos[3 * g] = qnan;
      out.pos[3 * g + 1] = qnan;
      out.pos[3 * g + 2] = qnan;
      out.weight[g] = 0.0f;
      continue;
    }
    const int y = (int)(li / C.W), x = (int)(li - (long long)y * C.W);
    const float z = Depth<DT>::z(D);
    float P[3];
    world_point(C, z, __ldg(&rays[C.ray_x + x].x), __ldg(&rays[C.ray_y + y].x), P);   // Eq. 8
    float sh = 0.0f, sl = 0.0f, mu;
    int nview = 0, m;
    if (rig.use_cons && rig.k1 > 0)
      residual_sum<DT>(t.bconst[cam], rig.k1, GlobalPairRays{t.pray, x, y}, rays, fp, z, sh, sl, nview);
    joint_weight(rig, rig.k1, sh, sl, c, mu, m);                          // Eq. 7, 10
    out.pos[3 * g] = __fmul_rn(P[0], out.unit_f);
    out.pos[3 * g + 1] = __fmul_rn(P[1], out.unit_f);
    out.pos[3 * g + 2] = __fmul_rn(P[2], out.unit_f);
    out.weight[g] = ldexpf(mu, -min(m, 1 << 30));
  }
  nv = __reduce_add_sync(0xffffffffu, nv);
  ng = __reduce_add_sync(0xffffffffu, ng);
  if ((threadIdx.x & 31) == 0) {
    if (nv) atomicAdd(&out.counts[0], (unsigned long long)nv);
    if (ng) atomicAdd(&out.counts[1], (unsigned long long)ng);
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

// Block b scans bitmap words [1024 b, 1024 b + 1024) and folds a share of the count step's
// per-block statistics into the frame counters; the last block to finish (a fenced
// counter, no waiting) scans the per-block sums and writes the frame statistics.
template <int NB>
__global__ void __launch_bounds__(1024) k_scan(const __grid_constant__ BatchArgs<NB> args) {
  __shared__ unsigned s_w[32];
  __shared__ unsigned long long s_l[3][32];
  __shared__ unsigned s_b[6][32];
  __shared__ bool s_last;
  const Tables& t = args.f[batch_frame_y<NB>()].t;
  const OutDev& out = args.f[batch_frame_y<NB>()].out;
  const unsigned nblk = (unsigned)t.n_wblocks;     // this frame's blocks (the grid may be wider)
  pdl_release();
  pdl_wait();
  if (blockIdx.x >= nblk) return;                  // uniform over the block
  const long long w = (long long)blockIdx.x * 1024 + threadIdx.x;
  const unsigned v = (w < t.n_words) ? __popc(t.bitmap[w]) : 0u;
  unsigned total;
  const unsigned ex = block_excl_scan_1024(v, s_w, total);
  if (w < t.n_words) t.wprefix[w] = ex;
  if (threadIdx.x == 0) t.bsum[blockIdx.x] = total;

  // statistics of the count step's blocks [b0, b1)
  const int per = (t.n_bstats + (int)nblk - 1) / (int)nblk;
  const int b0 = blockIdx.x * per, b1 = min(t.n_bstats, b0 + per);
  unsigned long long nv = 0, ng = 0, noor = 0;
  unsigned bmin[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, bmax[3] = {0u, 0u, 0u};
  for (int i = b0 + threadIdx.x; i < b1; i += 1024) {
    const BlockStats b = t.bstats[i];
    nv += b.n_valid;
    ng += b.n_gated;
    noor += b.n_oor;
    for (int k = 0; k < 3; ++k) { bmin[k] = min(bmin[k], b.bmin[k]); bmax[k] = max(bmax[k], b.bmax[k]); }
  }
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
    unsigned long long a0 = 0, a1 = 0, a2 = 0;
    unsigned mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
    for (int q = 0; q < 32; ++q) {
      a0 += s_l[0][q]; a1 += s_l[1][q]; a2 += s_l[2][q];
      for (int k = 0; k < 3; ++k) { mn[k] = min(mn[k], s_b[k][q]); mx[k] = max(mx[k], s_b[3 + k][q]); }
    }
    if (a0) atomicAdd(&t.cnt->n_valid, a0);
    if (a1) atomicAdd(&t.cnt->n_gated, a1);
    if (a2) atomicAdd(&t.cnt->n_oor, a2);
    for (int k = 0; k < 3; ++k) {
      if (mn[k] != 0xffffffffu) atomicMax(&t.cnt->bmin_inv[k], ~mn[k]);
      if (mx[k] != 0u) atomicMax(&t.cnt->bmax[k], mx[k]);
    }
    __threadfence();
    s_last = atomicAdd(&t.cnt->scan_done, 1u) == nblk - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: exclusive scan of the per-block sums, then the frame statistics
  unsigned carry = 0;
  for (int base = 0; base < t.n_wblocks; base += 1024) {
    const int i = base + threadIdx.x;
    const unsigned bv = (i < t.n_wblocks) ? __ldcg(&t.bsum[i]) : 0u;
    unsigned tot;
    const unsigned bex = block_excl_scan_1024(bv, s_w, tot);
    if (i < t.n_wblocks) t.bsum[i] = carry + bex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    const FrameCounters& c = *t.cnt;
    fuseflow_stats st = {};
    st.n_valid = (int64_t)__ldcg(&c.n_valid);
    st.n_gated = (int64_t)__ldcg(&c.n_gated);
    st.n_out_of_range = (int64_t)__ldcg(&c.n_oor);
    const unsigned nc = __ldcg(&c.n_cells);
    unsigned err = __ldcg(&c.error);
    if ((long long)nc > out.max_cells) err |= kErrCells;
    if (__ldcg(&c.n_partials) > t.max_partials) err |= kErrPartials;
    st.n_cells = (int64_t)(nc < out.max_cells ? nc : out.max_cells);
    for (int k = 0; k < 3; ++k) {
      const unsigned mn = ~__ldcg(&c.bmin_inv[k]), mx = __ldcg(&c.bmax[k]);
      st.bbox[k] = st.n_gated ? (float)((double)from_ordered(mn) * out.unit_m) : __int_as_float(0x7f800000);
      st.bbox[3 + k] = st.n_gated ? (float)((double)from_ordered(mx) * out.unit_m) : __int_as_float(0xff800000);
    }
    st.error = (int32_t)err;
    st.n_coarse = (int32_t)__ldcg(&c.n_coarse);
    *out.stats = st;
  }
}

// ------------------------------------------------------------------ emit
template <int NB>
__global__ void __launch_bounds__(kThreads) k_emit(const __grid_constant__ BatchArgs<NB> args) {
  const Tables& t = args.f[batch_frame_y<NB>()].t;
  const OutDev& out = args.f[batch_frame_y<NB>()].out;
  pdl_release();
  pdl_wait();
  const unsigned n_cells = (unsigned)min((long long)min(t.cnt->n_cells, t.max_slots), out.max_cells);
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

// Served frames: the cloud's first n cells (n = min(n_cells, capacity)) and the
// statistics, written into pinned host memory through its mapped addresses.
__global__ void __launch_bounds__(kThreads) k_copyout(fuseflow_cloud src, HostOutDev dst) {
  const long long nc = src.stats->n_cells;
  const long long n = nc < dst.capacity ? nc : dst.capacity;
  if (blockIdx.x == 0 && threadIdx.x == 0) *dst.stats = *src.stats;
  // word ranges of the six arrays, back to back: pos 3n, rgb 3n, weight n, count n,
  // rep n, key 2n
  const long long total = 11 * n;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
       w += (long long)gridDim.x * blockDim.x) {
    long long o = w;
    const uint32_t* from;
    uint32_t* to;
    if (o < 3 * n) { from = reinterpret_cast<const uint32_t*>(src.pos); to = reinterpret_cast<uint32_t*>(dst.pos); }
    else if ((o -= 3 * n) < 3 * n) { from = reinterpret_cast<const uint32_t*>(src.rgb); to = reinterpret_cast<uint32_t*>(dst.rgb); }
    else if ((o -= 3 * n) < n) { from = reinterpret_cast<const uint32_t*>(src.weight); to = reinterpret_cast<uint32_t*>(dst.weight); }
    else if ((o -= n) < n) { from = src.count; to = dst.count; }
    else if ((o -= n) < n) { from = src.rep; to = dst.rep; }
    else { o -= n; from = reinterpret_cast<const uint32_t*>(src.key); to = reinterpret_cast<uint32_t*>(dst.key); }
    if (to) to[o] = from[o];
  }
}

// ------------------------------------------------------------------ Eq. 12 (MC error)
// Per point P_k (world, metres): the cameras that see it (in front, nearest pixel inside
// the image, valid D_i there) and the mean of |z(T_i P_k) - D_i(pi(T_i P_k))| over them.
// Each block leaves the sum (depth units) and the number of points with a visible camera
// in bsum/bcnt; the host adds the blocks in order, so the mean does not depend on timing.
constexpr int kMcBlocks = 1024;

template <typename DT>
__global__ void __launch_bounds__(kThreads) k_mc(const RigDev* __restrict__ rigp, FramePtrs fp,
                                                 const float* __restrict__ pos, long long n,
                                                 float inv_unit, float unit_m, float occl_u,
                                                 float* err, int* nvis, double* bsum,
                                                 long long* bcnt) {
  __shared__ double s_sum[kThreads / 32];
  __shared__ long long s_cnt[kThreads / 32];
  const RigDev& rig = *rigp;
  double tsum = 0.0;
  long long tcnt = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const float P[3] = {__fmul_rn(pos[3 * k], inv_unit), __fmul_rn(pos[3 * k + 1], inv_unit),
                        __fmul_rn(pos[3 * k + 2], inv_unit)};
    float sum = 0.0f;
    int vis = 0;
    for (int i = 0; i < rig.n_cams; ++i) {
      const CamDev& C = rig.cam[i];
      const float d[3] = {__fsub_rn(P[0], C.cwc[0]), __fsub_rn(P[1], C.cwc[1]), __fsub_rn(P[2], C.cwc[2])};
      float a[3];
#pragma unroll
      for (int q = 0; q < 3; ++q)                     // T_i P = R (P - c), R = Rwc^T
        a[q] = __fmaf_rn(C.Rwc[q], d[0], __fmaf_rn(C.Rwc[3 + q], d[1], __fmul_rn(C.Rwc[6 + q], d[2])));
      if (!(a[2] > 0.0f)) continue;
      const float fu = __fadd_rn(__fmaf_rn(C.fx, __fdiv_rn(a[0], a[2]), C.cx), 0.5f);
      const float fv = __fadd_rn(__fmaf_rn(C.fy, __fdiv_rn(a[1], a[2]), C.cy), 0.5f);
      if (!(fu >= 0.0f && fu < (float)C.W && fv >= 0.0f && fv < (float)C.H)) continue;
      const int px = (int)fu, py = (int)fv;            // floor, both non-negative
      const DT D = __ldg(static_cast<const DT*>(fp.depth[i]) + (long long)py * C.W + px);
      if (!Depth<DT>::valid(D)) continue;
      const float zD = Depth<DT>::z(D);
      if (a[2] > __fadd_rn(zD, occl_u)) continue;       // hidden behind the observed surface
      sum = __fadd_rn(sum, fabsf(__fsub_rn(a[2], zD)));
      ++vis;
    }
    const float e = vis ? __fdiv_rn(sum, (float)vis) : __int_as_float(0x7fc00000);
    if (err) err[k] = vis ? __fmul_rn(e, unit_m) : e;
    if (nvis) nvis[k] = vis;
    if (vis) {
      tsum += (double)e;
      ++tcnt;
    }
  }
  // fixed-order block reduction
  for (int o = 16; o > 0; o >>= 1) {
    tsum += __shfl_down_sync(0xffffffffu, tsum, o);
    tcnt += __shfl_down_sync(0xffffffffu, tcnt, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { s_sum[warp] = tsum; s_cnt[warp] = tcnt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bs = 0.0;
    long long bc = 0;
    for (int w = 0; w < kThreads / 32; ++w) { bs += s_sum[w]; bc += s_cnt[w]; }
    bsum[blockIdx.x] = bs;
    bcnt[blockIdx.x] = bc;
  }
}

// ------------------------------------------------------------------ Eq. 3 confidence
// One 128x32 pixel tile per block, staged with its one-pixel halo in shared memory (raw
// depth samples; vector loads for the interior columns).  Each thread computes four
// consecutive pixels in each of four rows, 8 apart, and stores each quadruple as one float4;
// the four windows share one load of their 3x6 samples, and each window's variance is taken
// relative to its centre depth.  Depth
// gradient G: central difference where both neighbours are valid, one-sided with one, 0
// with none; sigma_local: population variance of the window's valid depths (m^2); C is
// normalised by alpha + gamma and is 0 where the depth is invalid.
constexpr int kConfW = 128, kConfH = 32;

template <typename DT>
__global__ void __launch_bounds__(kThreads) k_confidence(ConfArgs a) {
  constexpr int kVec = 16 / sizeof(DT);                  // samples per 16-byte load
  constexpr int kRowVecs = kConfW / kVec;
  constexpr int kOff = kVec;                             // tile column c at c + kOff: the
  constexpr int kRow = kConfW + 2 * kVec;                // interior starts 16-byte aligned
  __shared__ __align__(16) DT t[kConfH + 2][kRow];
  const int cam = blockIdx.z;
  const int W = a.W[cam], H = a.H[cam];
  const int x0 = blockIdx.x * kConfW, y0 = blockIdx.y * kConfH;
  if (x0 >= W || y0 >= H) return;                       // uniform over the block
  const DT* __restrict__ dep = static_cast<const DT*>(a.depth[cam]);
  const bool vec_ok = (W % kVec) == 0 && ((reinterpret_cast<uintptr_t>(dep) & 15) == 0);
  // interior columns: rows y0-1 .. y0+8, 16-byte loads where the whole vector is inside
  for (int i = threadIdx.x; i < (kConfH + 2) * kRowVecs; i += kThreads) {
    const int r = i / kRowVecs, v = i - r * kRowVecs;
    const int y = y0 - 1 + r, x = x0 + v * kVec;
    DT* dst = &t[r][kOff + v * kVec];
    if (y >= 0 && y < H && vec_ok && x + kVec <= W) {
      *reinterpret_cast<uint4*>(dst) = __ldcs(reinterpret_cast<const uint4*>(dep + (long long)y * W + x));
    } else {
#pragma unroll
      for (int k = 0; k < kVec; ++k)
        dst[k] = (y >= 0 && y < H && x + k < W) ? dep[(long long)y * W + x + k] : (DT)0;
    }
  }
  // halo columns x0-1 and x0+128 (invalid outside the image)
  if (threadIdx.x < 2 * (kConfH + 2)) {
    const int r = threadIdx.x >> 1, side = threadIdx.x & 1;
    const int y = y0 - 1 + r, x = side ? x0 + kConfW : x0 - 1;
    t[r][side ? kOff + kConfW : kOff - 1] = (y >= 0 && y < H && x >= 0 && x < W) ? dep[(long long)y * W + x] : (DT)0;
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, xb = x0 + 4 * tx;
  if (xb >= W) return;
  const int c0 = kOff + 4 * tx - 1;                       // smem column of pixel xb - 1
  for (int ty = threadIdx.x / 32; ty < kConfH; ty += kThreads / 32) {
    const int y = y0 + ty;
    if (y >= H) break;
    // the 3x6 samples of the thread's four windows, once, as depth (z) and validity
    float zz[3][6];
    bool vv[3][6];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const DT d = t[ty + r][c0 + c];
        vv[r][c] = Depth<DT>::valid(d);
        zz[r][c] = vv[r][c] ? Depth<DT>::z(d) : 0.0f;
      }
    float res[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (!vv[1][p + 1]) { res[p] = 0.0f; continue; }
      const float z0 = zz[1][p + 1];
      float g[2];
#pragma unroll
      for (int axis = 0; axis < 2; ++axis) {
        const bool vm = axis == 0 ? vv[1][p] : vv[0][p + 1];
        const bool vp = axis == 0 ? vv[1][p + 2] : vv[2][p + 1];
        const float zm = axis == 0 ? zz[1][p] : zz[0][p + 1];
        const float zp = axis == 0 ? zz[1][p + 2] : zz[2][p + 1];
        const float diff = vm && vp ? __fmul_rn(__fsub_rn(zp, zm), 0.5f)
                         : vp ? __fsub_rn(zp, z0) : vm ? __fsub_rn(z0, zm) : 0.0f;
        g[axis] = __fmul_rn(diff, a.scale);
      }
      const float G2 = __fmaf_rn(g[0], g[0], __fmul_rn(g[1], g[1]));
      const float G = G2 > 0.0f ? __fmul_rn(G2, rsqrtf(G2)) : 0.0f;   // |g|, a few ulp
      // window variance relative to the centre sample (one pass: the centre is one of the
      // samples, so the cancellation costs at most a factor 9 in relative precision)
      float n = 0.0f, sm = 0.0f, sq = 0.0f;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float e = vv[r][p + c] ? __fsub_rn(zz[r][p + c], z0) : 0.0f;
          n = __fadd_rn(n, vv[r][p + c] ? 1.0f : 0.0f);
          sm = __fadd_rn(sm, e);
          sq = __fmaf_rn(e, e, sq);
        }
      const float rn = __fdividef(1.0f, n);
      const float var = __fmul_rn(fmaxf(__fmul_rn(__fsub_rn(sq, __fmul_rn(__fmul_rn(sm, sm), rn)), rn), 0.0f),
                                  __fmul_rn(a.scale, a.scale));
      const float ta = __fdividef(a.alpha, __fmaf_rn(a.beta, G, 1.0f));
      const float tb = __fdividef(a.gamma, __fmaf_rn(a.delta, var, 1.0f));
      res[p] = __fmul_rn(__fadd_rn(ta, tb), a.inv_ag);
    }
    float* __restrict__ out = a.out[cam] + (long long)y * W + xb;
    if (xb + 4 <= W && (W & 3) == 0 && ((reinterpret_cast<uintptr_t>(a.out[cam]) & 15) == 0)) {
      __stcs(reinterpret_cast<float4*>(out), make_float4(res[0], res[1], res[2], res[3]));
    } else {
#pragma unroll
      for (int p = 0; p < 4; ++p)
        if (xb + p < W) out[p] = res[p];
    }
  }
}

__global__ void k_init_tables(Tables t, unsigned fcap, unsigned ccap) {
  const unsigned n = max(fcap, ccap);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < fcap) {
      t.frec[i].key = kKeyEmpty;
      t.frec[i].head = kSlotNone;
      t.frec[i].mmin = INT_MAX;
    }
    if (i < ccap) {
      t.coarse[i].key = kKeyEmpty;
      t.coarse[i].count = 0u;
    }
  }
}

// ------------------------------------------------------------------ depth screen
// D^r of Eq. 8 (stated rule: include/fuseflow.h, fuseflow_params): a valid sample within
// the depth-unit bounds is kept unless a valid in-bounds 4-neighbour differs from it by more
// than edge_rel times its value; every decision in float32, screened samples become 0.
template <typename DT>
__device__ __forceinline__ bool screen_keep(DT d, float min_u, float max_u) {
  if (!Depth<DT>::valid(d)) return false;
  const float z = Depth<DT>::z(d);
  return (min_u <= 0.0f || z >= min_u) && (max_u <= 0.0f || z <= max_u);
}

template <typename DT>
__global__ void __launch_bounds__(kThreads) k_screen(ScreenArgs a) {
  const int cam = blockIdx.y;
  const unsigned W = (unsigned)a.W[cam], H = (unsigned)a.H[cam], n = W * H;   // W H <= 2^30
  const DT* __restrict__ in = static_cast<const DT*>(a.in[cam]);
  DT* __restrict__ out = static_cast<DT*>(a.out[cam]);
  for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const DT d = __ldg(in + p);
    bool keep = screen_keep<DT>(d, a.min_u, a.max_u);
    if (keep && a.edge_rel > 0.0f) {
      const unsigned y = p / W, x = p - y * W;
      const float z = Depth<DT>::z(d), thr = __fmul_rn(a.edge_rel, z);
      auto jump = [&](unsigned q) {
        const DT e = __ldg(in + q);
        return screen_keep<DT>(e, a.min_u, a.max_u) && fabsf(__fsub_rn(z, Depth<DT>::z(e))) > thr;
      };
      if ((x > 0 && jump(p - 1)) || (x + 1 < W && jump(p + 1)) || (y > 0 && jump(p - W)) ||
          (y + 1 < H && jump(p + W)))
        keep = false;
    }
    out[p] = keep ? d : (DT)0;
  }
}

// The same screen for images whose rows start on 16-byte boundaries (every width a
// multiple of 8, 16-byte aligned buffers): a block covers 8 rows x 256 columns of one
// camera, a thread 8 consecutive pixels of one row, read and written as 16-byte vectors
// (two for float32).  The rows above and below come from the neighbouring warps' loads
// through L1/L2; left and right neighbours from the adjacent lanes, the warp's two outer
// ones by scalar loads.
template <typename DT>
__device__ __forceinline__ void load_row8(const DT* __restrict__ p, DT v[8]) {
  if constexpr (sizeof(DT) == 2) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) { v[2 * k] = (DT)(w[k] & 0xffffu); v[2 * k + 1] = (DT)(w[k] >> 16); }
  } else {
    const float4 f0 = __ldg(reinterpret_cast<const float4*>(p));
    const float4 f1 = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = f0.x; v[1] = f0.y; v[2] = f0.z; v[3] = f0.w;
    v[4] = f1.x; v[5] = f1.y; v[6] = f1.z; v[7] = f1.w;
  }
}

template <typename DT>
__device__ __forceinline__ void store_row8(DT* __restrict__ p, const DT v[8]) {
  if constexpr (sizeof(DT) == 2) {
    uint4 u;
    u.x = (unsigned)v[0] | ((unsigned)v[1] << 16);
    u.y = (unsigned)v[2] | ((unsigned)v[3] << 16);
    u.z = (unsigned)v[4] | ((unsigned)v[5] << 16);
    u.w = (unsigned)v[6] | ((unsigned)v[7] << 16);
    *reinterpret_cast<uint4*>(p) = u;
  } else {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
  }
}

template <typename DT>
__device__ __forceinline__ DT shfl_depth(DT v, int delta, bool up) {
  if constexpr (sizeof(DT) == 2) {
    const unsigned u = up ? __shfl_up_sync(0xffffffffu, (unsigned)v, delta)
                          : __shfl_down_sync(0xffffffffu, (unsigned)v, delta);
    return (DT)u;
  } else {
    return up ? __shfl_up_sync(0xffffffffu, v, delta) : __shfl_down_sync(0xffffffffu, v, delta);
  }
}

template <typename DT>
__global__ void __launch_bounds__(kThreads) k_screen_rows(ScreenArgs a) {
  const int cam = blockIdx.z;
  const int W = a.W[cam], H = a.H[cam];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int y = blockIdx.y * 8 + warp;
  const int x0 = blockIdx.x * 256 + lane * 8;
  const bool active = y < H && x0 < W;              // W % 8 == 0: all 8 pixels inside
  const DT* __restrict__ in = static_cast<const DT*>(a.in[cam]);
  DT v[8], up[8], dn[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) { v[k] = (DT)0; up[k] = (DT)0; dn[k] = (DT)0; }
  if (active) {
    const size_t row = (size_t)y * (size_t)W + (size_t)x0;
    load_row8<DT>(in + row, v);
    if (y > 0) load_row8<DT>(in + row - W, up);
    if (y + 1 < H) load_row8<DT>(in + row + W, dn);
  }
  // neighbours across the thread's 8-pixel group: adjacent lanes, or a scalar load at the
  // warp's edges (a sample outside the image counts as invalid: it never screens)
  DT left = shfl_depth<DT>(v[7], 1, true), right = shfl_depth<DT>(v[0], 1, false);
  if (lane == 0) left = (active && x0 > 0) ? __ldg(in + (size_t)y * W + x0 - 1) : (DT)0;
  if (lane == 31) right = (active && x0 + 8 < W) ? __ldg(in + (size_t)y * W + x0 + 8) : (DT)0;
  if (x0 + 8 >= W) right = (DT)0;
  if (!active) return;
  // valid and within the bounds as two compares: z >= lo and z <= hi, with lo the lower
  // bound or the smallest positive float (so that 0, negatives and NaN fail) and hi the
  // upper bound or the largest finite float (so that +inf fails); the same decision as
  // screen_keep (no flush of subnormals in this build)
  const float lo = a.min_u > 0.0f ? a.min_u : __int_as_float(1);
  const float hi = a.max_u > 0.0f ? a.max_u : __int_as_float(0x7f7fffff);
  float zc[8], zu[8], zd[8];
  bool oc[8], ou[8], od[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    zc[k] = Depth<DT>::z(v[k]);
    zu[k] = Depth<DT>::z(up[k]);
    zd[k] = Depth<DT>::z(dn[k]);
    oc[k] = zc[k] >= lo && zc[k] <= hi;
    ou[k] = zu[k] >= lo && zu[k] <= hi;
    od[k] = zd[k] >= lo && zd[k] <= hi;
  }
  const float zl = Depth<DT>::z(left), zr = Depth<DT>::z(right);
  const bool ol = zl >= lo && zl <= hi, orr = zr >= lo && zr <= hi;
  const float rel = a.edge_rel;
  DT o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    bool keep = oc[k];
    if (rel > 0.0f) {
      const float z = zc[k], thr = __fmul_rn(rel, z);
      const float zw = k > 0 ? zc[k - 1] : zl, ze = k < 7 ? zc[k + 1] : zr;
      const bool ow = k > 0 ? oc[k - 1] : ol, oe = k < 7 ? oc[k + 1] : orr;
      const bool jump = (ow && fabsf(__fsub_rn(z, zw)) > thr) || (oe && fabsf(__fsub_rn(z, ze)) > thr) ||
                        (ou[k] && fabsf(__fsub_rn(z, zu[k])) > thr) ||
                        (od[k] && fabsf(__fsub_rn(z, zd[k])) > thr);
      keep = keep && !jump;
    }
    o[k] = keep ? v[k] : (DT)0;
  }
  store_row8<DT>(static_cast<DT*>(a.out[cam]) + (size_t)y * W + x0, o);
}

template <typename DT, int TH>
cudaError_t set_assign_attributes_th() {
  const int sm = (int)AssignTile<TH>::smem(kMaxK1);
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_assign<DT, false, false, 1, TH>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_assign<DT, false, true, 1, TH>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_assign<DT, true, false, 1, TH>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_assign<DT, true, true, 1, TH>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_assign<DT, false, false, kMaxBatch, TH>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_assign<DT, true, false, kMaxBatch, TH>, at, sm);
  return e;
}

// Dynamic shared memory limit of the assign kernels for one depth type, set once per device
// (the first call comes from context creation, outside any stream capture).  The attribute
// call is idempotent, so two host threads that race here only repeat it.
template <typename DT>
cudaError_t set_assign_attributes() {
  static std::atomic<unsigned long long> done{0ull};       // one bit per device (< 64)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  cudaError_t e = set_assign_attributes_th<DT, 8>();
  if (e == cudaSuccess) e = set_assign_attributes_th<DT, 16>();
  if (e == cudaSuccess) e = set_assign_attributes_th<DT, 32>();
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Launch of one of the frame's kernels; pdl: programmatic stream serialization with the
// kernel before it on the stream (the kernel must call pdl_wait before using its results).
template <typename... P, typename... A>
cudaError_t launch_k(bool pdl, void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     A... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// The assign step over the batch's tiles (TH rows a tile; the traced instantiation exists for
// single frames only).
template <typename DT, int NB, int TH>
cudaError_t launch_assign(const BatchArgs<NB>& a, int n, bool top_k, bool traced, int max_k1, bool pdl,
                          cudaStream_t s) {
  const dim3 tiles(a.tile_first[n]), at(AssignTile<TH>::Threads);
  const size_t sm = AssignTile<TH>::smem(top_k ? 0 : max_k1);
  if constexpr (NB == 1) {
    if (traced)
      return top_k ? launch_k(pdl, k_assign<DT, true, true, NB, TH>, tiles, at, sm, s, a)
                   : launch_k(pdl, k_assign<DT, false, true, NB, TH>, tiles, at, sm, s, a);
  }
  return top_k ? launch_k(pdl, k_assign<DT, true, false, NB, TH>, tiles, at, sm, s, a)
               : launch_k(pdl, k_assign<DT, false, false, NB, TH>, tiles, at, sm, s, a);
}

// The frame kernels over n frames (NB = 1: one frame; NB = kMaxBatch: a batch of up to
// that many frames of any rigs, every kernel launched once for all of them).
template <typename DT, int NB>
cudaError_t launch_frames(const FrameLaunch* fr, int n, cudaStream_t s, cudaEvent_t* ev) {
  const cudaError_t ae = set_assign_attributes<DT>();
  if (ae != cudaSuccess) return ae;
  if (n < 1 || n > NB) return cudaErrorInvalidValue;
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], s); };
  mark(0);
  static thread_local BatchArgs<NB> a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  int emit = 1, pdl_level = 2, max_wblocks = 1, max_k1 = 0;
  const Geometry& g0 = *fr[0].geo;
  cudaError_t err = cudaSuccess;
  for (int f = 0; f < n; ++f) {
    const Geometry& geo = *fr[f].geo;
    const Tables& t = fr[f].t;
    err = cudaMemsetAsync(t.cnt, 0, sizeof(FrameCounters) + sizeof(unsigned) * (size_t)t.n_words, s);
    if (err != cudaSuccess) return err;
    FrameArgs& fa = a.f[f];
    fa.rig = fr[f].rig;
    fa.rays = fr[f].rays;
    fa.fp = fr[f].fp;
    fa.t = t;
    fa.tr = fr[f].tr;
    fa.out = fr[f].out;
    fa.ti = geo.tiles;
    fa.count_blocks_x = geo.count_blocks_x;
    fa.count_chunks = geo.count_chunks;
    fa.unit_m = (float)fr[f].out.unit_m;
    if (geo.screen) {                      // D^r of Eq. 8 into the context's buffers
      ScreenArgs sa = geo.scr;
      for (int i = 0; i < geo.n_cams; ++i) {
        sa.in[i] = fr[f].fp.depth[i];
        fa.fp.depth[i] = sa.out[i];
      }
      if ((err = launch_screen(sa, sizeof(DT) == 4, geo.max_px, s)) != cudaSuccess) return err;
    }
    a.count_first[f + 1] = a.count_first[f] + geo.count_blocks_x * geo.n_cams;
    a.tile_first[f + 1] = a.tile_first[f] + t.n_tiles;
    emit = std::max(emit, geo.emit_blocks);
    pdl_level = std::min(pdl_level, geo.pdl);
    max_wblocks = std::max(max_wblocks, t.n_wblocks);
    max_k1 = std::max(max_k1, geo.tiles.k1);
  }
  mark(1);
  // programmatic launches between the kernels when the geometry asks for them (level 2
  // also between the assign and reduce steps), never while stage events are recorded
  const bool pdl = pdl_level >= 1 && ev == nullptr;
  const bool pdl_reduce = pdl_level >= 2 && ev == nullptr;
  const dim3 eb(emit, n), th3(kThreads);
  if ((err = launch_k(false, k_count<DT, NB>, dim3(a.count_first[n]), th3, 0, s, a)) != cudaSuccess ||
      (err = launch_k(pdl, k_levels<NB>, eb, th3, 0, s, a)) != cudaSuccess)
    return err;
  mark(2);
  bool traced = false;
  for (int f = 0; f < n; ++f) {
    const TraceDev& tr = fr[f].tr;
    traced = traced || tr.pw || tr.omega || tr.e || tr.nview || tr.key;
  }
  const int th = g0.tiles.th;
  if (th == 8) err = launch_assign<DT, NB, 8>(a, n, g0.top_k != 0, traced, max_k1, pdl, s);
  else if (th == 32) err = launch_assign<DT, NB, 32>(a, n, g0.top_k != 0, traced, max_k1, pdl, s);
  else err = launch_assign<DT, NB, 16>(a, n, g0.top_k != 0, traced, max_k1, pdl, s);
  if (err != cudaSuccess) return err;
  mark(3);
  if (g0.top_k) {
    if ((err = launch_k(pdl_reduce, k_reduce_topk<DT, NB>, eb, th3, 0, s, a)) != cudaSuccess) return err;
  } else {
    if ((err = launch_k(pdl_reduce, k_reduce<NB>, eb, th3, 0, s, a)) != cudaSuccess) return err;
  }
  mark(4);
  if ((err = launch_k(pdl, k_scan<NB>, dim3(max_wblocks, n), dim3(1024), 0, s, a)) != cudaSuccess) return err;
  mark(5);
  if ((err = launch_k(pdl, k_emit<NB>, eb, th3, 0, s, a)) != cudaSuccess) return err;
  mark(6);
  return cudaGetLastError();
}

}  // namespace

namespace {
template <int TH>
int resident_th(int k1) {
  static std::atomic<int> cache[kMaxK1 + 1];             // 0: not yet asked
  k1 = std::max(0, std::min(k1, kMaxK1));
  const int known = cache[k1].load(std::memory_order_relaxed);
  if (known > 0) return known;
  int n = 0;
  const int sm = (int)AssignTile<TH>::smem(k1);
  if (set_assign_attributes<uint16_t>() != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_assign<uint16_t, false, false, 1, TH>,
                                                    AssignTile<TH>::Threads, sm) != cudaSuccess) {
    cudaGetLastError();
    return AssignTile<TH>::BlocksPerSM;
  }
  n = std::max(1, n);
  cache[k1].store(n, std::memory_order_relaxed);
  return n;
}
}  // namespace

int assign_resident_blocks(int th, int k1) {
  return th == 8 ? resident_th<8>(k1) : th == 32 ? resident_th<32>(k1) : resident_th<16>(k1);
}

int retile(TileIndex* ti, int th) {
  ti->th = th;
  int n = 0;
  for (int i = 0; i < ti->n_cams; ++i) {
    ti->first[i] = n;
    n += ((ti->W[i] + kTileW - 1) / kTileW) * ((ti->H[i] + th - 1) / th);
  }
  ti->first[ti->n_cams] = n;
  bool same = true;
  for (int i = 1; i < ti->n_cams; ++i) same = same && ti->W[i] == ti->W[0] && ti->H[i] == ti->H[0];
  ti->per_cam = same && ti->n_cams > 0 ? ti->first[1] : 0;
  return n;
}

int fill_tile_index(const RigDev& rig, TileIndex* out, int th) {
  memset(out, 0, sizeof(*out));
  out->n_cams = rig.n_cams;
  out->k1 = rig.k1;
  for (int i = 0; i < rig.n_cams; ++i) {
    out->W[i] = rig.cam[i].W;
    out->H[i] = rig.cam[i].H;
    out->off[i] = rig.cam[i].off;
    out->pray[i] = rig.k1 > 0 ? rig.pair[rig.cam[i].pair0].ga : 0;
  }
  out->ahead = kNoPrefetch;                      // no prefetch unless the caller sets it
  return retile(out, th);
}

void fill_block_consts(const RigDev& rig, BlockConst* out) {
  for (int i = 0; i < rig.n_cams; ++i) {
    BlockConst& b = out[i];
    memset(&b, 0, sizeof(b));
    b.cam = rig.cam[i];
    for (int q = 0; q < rig.k1; ++q) {
      b.pair[q] = rig.pair[rig.cam[i].pair0 + q];
      b.nb[q] = rig.cam[b.pair[q].j];
    }
  }
}

cudaError_t launch_init_tables(const Tables& t, unsigned fcap, unsigned ccap, cudaStream_t s) {
  k_init_tables<<<1024, 256, 0, s>>>(t, fcap, ccap);
  return cudaGetLastError();
}

cudaError_t launch_copyout(const fuseflow_cloud& src, const HostOutDev& dst, cudaStream_t s) {
  k_copyout<<<4 * 152, kThreads, 0, s>>>(src, dst);
  return cudaGetLastError();
}

cudaError_t launch_confidence(const ConfArgs& a, bool depth_f32, int max_w, int max_h,
                              cudaStream_t s) {
  const dim3 g((max_w + kConfW - 1) / kConfW, (max_h + kConfH - 1) / kConfH, a.n_cams);
  if (depth_f32) k_confidence<float><<<g, kThreads, 0, s>>>(a);
  else k_confidence<uint16_t><<<g, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

int mc_blocks(long long n) { return (int)std::max(1ll, std::min<long long>(kMcBlocks, (n + kThreads - 1) / kThreads)); }

cudaError_t launch_mc(const RigDev* rig, const FramePtrs& fp, bool depth_f32, const float* pos,
                      long long n, double unit_m, double occlusion_m, float* err, int* nvis,
                      double* bsum, long long* bcnt, cudaStream_t s) {
  const int g = mc_blocks(n);
  const float inv = (float)(1.0 / unit_m), um = (float)unit_m;
  const float occl = (float)(occlusion_m / unit_m);      // +inf stays +inf
  if (depth_f32) k_mc<float><<<g, kThreads, 0, s>>>(rig, fp, pos, n, inv, um, occl, err, nvis, bsum, bcnt);
  else k_mc<uint16_t><<<g, kThreads, 0, s>>>(rig, fp, pos, n, inv, um, occl, err, nvis, bsum, bcnt);
  return cudaGetLastError();
}

cudaError_t launch_points(const RigDev* rig, const float2* rays, const FramePtrs& fp, const Tables& t,
                          const PointsDev& out, bool depth_f32, int n_cams, long long max_px,
                          cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out.counts, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const long long per = (max_px + kThreads - 1) / kThreads;
  const dim3 g((unsigned)std::max(1ll, std::min<long long>(per, 4 * 152)), n_cams);
  if (depth_f32) k_points<float><<<g, kThreads, 0, s>>>(rig, rays, fp, t, out);
  else k_points<uint16_t><<<g, kThreads, 0, s>>>(rig, rays, fp, t, out);
  return cudaGetLastError();
}

cudaError_t launch_screen(const ScreenArgs& a, bool depth_f32, long long max_px, cudaStream_t s) {
  bool rows = true;                                   // 16-byte rows: the vector kernel
  int max_w = 1, max_h = 1;
  for (int i = 0; i < a.n_cams; ++i) {
    rows = rows && a.W[i] % 8 == 0 && (reinterpret_cast<uintptr_t>(a.in[i]) & 15) == 0 &&
           (reinterpret_cast<uintptr_t>(a.out[i]) & 15) == 0;
    max_w = std::max(max_w, a.W[i]);
    max_h = std::max(max_h, a.H[i]);
  }
  if (rows) {
    const dim3 grid((unsigned)((max_w + 255) / 256), (unsigned)((max_h + 7) / 8), (unsigned)a.n_cams);
    if (depth_f32) k_screen_rows<float><<<grid, kThreads, 0, s>>>(a);
    else k_screen_rows<uint16_t><<<grid, kThreads, 0, s>>>(a);
  } else {
    const unsigned bx = (unsigned)std::min<long long>((max_px + kThreads - 1) / kThreads, 4096);
    const dim3 grid(std::max(1u, bx), a.n_cams);
    if (depth_f32) k_screen<float><<<grid, kThreads, 0, s>>>(a);
    else k_screen<uint16_t><<<grid, kThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t prepare_launch(bool depth_f32) {
  return depth_f32 ? set_assign_attributes<float>() : set_assign_attributes<uint16_t>();
}

cudaError_t launch_frame(const RigDev* rig, const float2* rays, const FramePtrs& fp, const Tables& t,
                         const TraceDev& tr, const OutDev& out, const Geometry& geo, cudaStream_t s,
                         cudaEvent_t* ev) {
  const FrameLaunch fl{rig, rays, fp, t, tr, out, &geo};
  if (geo.depth_f32) return launch_frames<float, 1>(&fl, 1, s, ev);
  return launch_frames<uint16_t, 1>(&fl, 1, s, ev);
}

cudaError_t launch_batch(const FrameLaunch* frames, int n, cudaStream_t s) {
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  for (int f = 1; f < n; ++f)                       // one depth type and one fusion variant
    if (frames[f].geo->depth_f32 != frames[0].geo->depth_f32 || frames[f].geo->top_k != frames[0].geo->top_k ||
        frames[f].geo->tiles.th != frames[0].geo->tiles.th)
      return cudaErrorInvalidValue;
  if (frames[0].geo->depth_f32) return launch_frames<float, kMaxBatch>(frames, n, s, nullptr);
  return launch_frames<uint16_t, kMaxBatch>(frames, n, s, nullptr);
}

}  // namespace ffl
