// ff_kernels.cu - sm_103a kernels of the FUSE-Flow per-frame fusion path.
//
// Launch sequence of one frame (all on the caller's stream):
//   memset   frame counters + representative bitmap
//   count    (a) decode + gate + back-project (Eq. 8, 9), coarse density n_c (Sec. II.5(1)c),
//            per-block pixel counts and extent (Sec. II.5(1)b)
//   assign   (b) consistency V (Eq. 4-7), omega = C V (Eq. 10) as mantissa/exponent;
//            (c) level per coarse cell (Sec. II.5(1)d), cell key (Sec. II.5(1)e), fine
//            hash insertion; per-cell member count, representative (Sec. II.5(2)a) and
//            smallest weight exponent
//   accum    (d) exact fixed-point sums of omega, omega P, omega RGB per cell (Eq. 11)
//   scan     ranks of the representatives (output order), frame statistics
//   emit     fused cells, then the used hash slots are cleared for the next frame
//
// Reductions are order-independent: integer atomics only (counts, max, min and
// fixed-point sums), so the output is bitwise reproducible.
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
    unsigned long long cur = __ldcg(&t.meta[h].key);
    if (cur == key) return h;
    if (cur == kKeyEmpty) {
      cur = atomicCAS(&t.meta[h].key, kKeyEmpty, key);
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
    const K prev = atomicCAS(&tab[h], empty, key);
    if (prev == empty || prev == key) return (int)h;
    h = (h + 1) & (TS - 1);
  }
  return -1;
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
__device__ __forceinline__ void residual_sum(const RigDev& rig, const CamDev& C,
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
  for (int q = 0; q < rig.k1; ++q) {
    const PairDev& P = rig.pair[C.pair0 + q];
    const CamDev& J = rig.cam[P.j];
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
    const DT Dj = static_cast<const DT*>(fp.depth[P.j])[(long long)py * J.W + px];
    if (!Depth<DT>::valid(Dj)) continue;
    if (!have) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
        ff_affine_row(P.Rh + 3 * k, P.Rl + 3 * k, P.th[k], P.tl[k], pxh, pxl, pyh, pyl, z,
                      ah[k], al[k]);
    }
    // Eq. 5: Q = D_j(u_j) (rx_j, ry_j, 1) in camera-j coordinates (rigid motion keeps d).
    const float zj = Depth<DT>::z(Dj);
    const float2 qx = rays[J.ray_x + px], qy = rays[J.ray_y + py];
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
__global__ void __launch_bounds__(kThreads)
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
  DT dv[4];
  float cv[4];
  unsigned nv = 0, ng = 0, noor = 0;
  unsigned bmin[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, bmax[3] = {0u, 0u, 0u};
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
          world_point(C, Depth<DT>::z(dv[k]), rays[C.ray_x + x].x, rays[C.ray_y + y].x, P);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const unsigned o = ordered(P[a]);
            bmin[a] = min(bmin[a], o);
            bmax[a] = max(bmax[a], o);
          }
          if (grid_coords(rig, P, r)) {
            const int h = local_pos<TS>(s_key, kKeyEmpty, coarse_key(r));
            if (h >= 0) atomicAdd(&s_cnt[h], 1u);
            else atomicOr(&t.cnt->error, kErrCoarseFull);
          } else {
            ++noor;
          }
        }
      }
      if (++x == C.W) { x = 0; ++y; }
    }
  }
  // per-block pixel counts and extent
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  // flush the block's coarse counts (Sec. II.5(1)c density estimate)
  for (int i = threadIdx.x; i < TS; i += kThreads) {
    const unsigned long long key = s_key[i];
    if (key == kKeyEmpty) continue;
    const unsigned slot = coarse_insert(t, key);
    if (slot != kSlotNone) atomicAdd(&t.ccount[slot], s_cnt[i]);
  }
}

// ------------------------------------------------------------------ assign step
template <typename DT>
__global__ void __launch_bounds__(kThreads)
k_assign(const RigDev* __restrict__ rigp, const float2* __restrict__ rays, FramePtrs fp, Tables t,
         TraceDev tr, float unit_m) {
  constexpr int TS = 2 * kTilePx;
  __shared__ unsigned long long s_ck[TS];
  __shared__ unsigned char s_cl[TS];
  __shared__ unsigned long long s_fk[TS];
  __shared__ unsigned s_fcnt[TS];
  __shared__ unsigned long long s_frep[TS];
  __shared__ int s_fmin[TS];
  __shared__ unsigned s_fslot[TS];
  const RigDev& rig = *rigp;
  const int cam = blockIdx.y;
  const CamDev& C = rig.cam[cam];
  const int tiles_x = (C.W + kTileW - 1) / kTileW;
  const int tiles_y = (C.H + kTileH - 1) / kTileH;
  if ((int)blockIdx.x >= tiles_x * tiles_y) return;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < TS; i += kThreads) {
    s_ck[i] = kKeyEmpty;
    s_fk[i] = kKeyEmpty;
    s_fcnt[i] = 0;
    s_frep[i] = 0ull;
    s_fmin[i] = INT_MAX;
  }
  __syncthreads();

  const DT* __restrict__ dep = static_cast<const DT*>(fp.depth[cam]);
  const float* __restrict__ cf = fp.conf[cam];
  const bool trace = tr.pw || tr.omega || tr.e || tr.nview || tr.key;
  float r[2][3];
  bool has[2] = {false, false};
  bool inb[2] = {false, false};
  float mu[2] = {0.0f, 0.0f};
  int mexp[2] = {0, 0};
  unsigned long long rank[2] = {0ull, 0ull};
  int hc[2] = {-1, -1}, hf[2] = {-1, -1};
  long long gi[2] = {0, 0};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int x = tx * kTileW + lane, y = ty * kTileH + warp + 8 * k;
    if (x >= C.W || y >= C.H) continue;
    inb[k] = true;
    const long long li = (long long)y * C.W + x;
    gi[k] = C.off + li;
    const DT D = dep[li];
    const float c = cf[li];
    float eh = __int_as_float(0x7fc00000), P[3] = {eh, eh, eh};
    int nview = -1;
    if (Depth<DT>::valid(D) && (!rig.use_conf || c > rig.tau)) {   // Eq. 9
      const float z = Depth<DT>::z(D);
      const float2 rx = rays[C.ray_x + x], ry = rays[C.ray_y + y];
      world_point(C, z, rx.x, ry.x, P);                               // Eq. 8
      float sh = 0.0f, sl = 0.0f, el = 0.0f;
      nview = 0;
      eh = 0.0f;
      if (rig.use_cons && rig.k1 > 0) {
        residual_sum<DT>(rig, C, rays, fp, z, rx, ry, sh, sl, nview);
        fast_two_sum(sh, sl, sh, sl);
        two_prod(sh, rig.einv_h, eh, el);                             // Eq. 7 exponent
        el = __fmaf_rn(sh, rig.einv_l, __fmaf_rn(sl, rig.einv_h, el));
        fast_two_sum(eh, el, eh, el);
      }
      // omega = C exp(-e) = mu 2^-m with e = m ln2 + f, f in [0, ln2): mu never underflows
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
      const float base = rig.use_conf ? c : 1.0f;                     // Eq. 10
      mu[k] = __fmul_rn(__fmul_rn(base, expf(-fh)), __fsub_rn(1.0f, fl));
      mexp[k] = m;
      rank[k] = ((unsigned long long)ordered(c) << 32) | (unsigned)(~(unsigned)gi[k]);
      if (grid_coords(rig, P, r[k])) {
        has[k] = true;
        hc[k] = local_pos<TS>(s_ck, kKeyEmpty, coarse_key(r[k]));
        if (hc[k] < 0) { has[k] = false; atomicOr(&t.cnt->error, kErrCoarseFull); }
      }
    }
    if (trace) {
      if (tr.pw) {
        tr.pw[3 * gi[k] + 0] = P[0] * unit_m;
        tr.pw[3 * gi[k] + 1] = P[1] * unit_m;
        tr.pw[3 * gi[k] + 2] = P[2] * unit_m;
      }
      if (tr.e) tr.e[gi[k]] = eh;
      if (tr.omega) tr.omega[gi[k]] = nview >= 0 ? ldexpf(mu[k], -mexp[k]) : __int_as_float(0x7fc00000);
      if (tr.nview) tr.nview[gi[k]] = nview;
    }
  }
  __syncthreads();
  // Sec. II.5(1)d: the level of each coarse cell present in the tile
  for (int i = threadIdx.x; i < TS; i += kThreads) {
    const unsigned long long ck = s_ck[i];
    if (ck == kKeyEmpty) continue;
    s_cl[i] = (unsigned char)level_for(coarse_count_of(t, ck), rig.n_min, rig.max_level);
  }
  __syncthreads();
  // Sec. II.5(1)e: cell key; block-local member count, representative, weight exponent
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    unsigned long long fk = kKeyEmpty;
    if (has[k]) {
      fk = fine_key(r[k], s_cl[hc[k]]);
      hf[k] = local_pos<TS>(s_fk, kKeyEmpty, fk);
      if (hf[k] >= 0) {
        atomicAdd(&s_fcnt[hf[k]], 1u);
        atomicMax(&s_frep[hf[k]], rank[k]);
        atomicMin(&s_fmin[hf[k]], mexp[k]);
      } else {
        has[k] = false;
        atomicOr(&t.cnt->error, kErrFineFull);
      }
    }
    if (trace && tr.key && inb[k]) tr.key[gi[k]] = has[k] ? fk : kKeyEmpty;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TS; i += kThreads) {
    const unsigned long long fk = s_fk[i];
    if (fk == kKeyEmpty) continue;
    const unsigned slot = fine_insert(t, fk);
    s_fslot[i] = slot;
    if (slot != kSlotNone) {
      atomicAdd(&t.meta[slot].count, s_fcnt[i]);
      atomicMax(&t.meta[slot].rep, s_frep[i]);
      atomicMin(&t.meta[slot].mmin, s_fmin[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (!inb[k]) continue;
    Rec rc;
    rc.slot = has[k] ? s_fslot[hf[k]] : kSlotNone;
    rc.mu = mu[k];
    rc.m = mexp[k];
    t.rec[gi[k]] = rc;
  }
}

// ------------------------------------------------------------------ accumulate step
template <typename DT>
__global__ void __launch_bounds__(kThreads)
k_accum(const RigDev* __restrict__ rigp, const float2* __restrict__ rays, FramePtrs fp, Tables t) {
  constexpr int TS = 2 * kTilePx;
  constexpr int NL = kTilePx;
  __shared__ unsigned s_hk[TS];
  __shared__ int s_hi[TS];
  __shared__ unsigned s_slot[NL];
  __shared__ unsigned long long s_key[NL];
  __shared__ unsigned s_repg[NL];
  __shared__ int s_min[NL];
  __shared__ unsigned long long s_acc[7][NL];
  __shared__ unsigned s_n;
  const RigDev& rig = *rigp;
  const int cam = blockIdx.y;
  const CamDev& C = rig.cam[cam];
  const int tiles_x = (C.W + kTileW - 1) / kTileW;
  const int tiles_y = (C.H + kTileH - 1) / kTileH;
  if ((int)blockIdx.x >= tiles_x * tiles_y) return;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < TS; i += kThreads) s_hk[i] = kSlotNone;
  for (int i = threadIdx.x; i < NL; i += kThreads)
    for (int a = 0; a < 7; ++a) s_acc[a][i] = 0ull;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();

  const DT* __restrict__ dep = static_cast<const DT*>(fp.depth[cam]);
  const uint8_t* __restrict__ col = fp.rgb[cam];
  Rec rc[2];
  int h[2] = {-1, -1};
  int xs[2], ys[2];
  long long gi[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    xs[k] = tx * kTileW + lane;
    ys[k] = ty * kTileH + warp + 8 * k;
    rc[k].slot = kSlotNone;
    gi[k] = 0;
    if (xs[k] >= C.W || ys[k] >= C.H) continue;
    gi[k] = C.off + (long long)ys[k] * C.W + xs[k];
    rc[k] = t.rec[gi[k]];
    if (rc[k].slot != kSlotNone) h[k] = local_pos<TS>(s_hk, kSlotNone, rc[k].slot);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TS; i += kThreads) {
    const unsigned slot = s_hk[i];
    if (slot == kSlotNone) continue;
    const int idx = (int)atomicAdd(&s_n, 1u);
    s_hi[i] = idx;
    s_slot[idx] = slot;
    const SlotMeta m = t.meta[slot];
    s_key[idx] = m.key;
    s_repg[idx] = ~(unsigned)(m.rep & 0xffffffffull);
    s_min[idx] = m.mmin;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (h[k] < 0) continue;
    const int idx = s_hi[h[k]];
    const long long li = (long long)ys[k] * C.W + xs[k];
    float P[3], r[3];
    world_point(C, Depth<DT>::z(dep[li]), rays[C.ray_x + xs[k]].x, rays[C.ray_y + ys[k]].x, P);
    grid_coords(rig, P, r);
    const unsigned long long key = s_key[idx];
    const int l = (int)(key >> 60);
    const int kk[3] = {(int)((key >> 40) & 0xfffff) - kKeyBias, (int)((key >> 20) & 0xfffff) - kKeyBias,
                       (int)(key & 0xfffff) - kKeyBias};
    const int sh = rc[k].m - s_min[idx];
    const float w = sh > 62 ? 0.0f : ldexpf(rc[k].mu, kFixShift - sh);
    unsigned long long q[7];
    q[0] = __float2ull_rn(w);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float frac = __fsub_rn(ldexpf(r[a], l), (float)kk[a]);  // in [0, 1]
      q[1 + a] = __float2ull_rn(__fmul_rn(w, frac));
    }
    const uint8_t* px = col + 3 * li;
#pragma unroll
    for (int a = 0; a < 3; ++a) q[4 + a] = __float2ull_rn(__fmul_rn(w, (float)px[a] * 0.00390625f));
#pragma unroll
    for (int a = 0; a < 7; ++a) atomicAdd(&s_acc[a][idx], q[a]);
    if ((unsigned)gi[k] == s_repg[idx])
      atomicOr(&t.bitmap[gi[k] >> 5], 1u << (gi[k] & 31));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (int)s_n; i += kThreads) {
    SlotAcc* A = &t.acc[s_slot[i]];
    atomicAdd(&A->w, s_acc[0][i]);
    atomicAdd(&A->x, s_acc[1][i]);
    atomicAdd(&A->y, s_acc[2][i]);
    atomicAdd(&A->z, s_acc[3][i]);
    atomicAdd(&A->r, s_acc[4][i]);
    atomicAdd(&A->g, s_acc[5][i]);
    atomicAdd(&A->b, s_acc[6][i]);
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

// ------------------------------------------------------------------ emit + clear
__global__ void __launch_bounds__(kThreads) k_emit(Tables t, OutDev out) {
  const unsigned n_cells = min(t.cnt->n_cells, t.fmask + 1u);
  const unsigned n_coarse = min(t.cnt->n_coarse, t.cmask + 1u);
  const unsigned n = max(n_cells, n_coarse);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < n_cells) {
      const unsigned slot = t.fused[i];
      const SlotMeta m = t.meta[slot];
      const SlotAcc A = t.acc[slot];
      const unsigned g = ~(unsigned)(m.rep & 0xffffffffull);
      const unsigned w = g >> 5;
      const unsigned long long rnk = (unsigned long long)t.bsum[w >> 10] + t.wprefix[w] +
                                     __popc(t.bitmap[w] & ((1u << (g & 31)) - 1u));
      if (rnk < (unsigned long long)out.max_cells) {
        const int l = (int)(m.key >> 60);
        const double edge = ldexp(out.s0_m, -l);
        const double kx = (double)((int)((m.key >> 40) & 0xfffff) - kKeyBias);
        const double ky = (double)((int)((m.key >> 20) & 0xfffff) - kKeyBias);
        const double kz = (double)((int)(m.key & 0xfffff) - kKeyBias);
        const double W = (double)A.w;
        const double inv = A.w ? 1.0 / W : __longlong_as_double(0x7ff8000000000000ll);
        out.pos[3 * rnk + 0] = (float)(edge * (kx + (double)A.x * inv));
        out.pos[3 * rnk + 1] = (float)(edge * (ky + (double)A.y * inv));
        out.pos[3 * rnk + 2] = (float)(edge * (kz + (double)A.z * inv));
        out.rgb[3 * rnk + 0] = (float)(256.0 * (double)A.r * inv);
        out.rgb[3 * rnk + 1] = (float)(256.0 * (double)A.g * inv);
        out.rgb[3 * rnk + 2] = (float)(256.0 * (double)A.b * inv);
        out.weight[rnk] = (float)ldexp(W, -kFixShift - m.mmin);
        out.count[rnk] = m.count;
        out.rep[rnk] = g;
        out.key[rnk] = m.key;
      }
      SlotMeta z;
      z.key = kKeyEmpty;
      z.rep = 0ull;
      z.mmin = INT_MAX;
      z.count = 0u;
      z.pad = 0ull;
      t.meta[slot] = z;
      SlotAcc za = {};
      t.acc[slot] = za;
    }
    if (i < n_coarse) {
      const unsigned cs = t.cused[i];
      t.ckey[cs] = kKeyEmpty;
      t.ccount[cs] = 0u;
    }
  }
}

__global__ void k_init_tables(Tables t, unsigned fcap, unsigned ccap) {
  const unsigned n = max(fcap, ccap);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < fcap) {
      SlotMeta z;
      z.key = kKeyEmpty;
      z.rep = 0ull;
      z.mmin = INT_MAX;
      z.count = 0u;
      z.pad = 0ull;
      t.meta[i] = z;
      SlotAcc za = {};
      t.acc[i] = za;
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
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], s); };
  mark(0);
  cudaError_t err = cudaMemsetAsync(t.cnt, 0, sizeof(FrameCounters) + sizeof(unsigned) * (size_t)t.n_words, s);
  if (err != cudaSuccess) return err;
  mark(1);
  k_count<DT><<<dim3(geo.count_blocks_x, geo.n_cams), kThreads, 0, s>>>(rig, rays, fp, t, geo.count_blocks_x);
  mark(2);
  k_assign<DT><<<dim3(geo.tiles_max, geo.n_cams), kThreads, 0, s>>>(rig, rays, fp, t, tr, (float)out.unit_m);
  mark(3);
  k_accum<DT><<<dim3(geo.tiles_max, geo.n_cams), kThreads, 0, s>>>(rig, rays, fp, t);
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
