// ff_api.cu - host side of the C ABI declared in include/fuseflow.h.
//
// Create time (host, double precision): relative poses T_ji = T_j T_i^-1 of Eq. 4, the
// static neighbour table of Sec. II.5(2)b, per-camera ray tables (x - cx)/fx and
// (y - cy)/fy, all split into float32 hi/lo pairs for the device; device tables are
// allocated once and reused by every frame.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ff_internal.h"

using namespace ffl;

struct fuseflow_ctx {
  int device = 0;
  int n_cams = 0;
  int k1 = 0;
  fuseflow_params params{};
  std::vector<fuseflow_intrinsics> intr;
  std::vector<fuseflow_extrinsics> extr;
  std::vector<int32_t> nbr;
  long long n_px = 0;
  long long max_cells = 0;
  unsigned max_slots = 0, ccap = 0;
  RigDev* d_rig = nullptr;
  float2* d_rays = nullptr;
  void* d_blocks = nullptr;            // tile list + per-camera block constants
  Tables tab{};
  void* d_tables = nullptr;            // one allocation for every table
  size_t table_bytes = 0;
  OutDev out{};
  void* d_out = nullptr;
  size_t out_bytes = 0;
  TraceDev trace{};
  Geometry geo{};
  long long max_chunks = 0;            // 2048-pixel chunks of the largest camera
  int bstats_cap = 0;                  // count-step block statistics allocated (chunks = 1)
  // staging for the host-buffer entry point
  void* d_stage = nullptr;
  size_t stage_bytes = 0;
  // per-block sums of the MC error (Eq. 12)
  void* d_mc = nullptr;
  // D^r of Eq. 8 when a depth screen is set (per camera, 256-byte aligned)
  void* d_screen = nullptr;
  size_t screen_bytes = 0;
  // stage timing ring
  bool timing = false;
  std::vector<cudaEvent_t> events;     // kTimingRing * (FUSEFLOW_N_STAGES + 1)
  long long timed_frames = 0;
};

// Contexts fused together by one launch of each frame kernel (launch_batch).
struct fuseflow_batch {
  std::vector<fuseflow_ctx*> ctx;
};

// One fuse call captured as a CUDA graph (the memset and kernels of launch_frame).
struct fuseflow_graph {
  fuseflow_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static constexpr int kTimingRing = 1024;
static constexpr int kEv = FUSEFLOW_N_STAGES + 1;

namespace {

void split(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

unsigned next_pow2(unsigned long long v) {
  unsigned long long p = 1;
  while (p < v) p <<= 1;
  return (unsigned)std::min<unsigned long long>(p, 1ull << 31);
}

// camera centre c = -R^T t and optical axis R^T e_z in world coordinates
void centre_axis(const fuseflow_extrinsics& e, double c[3], double a[3]) {
  for (int k = 0; k < 3; ++k) {
    c[k] = -(e.R[0 + k] * e.t[0] + e.R[3 + k] * e.t[1] + e.R[6 + k] * e.t[2]);
    a[k] = e.R[6 + k];
  }
}

// Sec. II.5(2)b read as a static list: the other cameras by optical-axis angle, then
// centre distance, then index (values closer than 1e-9 count as equal).
std::vector<int32_t> neighbour_table(const std::vector<fuseflow_extrinsics>& ex, int k1) {
  const int n = (int)ex.size();
  std::vector<int32_t> out((size_t)n * k1);
  struct Cand { double angle, dist; int j; };
  for (int i = 0; i < n; ++i) {
    double ci[3], ai[3];
    centre_axis(ex[i], ci, ai);
    const double ni = std::sqrt(ai[0] * ai[0] + ai[1] * ai[1] + ai[2] * ai[2]);
    std::vector<Cand> cand;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double cj[3], aj[3];
      centre_axis(ex[j], cj, aj);
      const double nj = std::sqrt(aj[0] * aj[0] + aj[1] * aj[1] + aj[2] * aj[2]);
      double cs = (ai[0] * aj[0] + ai[1] * aj[1] + ai[2] * aj[2]) / (ni * nj);
      cs = std::max(-1.0, std::min(1.0, cs));
      const double dx = ci[0] - cj[0], dy = ci[1] - cj[1], dz = ci[2] - cj[2];
      cand.push_back({std::acos(cs), std::sqrt(dx * dx + dy * dy + dz * dz), j});
    }
    // stable insertion order on a tolerance-based key
    for (size_t a = 1; a < cand.size(); ++a) {
      Cand v = cand[a];
      size_t b = a;
      auto before = [](const Cand& x, const Cand& y) {
        if (std::fabs(x.angle - y.angle) > 1e-9) return x.angle < y.angle;
        if (std::fabs(x.dist - y.dist) > 1e-9) return x.dist < y.dist;
        return x.j < y.j;
      };
      while (b > 0 && before(v, cand[b - 1])) { cand[b] = cand[b - 1]; --b; }
      cand[b] = v;
    }
    for (int q = 0; q < k1; ++q) out[(size_t)i * k1 + q] = cand[q].j;
  }
  return out;
}

bool finite(double v) { return std::isfinite(v); }

int validate(const fuseflow_intrinsics* intr, const fuseflow_extrinsics* extr, int32_t n,
             const fuseflow_params* p) {
  if (!intr || !extr || !p) return FUSEFLOW_ERR_INVALID_ARG;
  if (n < 1 || n > kMaxCams) return FUSEFLOW_ERR_INVALID_ARG;
  long long px = 0;
  for (int i = 0; i < n; ++i) {
    const fuseflow_intrinsics& k = intr[i];
    if (!(k.fx > 0) || !(k.fy > 0) || !finite(k.fx) || !finite(k.fy) || !finite(k.cx) ||
        !finite(k.cy) || k.width < 1 || k.height < 1)
      return FUSEFLOW_ERR_INVALID_ARG;
    if ((long long)k.width * k.height > (1ll << 30)) return FUSEFLOW_ERR_INVALID_ARG;
    px += (long long)k.width * k.height;
    for (int a = 0; a < 9; ++a) if (!finite(extr[i].R[a])) return FUSEFLOW_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) if (!finite(extr[i].t[a])) return FUSEFLOW_ERR_INVALID_ARG;
  }
  if (px >= (1ll << 32) - 1) return FUSEFLOW_ERR_INVALID_ARG;   // pixel index is 32-bit
  const int K = std::min<int>(p->k_views, n);
  if (p->k_views < 1 || K - 1 > kMaxK1) return FUSEFLOW_ERR_INVALID_ARG;
  if (!(p->tau >= 0.0f) || !std::isfinite(p->tau)) return FUSEFLOW_ERR_INVALID_ARG;
  if (!(p->sigma_m > 0) || !finite(p->sigma_m)) return FUSEFLOW_ERR_INVALID_ARG;
  if (!(p->coarse_cell_m > 0) || !finite(p->coarse_cell_m)) return FUSEFLOW_ERR_INVALID_ARG;
  if (p->max_level < 0 || p->max_level > 14 || p->n_min < 1) return FUSEFLOW_ERR_INVALID_ARG;
  if (p->depth_format != FUSEFLOW_DEPTH_U16 && p->depth_format != FUSEFLOW_DEPTH_F32)
    return FUSEFLOW_ERR_INVALID_ARG;
  if (!(p->depth_scale > 0) || !finite(p->depth_scale)) return FUSEFLOW_ERR_INVALID_ARG;
  if (p->max_cells < 0 || p->max_cells > (1ll << 30)) return FUSEFLOW_ERR_INVALID_ARG;
  if (p->top_k < 0 || p->top_k > kMaxTopK) return FUSEFLOW_ERR_INVALID_ARG;
  if (!finite(p->screen_min_m) || !finite(p->screen_max_m) || !std::isfinite(p->screen_edge_rel) ||
      p->reserved1 != 0)
    return FUSEFLOW_ERR_INVALID_ARG;
  if (p->screen_min_m > 0 && p->screen_max_m > 0 && p->screen_min_m > p->screen_max_m)
    return FUSEFLOW_ERR_INVALID_ARG;
  return FUSEFLOW_OK;
}

bool screen_set(const fuseflow_params* p) {
  return p->screen_min_m > 0 || p->screen_max_m > 0 || p->screen_edge_rel > 0.0f;
}

// Screen bounds in depth units and image sizes (the buffers are filled in by the caller).
ScreenArgs screen_args(const fuseflow_intrinsics* intr, int n_cams, const fuseflow_params* p) {
  ScreenArgs a{};
  a.n_cams = n_cams;
  for (int i = 0; i < n_cams; ++i) { a.W[i] = intr[i].width; a.H[i] = intr[i].height; }
  a.min_u = p->screen_min_m > 0 ? (float)(p->screen_min_m / p->depth_scale) : 0.0f;
  a.max_u = p->screen_max_m > 0 ? (float)(p->screen_max_m / p->depth_scale) : 0.0f;
  a.edge_rel = p->screen_edge_rel > 0.0f ? p->screen_edge_rel : 0.0f;
  return a;
}

// Rig constants shared by fuseflow_create and the static entry point: per-camera
// intrinsics and poses, the ray tables rx(x) = (x - cx)/fx and ry(y) = (y - cy)/fy as ff,
// the relative poses of Eq. 4 (T_ji = T_j T_i^-1) and the separable pair rays.
// `rays` holds sum(W + H) entries and `pray` 2 k1 sum(W + H) float4.
void build_rig(const fuseflow_intrinsics* intr, const fuseflow_extrinsics* extr, int n_cams,
               const fuseflow_params* params, const int32_t* nbr, int k1, RigDev& rig,
               float2* rays, float4* pray) {
  const double unit = params->depth_scale;
  std::memset(&rig, 0, sizeof(rig));
  rig.n_cams = n_cams;
  rig.k1 = k1;
  rig.tau = params->tau;
  rig.use_conf = params->use_conf ? 1 : 0;
  rig.use_cons = params->use_consistency ? 1 : 0;
  rig.max_level = params->max_level;
  rig.n_min = params->n_min;
  rig.inv_s0u = (float)(unit / params->coarse_cell_m);
  const double sig_u = params->sigma_m / unit;
  if (k1 > 0) split(1.0 / (sig_u * sig_u * k1), rig.einv_h, rig.einv_l);
  rig.depth_f32 = params->depth_format == FUSEFLOW_DEPTH_F32;
  rig.top_k = params->top_k;
  int nr = 0, np = 0;
  long long off = 0;
  for (int i = 0; i < n_cams; ++i) {
    const fuseflow_intrinsics& k = intr[i];
    const fuseflow_extrinsics& e = extr[i];
    CamDev& c = rig.cam[i];
    c.W = k.width;
    c.H = k.height;
    c.off = off;
    off += (long long)k.width * k.height;
    c.fx = (float)k.fx; c.fy = (float)k.fy; c.cx = (float)k.cx; c.cy = (float)k.cy;
    split(k.fx, c.fxh, c.fxl);
    split(k.fy, c.fyh, c.fyl);
    split(k.cx, c.cxh, c.cxl);
    split(k.cy, c.cyh, c.cyl);
    double cen[3], ax[3];
    centre_axis(e, cen, ax);
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) c.Rwc[3 * r + q] = (float)e.R[3 * q + r];
      c.cwc[r] = (float)(cen[r] / unit);
    }
    c.ray_x = nr;
    for (int x = 0; x < k.width; ++x, ++nr) split(((double)x - k.cx) / k.fx, rays[nr].x, rays[nr].y);
    c.ray_y = nr;
    for (int y = 0; y < k.height; ++y, ++nr) split(((double)y - k.cy) / k.fy, rays[nr].x, rays[nr].y);
    c.pair0 = i * k1;
    for (int q = 0; q < k1; ++q) {
      const int j = nbr[i * k1 + q];
      const fuseflow_extrinsics& ej = extr[j];
      PairDev& P = rig.pair[c.pair0 + q];
      P.j = j;
      double Rji[9], tji[3];
      for (int r = 0; r < 3; ++r)
        for (int s2 = 0; s2 < 3; ++s2) {
          double acc = 0;
          for (int m = 0; m < 3; ++m) acc += ej.R[3 * r + m] * e.R[3 * s2 + m];   // R_j R_i^T
          Rji[3 * r + s2] = acc;
        }
      for (int r = 0; r < 3; ++r)
        tji[r] = ej.t[r] - (Rji[3 * r] * e.t[0] + Rji[3 * r + 1] * e.t[1] + Rji[3 * r + 2] * e.t[2]);
      for (int a = 0; a < 9; ++a) split(Rji[a], P.Rh[a], P.Rl[a]);
      for (int a = 0; a < 3; ++a) split(tji[a] / unit, P.th[a], P.tl[a]);
      // separable pair rays A_k(x) = R[k][0] rx(x) + R[k][2], B_k(y) = R[k][1] ry(y)
      auto put = [&](double v0, double v1, double v2) {
        float4& u = pray[np++];
        float4& w = pray[np++];
        split(v0, u.x, u.y);
        split(v1, u.z, u.w);
        split(v2, w.x, w.y);
        w.z = 0.0f;
        w.w = 0.0f;
      };
      P.ga = np;
      for (int x = 0; x < k.width; ++x) {
        const double rx = ((double)x - k.cx) / k.fx;
        put(Rji[0] * rx + Rji[2], Rji[3] * rx + Rji[5], Rji[6] * rx + Rji[8]);
      }
      P.gb = np;
      for (int y = 0; y < k.height; ++y) {
        const double ry = ((double)y - k.cy) / k.fy;
        put(Rji[1] * ry, Rji[4] * ry, Rji[7] * ry);
      }
    }
  }
  rig.n_px = off;
}

}  // namespace

extern "C" {

void fuseflow_default_params(fuseflow_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->tau = 0.6f;             // Eq. 9
  p->k_views = 4;
  p->sigma_m = 0.03;
  p->coarse_cell_m = 0.32;
  p->max_level = 4;
  p->n_min = 32;
  p->depth_format = FUSEFLOW_DEPTH_U16;
  p->use_conf = 1;
  p->depth_scale = 0.001;
  p->use_consistency = 1;
  p->max_cells = 0;
}

const char* fuseflow_status_string(int s) {
  switch (s) {
    case FUSEFLOW_OK: return "ok";
    case FUSEFLOW_ERR_INVALID_ARG: return "invalid argument";
    case FUSEFLOW_ERR_OUT_OF_MEMORY: return "out of memory";
    case FUSEFLOW_ERR_CAPACITY: return "capacity exceeded (max_cells, cell slots or a table)";
    case FUSEFLOW_ERR_CUDA: return "CUDA runtime error";
    case FUSEFLOW_ERR_TIMEOUT: return "device wait timed out";
    case FUSEFLOW_ERR_INTERNAL: return "internal device check failed";
    case FUSEFLOW_ERR_CANCELLED: return "cancelled before it started (its rig was removed)";
    default: return "unknown status";
  }
}

void fuseflow_destroy(fuseflow_ctx* ctx) {
  if (!ctx) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaFree(ctx->d_rig);
  cudaFree(ctx->d_rays);
  cudaFree(ctx->d_mc);
  cudaFree(ctx->d_blocks);
  cudaFree(ctx->d_tables);
  cudaFree(ctx->d_out);
  cudaFree(ctx->d_stage);
  cudaFree(ctx->d_screen);
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  cudaSetDevice(prev);
  delete ctx;
}

int fuseflow_create(const fuseflow_intrinsics* intr, const fuseflow_extrinsics* extr,
                    int32_t n_cams, const fuseflow_params* params, fuseflow_ctx** out) {
  if (!out) return FUSEFLOW_ERR_INVALID_ARG;
  *out = nullptr;
  const int v = validate(intr, extr, n_cams, params);
  if (v != FUSEFLOW_OK) return v;
  fuseflow_ctx* ctx = new (std::nothrow) fuseflow_ctx();
  if (!ctx) return FUSEFLOW_ERR_OUT_OF_MEMORY;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) { delete ctx; return FUSEFLOW_ERR_CUDA; }
  ctx->n_cams = n_cams;
  ctx->params = *params;
  ctx->intr.assign(intr, intr + n_cams);
  ctx->extr.assign(extr, extr + n_cams);
  const int K = std::min<int>(params->k_views, n_cams);
  ctx->k1 = K - 1;
  ctx->nbr = neighbour_table(ctx->extr, ctx->k1);
  const double unit = params->depth_scale;

  // ---------------------------------------------------------------- rig constants
  RigDev* rig = new (std::nothrow) RigDev();
  if (!rig) { delete ctx; return FUSEFLOW_ERR_OUT_OF_MEMORY; }
  long long off = 0, n_rays = 0, max_px = 0;
  for (int i = 0; i < n_cams; ++i) {
    off += (long long)intr[i].width * intr[i].height;
    n_rays += intr[i].width + intr[i].height;
    max_px = std::max(max_px, (long long)intr[i].width * intr[i].height);
  }
  std::vector<float2> rays((size_t)n_rays);
  std::vector<float4> pray((size_t)std::max<long long>(1, 2 * ctx->k1 * n_rays));
  build_rig(intr, extr, n_cams, params, ctx->nbr.data(), ctx->k1, *rig, rays.data(), pray.data());
  ctx->n_px = off;
  ctx->max_cells = params->max_cells > 0 ? params->max_cells : std::max<long long>(65536, off / 8);
  // A coarse cell at level l >= 1 holds n_c >= n_min 4^l points, so its 8^l dense slots are
  // at most 2^Lmax n_c / n_min; level-0 coarse cells need one slot each.
  const long long slot_bound = off + (((long long)1 << params->max_level) * off) / params->n_min;
  ctx->max_slots = (unsigned)std::max<long long>(4096, std::min<long long>(slot_bound, 1ll << 26));
  ctx->ccap = next_pow2((unsigned long long)std::max<long long>(4096, 2 * ctx->max_cells));

  // ---------------------------------------------------------------- launch geometry
  ctx->geo.n_cams = n_cams;
  ctx->geo.top_k = params->top_k;
  ctx->geo.depth_f32 = rig->depth_f32;
  ctx->geo.max_px = max_px;
  ctx->geo.scr = screen_args(intr, n_cams, params);
  ctx->geo.screen = screen_set(params) ? 1 : 0;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  {
    // several 2048-pixel chunks per count block: one wave of 4 blocks per SM (the kernel's
    // residency), but at most 6 chunks, since a block's table of coarse cells (2048
    // entries) spills to the global table when one block covers too much of the scene
    long long total_chunks = 0;
    for (int i = 0; i < n_cams; ++i) total_chunks += ((long long)intr[i].width * intr[i].height + 2047) / 2048;
    const long long per = (total_chunks + 4ll * sms - 1) / (4ll * sms);
    ctx->geo.count_chunks = (int)std::max<long long>(1, std::min<long long>(6, per));
    ctx->max_chunks = (max_px + 2047) / 2048;
    ctx->geo.count_blocks_x = (int)((ctx->max_chunks + ctx->geo.count_chunks - 1) / ctx->geo.count_chunks);
  }
  ctx->geo.emit_blocks = std::max(1, sms * 8);
  ctx->geo.pdl = off < (1ll << 21) ? 2 : 1;

  // ---------------------------------------------------------------- device memory
  int status = FUSEFLOW_OK;
  const long long n_words = (off + 31) / 32;
  const int n_wblocks = (int)((n_words + 1023) / 1024);
  // block statistics for the finest count geometry a tuning may choose (one chunk a block)
  ctx->bstats_cap = (int)(ctx->max_chunks * n_cams);
  const int n_bstats = ctx->geo.count_blocks_x * n_cams;
  size_t o = 0;
  auto take = [&](size_t bytes, size_t align) { o = align_up(o, align); size_t at = o; o += bytes; return at; };
  // (tile, cell) partials: at most one per gated pixel
  const unsigned max_partials = (unsigned)std::min<long long>(off, 0xfffffffell);
  const size_t o_frec = take(sizeof(SlotRec) * ctx->max_slots, 256);
  const size_t o_fused = take(sizeof(unsigned) * ctx->max_slots, 256);
  const size_t o_coarse = take(sizeof(CoarseEntry) * ctx->ccap, 256);
  const size_t o_cused = take(sizeof(unsigned) * ctx->ccap, 256);
  const size_t o_cnt = take(sizeof(FrameCounters) + sizeof(unsigned) * (size_t)n_words, 256);
  const size_t o_bst = take(sizeof(BlockStats) * (size_t)ctx->bstats_cap, 256);
  const size_t o_part = take(sizeof(Partial) * (size_t)max_partials, 256);
  const size_t o_staged = take(sizeof(CellOut) * (size_t)ctx->max_cells, 256);
  const size_t o_wpre = take(sizeof(unsigned) * (size_t)n_words, 256);
  const size_t o_bsum = take(sizeof(unsigned) * (size_t)n_wblocks, 256);
  ctx->table_bytes = o;
  size_t po = 0;
  auto take_out = [&](size_t bytes) { po = align_up(po, 256); size_t at = po; po += bytes; return at; };
  const size_t q_stats = take_out(sizeof(fuseflow_stats));
  const size_t q_pos = take_out(sizeof(float) * 3 * (size_t)ctx->max_cells);
  const size_t q_rgb = take_out(sizeof(float) * 3 * (size_t)ctx->max_cells);
  const size_t q_w = take_out(sizeof(float) * (size_t)ctx->max_cells);
  const size_t q_cnt = take_out(sizeof(uint32_t) * (size_t)ctx->max_cells);
  const size_t q_rep = take_out(sizeof(uint32_t) * (size_t)ctx->max_cells);
  const size_t q_key = take_out(sizeof(unsigned long long) * (size_t)ctx->max_cells);
  ctx->out_bytes = po;

  const int n_tiles = fill_tile_index(*rig, &ctx->geo.tiles, 16);
  ctx->geo.tiles.ahead = assign_resident_blocks(16, rig->k1) * sms;
  std::vector<BlockConst> bconst((size_t)n_cams);
  fill_block_consts(*rig, bconst.data());
  const size_t pray_at = align_up(sizeof(BlockConst) * (size_t)n_cams, 256);
  const size_t blocks_bytes = pray_at + sizeof(float4) * pray.size();
  if (ctx->geo.screen) {
    const size_t dsz = rig->depth_f32 ? 4 : 2;
    std::vector<size_t> at((size_t)n_cams);
    for (int i = 0; i < n_cams; ++i) {
      at[i] = ctx->screen_bytes;
      ctx->screen_bytes += align_up((size_t)intr[i].width * intr[i].height * dsz, 256);
    }
    if (cudaMalloc(&ctx->d_screen, ctx->screen_bytes) != cudaSuccess) {
      ctx->d_screen = nullptr;
      status = FUSEFLOW_ERR_OUT_OF_MEMORY;
    } else {
      for (int i = 0; i < n_cams; ++i) ctx->geo.scr.out[i] = static_cast<char*>(ctx->d_screen) + at[i];
    }
  }
  if (status == FUSEFLOW_OK &&
      (cudaMalloc(&ctx->d_rig, sizeof(RigDev)) != cudaSuccess ||
       cudaMalloc(&ctx->d_rays, sizeof(float2) * rays.size()) != cudaSuccess ||
       cudaMalloc(&ctx->d_blocks, blocks_bytes) != cudaSuccess ||
       cudaMalloc(&ctx->d_tables, ctx->table_bytes) != cudaSuccess ||
       cudaMalloc(&ctx->d_out, ctx->out_bytes) != cudaSuccess))
    status = FUSEFLOW_ERR_OUT_OF_MEMORY;
  if (status == FUSEFLOW_OK) {
    char* b = static_cast<char*>(ctx->d_tables);
    Tables& t = ctx->tab;
    t.frec = reinterpret_cast<SlotRec*>(b + o_frec);
    t.fused = reinterpret_cast<unsigned*>(b + o_fused);
    t.max_slots = ctx->max_slots;
    t.coarse = reinterpret_cast<CoarseEntry*>(b + o_coarse);
    t.n_min = params->n_min;
    t.max_level = params->max_level;
    t.bconst = static_cast<const BlockConst*>(ctx->d_blocks);
    t.pray = reinterpret_cast<const float4*>(static_cast<char*>(ctx->d_blocks) + pray_at);
    t.n_tiles = n_tiles;
    t.cused = reinterpret_cast<unsigned*>(b + o_cused);
    t.cmask = ctx->ccap - 1;
    t.cnt = reinterpret_cast<FrameCounters*>(b + o_cnt);
    t.bitmap = reinterpret_cast<unsigned*>(t.cnt + 1);
    t.bstats = reinterpret_cast<BlockStats*>(b + o_bst);
    t.n_bstats = n_bstats;
    t.part = reinterpret_cast<Partial*>(b + o_part);
    t.max_partials = max_partials;
    t.staged = reinterpret_cast<CellOut*>(b + o_staged);
    t.wprefix = reinterpret_cast<unsigned*>(b + o_wpre);
    t.bsum = reinterpret_cast<unsigned*>(b + o_bsum);
    t.n_words = n_words;
    t.n_wblocks = n_wblocks;
    char* q = static_cast<char*>(ctx->d_out);
    OutDev& od = ctx->out;
    od.stats = reinterpret_cast<fuseflow_stats*>(q + q_stats);
    od.pos = reinterpret_cast<float*>(q + q_pos);
    od.rgb = reinterpret_cast<float*>(q + q_rgb);
    od.weight = reinterpret_cast<float*>(q + q_w);
    od.count = reinterpret_cast<uint32_t*>(q + q_cnt);
    od.rep = reinterpret_cast<uint32_t*>(q + q_rep);
    od.key = reinterpret_cast<unsigned long long*>(q + q_key);
    od.max_cells = ctx->max_cells;
    od.s0_m = params->coarse_cell_m;
    od.unit_m = unit;
  od.unit_f = (float)unit;
    if (cudaMemcpy(ctx->d_rig, rig, sizeof(RigDev), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_rays, rays.data(), sizeof(float2) * rays.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_blocks, bconst.data(), sizeof(BlockConst) * (size_t)n_cams,
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(static_cast<char*>(ctx->d_blocks) + pray_at, pray.data(), sizeof(float4) * pray.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(ctx->d_tables, 0, ctx->table_bytes) != cudaSuccess ||
        cudaMemset(ctx->d_out, 0, ctx->out_bytes) != cudaSuccess ||
        launch_init_tables(t, ctx->max_slots, ctx->ccap, 0) != cudaSuccess ||
        prepare_launch(rig->depth_f32 != 0) != cudaSuccess ||
        cudaStreamSynchronize(0) != cudaSuccess)     // this context's set-up only: work on
                                                     // non-blocking streams keeps running
      status = FUSEFLOW_ERR_CUDA;
  }
  delete rig;
  if (status != FUSEFLOW_OK) {
    cudaGetLastError();
    fuseflow_destroy(ctx);
    return status;
  }
  *out = ctx;
  return FUSEFLOW_OK;
}

static FramePtrs frame_ptrs(const fuseflow_ctx* ctx, const void* const* depth, const float* const* conf,
                            const uint8_t* const* rgb, int* ok) {
  FramePtrs fp{};
  *ok = depth && conf && rgb;
  for (int i = 0; *ok && i < ctx->n_cams; ++i) {
    if (!depth[i] || !conf[i] || !rgb[i]) { *ok = 0; break; }
    fp.depth[i] = depth[i];
    fp.conf[i] = conf[i];
    fp.rgb[i] = rgb[i];
  }
  return fp;
}

static void fill_cloud(const fuseflow_ctx* ctx, fuseflow_cloud* out) {
  out->stats = ctx->out.stats;
  out->pos = ctx->out.pos;
  out->rgb = ctx->out.rgb;
  out->weight = ctx->out.weight;
  out->count = ctx->out.count;
  out->rep = ctx->out.rep;
  out->key = reinterpret_cast<uint64_t*>(ctx->out.key);
  out->capacity = ctx->max_cells;
}

int fuseflow_fuse_frame(fuseflow_ctx* ctx, const void* const* depth, const float* const* conf,
                        const uint8_t* const* rgb, fuseflow_cloud* out, void* stream) {
  if (!ctx) return FUSEFLOW_ERR_INVALID_ARG;
  int ok = 0;
  const FramePtrs fp = frame_ptrs(ctx, depth, conf, rgb, &ok);
  if (!ok) return FUSEFLOW_ERR_INVALID_ARG;
  cudaEvent_t* ev = nullptr;
  if (ctx->timing) {
    ev = &ctx->events[(size_t)(ctx->timed_frames % kTimingRing) * kEv];
    ++ctx->timed_frames;
  }
  const cudaError_t e = launch_frame(ctx->d_rig, ctx->d_rays, fp, ctx->tab, ctx->trace, ctx->out,
                                     ctx->geo, static_cast<cudaStream_t>(stream), ev);
  if (e != cudaSuccess) return FUSEFLOW_ERR_CUDA;
  if (out) fill_cloud(ctx, out);
  return FUSEFLOW_OK;
}

int fuseflow_graph_create(fuseflow_ctx* ctx, const void* const* depth, const float* const* conf,
                          const uint8_t* const* rgb, fuseflow_graph** out) {
  if (!ctx || !out) return FUSEFLOW_ERR_INVALID_ARG;
  *out = nullptr;
  int ok = 0;
  const FramePtrs fp = frame_ptrs(ctx, depth, conf, rgb, &ok);
  if (!ok) return FUSEFLOW_ERR_INVALID_ARG;
  fuseflow_graph* g = new (std::nothrow) fuseflow_graph();
  if (!g) return FUSEFLOW_ERR_OUT_OF_MEMORY;
  g->ctx = ctx;
  cudaStream_t s = nullptr;
  int st = FUSEFLOW_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    s = nullptr;
    st = FUSEFLOW_ERR_CUDA;
  } else if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    st = FUSEFLOW_ERR_CUDA;
  } else {
    const cudaError_t e = launch_frame(ctx->d_rig, ctx->d_rays, fp, ctx->tab, ctx->trace, ctx->out,
                                       ctx->geo, s, nullptr);
    const cudaError_t e2 = cudaStreamEndCapture(s, &g->graph);
    if (e != cudaSuccess || e2 != cudaSuccess || !g->graph ||
        cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess)
      st = FUSEFLOW_ERR_CUDA;
  }
  if (s) cudaStreamDestroy(s);
  if (st != FUSEFLOW_OK) {
    cudaGetLastError();
    fuseflow_graph_destroy(g);
    return st;
  }
  *out = g;
  return FUSEFLOW_OK;
}

int fuseflow_get_cloud(const fuseflow_ctx* ctx, fuseflow_cloud* out) {
  if (!ctx || !out) return FUSEFLOW_ERR_INVALID_ARG;
  fill_cloud(ctx, out);
  return FUSEFLOW_OK;
}

int fuseflow_batch_create(fuseflow_ctx* const* ctxs, int32_t n, fuseflow_batch** out) {
  if (!out) return FUSEFLOW_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctxs || n < 1 || n > kMaxBatch) return FUSEFLOW_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || ctxs[i]->geo.screen || ctxs[i]->device != ctxs[0]->device ||
        ctxs[i]->geo.depth_f32 != ctxs[0]->geo.depth_f32 || ctxs[i]->geo.top_k != ctxs[0]->geo.top_k)
      return FUSEFLOW_ERR_INVALID_ARG;
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return FUSEFLOW_ERR_INVALID_ARG;   // one frame per context
  }
  fuseflow_batch* b = new (std::nothrow) fuseflow_batch();
  if (!b) return FUSEFLOW_ERR_OUT_OF_MEMORY;
  b->ctx.assign(ctxs, ctxs + n);
  *out = b;
  return FUSEFLOW_OK;
}

void fuseflow_batch_destroy(fuseflow_batch* b) { delete b; }

// The frames of a batch call: each context's images, tables and geometry (no trace).
static int batch_frames(const fuseflow_batch* b, const void* const* const* depth,
                        const float* const* const* conf, const uint8_t* const* const* rgb,
                        FrameLaunch* fl) {
  if (!b || !depth || !conf || !rgb) return FUSEFLOW_ERR_INVALID_ARG;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    const fuseflow_ctx* c = b->ctx[i];
    // one assign kernel serves the batch: its contexts share the tile height at call time
    if (c->geo.tiles.th != b->ctx[0]->geo.tiles.th) return FUSEFLOW_ERR_INVALID_ARG;
    int ok = 0;
    fl[i].fp = frame_ptrs(c, depth[i], conf[i], rgb[i], &ok);
    if (!ok) return FUSEFLOW_ERR_INVALID_ARG;
    fl[i].rig = c->d_rig;
    fl[i].rays = c->d_rays;
    fl[i].t = c->tab;
    fl[i].tr = TraceDev{};
    fl[i].out = c->out;
    fl[i].geo = &c->geo;
  }
  return FUSEFLOW_OK;
}

int fuseflow_batch_fuse(fuseflow_batch* b, const void* const* const* depth, const float* const* const* conf,
                        const uint8_t* const* const* rgb, void* stream) {
  FrameLaunch fl[kMaxBatch];
  const int st = batch_frames(b, depth, conf, rgb, fl);
  if (st != FUSEFLOW_OK) return st;
  return launch_batch(fl, (int)b->ctx.size(), static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FUSEFLOW_OK : FUSEFLOW_ERR_CUDA;
}

int fuseflow_batch_graph_create(fuseflow_batch* b, const void* const* const* depth,
                                const float* const* const* conf, const uint8_t* const* const* rgb,
                                fuseflow_graph** out) {
  if (!out) return FUSEFLOW_ERR_INVALID_ARG;
  *out = nullptr;
  FrameLaunch fl[kMaxBatch];
  int st = batch_frames(b, depth, conf, rgb, fl);
  if (st != FUSEFLOW_OK) return st;
  fuseflow_graph* g = new (std::nothrow) fuseflow_graph();
  if (!g) return FUSEFLOW_ERR_OUT_OF_MEMORY;
  g->ctx = b->ctx[0];
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    s = nullptr;
    st = FUSEFLOW_ERR_CUDA;
  } else if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    st = FUSEFLOW_ERR_CUDA;
  } else {
    const cudaError_t e = launch_batch(fl, (int)b->ctx.size(), s);
    const cudaError_t e2 = cudaStreamEndCapture(s, &g->graph);
    if (e != cudaSuccess || e2 != cudaSuccess || !g->graph ||
        cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess)
      st = FUSEFLOW_ERR_CUDA;
  }
  if (s) cudaStreamDestroy(s);
  if (st != FUSEFLOW_OK) {
    cudaGetLastError();
    fuseflow_graph_destroy(g);
    return st;
  }
  *out = g;
  return FUSEFLOW_OK;
}

int fuseflow_graph_launch(fuseflow_graph* g, fuseflow_cloud* out, void* stream) {
  if (!g || !g->exec) return FUSEFLOW_ERR_INVALID_ARG;
  if (cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return FUSEFLOW_ERR_CUDA;
  if (out) fill_cloud(g->ctx, out);
  return FUSEFLOW_OK;
}

void fuseflow_graph_destroy(fuseflow_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

int fuseflow_read_stats(fuseflow_ctx* ctx, fuseflow_stats* host_stats, void* stream) {
  if (!ctx || !host_stats) return FUSEFLOW_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(host_stats, ctx->out.stats, sizeof(fuseflow_stats), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FUSEFLOW_ERR_CUDA;
  return ffl::status_of_error((unsigned)host_stats->error);
}

int fuseflow_fuse_frame_host(fuseflow_ctx* ctx, const void* const* depth, const float* const* conf,
                             const uint8_t* const* rgb, float* pos, float* rgb_out, float* weight,
                             uint32_t* count, uint32_t* rep, uint64_t* key, fuseflow_stats* host_stats,
                             void* stream) {
  if (!ctx || !depth || !conf || !rgb || !host_stats) return FUSEFLOW_ERR_INVALID_ARG;
  const size_t dsz = ctx->params.depth_format == FUSEFLOW_DEPTH_F32 ? 4 : 2;
  if (!ctx->d_stage) {
    ctx->stage_bytes = 0;
    for (int i = 0; i < ctx->n_cams; ++i) {
      const size_t px = (size_t)ctx->intr[i].width * ctx->intr[i].height;
      ctx->stage_bytes += align_up(px * dsz, 256) + align_up(px * 4, 256) + align_up(px * 3, 256);
    }
    if (cudaMalloc(&ctx->d_stage, ctx->stage_bytes) != cudaSuccess) {
      ctx->d_stage = nullptr;
      return FUSEFLOW_ERR_OUT_OF_MEMORY;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<const void*> dp(ctx->n_cams);
  std::vector<const float*> cp(ctx->n_cams);
  std::vector<const uint8_t*> rp(ctx->n_cams);
  char* b = static_cast<char*>(ctx->d_stage);
  size_t o = 0;
  for (int i = 0; i < ctx->n_cams; ++i) {
    if (!depth[i] || !conf[i] || !rgb[i]) return FUSEFLOW_ERR_INVALID_ARG;
    const size_t px = (size_t)ctx->intr[i].width * ctx->intr[i].height;
    char* d = b + o; o += align_up(px * dsz, 256);
    char* c = b + o; o += align_up(px * 4, 256);
    char* r = b + o; o += align_up(px * 3, 256);
    if (cudaMemcpyAsync(d, depth[i], px * dsz, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c, conf[i], px * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(r, rgb[i], px * 3, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return FUSEFLOW_ERR_CUDA;
    dp[i] = d;
    cp[i] = reinterpret_cast<const float*>(c);
    rp[i] = reinterpret_cast<const uint8_t*>(r);
  }
  fuseflow_cloud cl;
  int st = fuseflow_fuse_frame(ctx, dp.data(), cp.data(), rp.data(), &cl, stream);
  if (st != FUSEFLOW_OK) return st;
  st = fuseflow_read_stats(ctx, host_stats, stream);
  const size_t n = (size_t)std::max<int64_t>(0, host_stats->n_cells);
  if (n) {
    struct { void* dst; const void* src; size_t sz; } cp_list[6] = {
        {pos, cl.pos, 12}, {rgb_out, cl.rgb, 12}, {weight, cl.weight, 4},
        {count, cl.count, 4}, {rep, cl.rep, 4}, {key, cl.key, 8}};
    for (auto& c : cp_list)
      if (c.dst && cudaMemcpyAsync(c.dst, c.src, c.sz * n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FUSEFLOW_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FUSEFLOW_ERR_CUDA;
  }
  return st;
}

int fuseflow_screen_depth(fuseflow_ctx* ctx, const void* const* depth_in, void* const* depth_out,
                          void* stream) {
  if (!ctx || !depth_in || !depth_out) return FUSEFLOW_ERR_INVALID_ARG;
  ScreenArgs a = ctx->geo.scr;
  for (int i = 0; i < ctx->n_cams; ++i) {
    if (!depth_in[i] || !depth_out[i] || depth_in[i] == depth_out[i]) return FUSEFLOW_ERR_INVALID_ARG;
    a.in[i] = depth_in[i];
    a.out[i] = depth_out[i];
  }
  return launch_screen(a, ctx->geo.depth_f32 != 0, ctx->geo.max_px, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? FUSEFLOW_OK
             : FUSEFLOW_ERR_CUDA;
}

void fuseflow_default_conf_params(fuseflow_conf_params* cp) {
  if (!cp) return;
  cp->alpha = 0.5;
  cp->beta = 0.5;
  cp->gamma = 1.0;
  cp->delta = 1.0;
}

int fuseflow_confidence(fuseflow_ctx* ctx, const void* const* depth, float* const* conf_out,
                        const fuseflow_conf_params* cp, void* stream) {
  if (!ctx || !depth || !conf_out) return FUSEFLOW_ERR_INVALID_ARG;
  fuseflow_conf_params p;
  fuseflow_default_conf_params(&p);
  if (cp) p = *cp;
  if (!(p.alpha >= 0.0) || !(p.beta >= 0.0) || !(p.gamma >= 0.0) || !(p.delta >= 0.0) ||
      !(p.alpha + p.gamma > 0.0))
    return FUSEFLOW_ERR_INVALID_ARG;
  ConfArgs a{};
  a.n_cams = ctx->n_cams;
  a.scale = (float)ctx->params.depth_scale;
  a.alpha = (float)p.alpha;
  a.beta = (float)p.beta;
  a.gamma = (float)p.gamma;
  a.delta = (float)p.delta;
  a.inv_ag = (float)(1.0 / (p.alpha + p.gamma));
  int max_w = 0, max_h = 0;
  for (int i = 0; i < ctx->n_cams; ++i) {
    if (!depth[i] || !conf_out[i]) return FUSEFLOW_ERR_INVALID_ARG;
    a.depth[i] = depth[i];
    a.out[i] = conf_out[i];
    a.W[i] = ctx->intr[i].width;
    a.H[i] = ctx->intr[i].height;
    max_w = std::max(max_w, a.W[i]);
    max_h = std::max(max_h, a.H[i]);
  }
  return launch_confidence(a, ctx->params.depth_format == FUSEFLOW_DEPTH_F32, max_w, max_h,
                           static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FUSEFLOW_OK : FUSEFLOW_ERR_CUDA;
}

// Small per-context device buffers, allocated on first use: the per-block sums of the MC
// error (kMcBytes) followed by the two counters of the point-wise path.
constexpr size_t kMcBytes = 1024 * (sizeof(double) + sizeof(long long));
static bool small_buffers(fuseflow_ctx* ctx) {
  if (ctx->d_mc) return true;
  if (cudaMalloc(&ctx->d_mc, kMcBytes + 2 * sizeof(unsigned long long)) != cudaSuccess) {
    ctx->d_mc = nullptr;
    cudaGetLastError();
    return false;
  }
  return true;
}

int fuseflow_mc_error(fuseflow_ctx* ctx, const float* pos, int64_t n_points,
                      const void* const* depth, double occlusion_m, float* err_m,
                      int32_t* n_visible, double* mc_m, int64_t* n_used, void* stream) {
  if (!ctx || n_points < 0 || (n_points > 0 && !pos) || !depth || !mc_m || !n_used ||
      !(occlusion_m >= 0.0))
    return FUSEFLOW_ERR_INVALID_ARG;
  for (int i = 0; i < ctx->n_cams; ++i)
    if (!depth[i]) return FUSEFLOW_ERR_INVALID_ARG;
  const int blocks = ffl::mc_blocks(n_points);
  if (!small_buffers(ctx)) return FUSEFLOW_ERR_OUT_OF_MEMORY;
  double* bsum = static_cast<double*>(ctx->d_mc);
  long long* bcnt = reinterpret_cast<long long*>(bsum + 1024);
  FramePtrs fp{};
  for (int i = 0; i < ctx->n_cams; ++i) fp.depth[i] = depth[i];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<double> hs(blocks);
  std::vector<long long> hc(blocks);
  if (launch_mc(ctx->d_rig, fp, ctx->params.depth_format == FUSEFLOW_DEPTH_F32, pos, n_points,
                ctx->params.depth_scale, occlusion_m, err_m, n_visible, bsum, bcnt, s) != cudaSuccess ||
      cudaMemcpyAsync(hs.data(), bsum, sizeof(double) * blocks, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hc.data(), bcnt, sizeof(long long) * blocks, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FUSEFLOW_ERR_CUDA;
  double sum = 0.0;
  long long cnt = 0;
  for (int b = 0; b < blocks; ++b) { sum += hs[b]; cnt += hc[b]; }
  *n_used = cnt;
  *mc_m = cnt ? sum / (double)cnt * ctx->params.depth_scale : std::nan("");
  return FUSEFLOW_OK;
}

int fuseflow_fuse_points(fuseflow_ctx* ctx, const void* const* depth, const float* const* conf,
                         const uint8_t* const* rgb, float* pos, float* weight, uint8_t* rgb_out,
                         int64_t* n_valid, int64_t* n_gated, void* stream) {
  if (!ctx || !pos || !weight || !rgb_out) return FUSEFLOW_ERR_INVALID_ARG;
  if (ctx->geo.screen) return FUSEFLOW_ERR_INVALID_ARG;          // D^r is not applied here
  int ok = 0;
  const FramePtrs fp = frame_ptrs(ctx, depth, conf, rgb, &ok);
  if (!ok) return FUSEFLOW_ERR_INVALID_ARG;
  if (!small_buffers(ctx)) return FUSEFLOW_ERR_OUT_OF_MEMORY;
  PointsDev pd{pos, weight, rgb_out,
               reinterpret_cast<unsigned long long*>(static_cast<char*>(ctx->d_mc) + kMcBytes),
               (float)ctx->params.depth_scale};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (launch_points(ctx->d_rig, ctx->d_rays, fp, ctx->tab, pd, ctx->geo.depth_f32 != 0, ctx->n_cams,
                    ctx->geo.max_px, s) != cudaSuccess)
    return FUSEFLOW_ERR_CUDA;
  if (n_valid || n_gated) {
    unsigned long long h[2] = {0ull, 0ull};
    if (cudaMemcpyAsync(h, pd.counts, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return FUSEFLOW_ERR_CUDA;
    if (n_valid) *n_valid = (int64_t)h[0];
    if (n_gated) *n_gated = (int64_t)h[1];
  }
  return FUSEFLOW_OK;
}

int fuseflow_set_trace(fuseflow_ctx* ctx, const fuseflow_trace* trace) {
  if (!ctx) return FUSEFLOW_ERR_INVALID_ARG;
  ctx->trace = TraceDev{};
  if (trace) {
    ctx->trace.pw = trace->pw;
    ctx->trace.omega = trace->omega;
    ctx->trace.e = trace->e;
    ctx->trace.nview = trace->nview;
    ctx->trace.key = reinterpret_cast<unsigned long long*>(trace->key);
  }
  return FUSEFLOW_OK;
}

int fuseflow_get_neighbours(const fuseflow_ctx* ctx, int32_t* out, int32_t* k_minus_1) {
  if (!ctx || !k_minus_1) return FUSEFLOW_ERR_INVALID_ARG;
  *k_minus_1 = ctx->k1;
  if (out && !ctx->nbr.empty()) std::memcpy(out, ctx->nbr.data(), sizeof(int32_t) * ctx->nbr.size());
  return FUSEFLOW_OK;
}

int fuseflow_enable_stage_timing(fuseflow_ctx* ctx, int enable) {
  if (!ctx) return FUSEFLOW_ERR_INVALID_ARG;
  if (enable && ctx->events.empty()) {
    ctx->events.resize((size_t)kTimingRing * kEv);
    for (auto& e : ctx->events)
      if (cudaEventCreate(&e) != cudaSuccess) return FUSEFLOW_ERR_CUDA;
  }
  ctx->timing = enable != 0;
  ctx->timed_frames = 0;
  return FUSEFLOW_OK;
}

int fuseflow_read_stage_times(fuseflow_ctx* ctx, double* ms, int64_t* n_frames) {
  if (!ctx || !ms || !n_frames) return FUSEFLOW_ERR_INVALID_ARG;
  for (int k = 0; k < FUSEFLOW_N_STAGES; ++k) ms[k] = 0.0;
  const long long n = std::min<long long>(ctx->timed_frames, kTimingRing);
  *n_frames = n;
  if (n == 0) return FUSEFLOW_OK;
  const long long last = (ctx->timed_frames - 1) % kTimingRing;
  if (cudaEventSynchronize(ctx->events[(size_t)last * kEv + kEv - 1]) != cudaSuccess)
    return FUSEFLOW_ERR_CUDA;
  for (long long f = 0; f < n; ++f) {
    const cudaEvent_t* ev = &ctx->events[(size_t)f * kEv];
    for (int k = 0; k < FUSEFLOW_N_STAGES; ++k) {
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, ev[k], ev[k + 1]) != cudaSuccess) return FUSEFLOW_ERR_CUDA;
      ms[k] += t;
    }
  }
  ctx->timed_frames = 0;
  return FUSEFLOW_OK;
}

// Launch geometry from a (validated) tuning: the count step's grid follows its chunks per
// block, and the scan step reads exactly the block statistics that grid writes.
static void apply_tuning(fuseflow_ctx* ctx, const fuseflow_tuning& tu) {
  ctx->geo.count_chunks = tu.count_chunks;
  ctx->geo.count_blocks_x = (int)((ctx->max_chunks + tu.count_chunks - 1) / tu.count_chunks);
  ctx->tab.n_bstats = ctx->geo.count_blocks_x * ctx->n_cams;
  ctx->geo.emit_blocks = tu.emit_blocks;
  ctx->geo.tiles.ahead = tu.prefetch_tiles == 0 ? kNoPrefetch : std::min(tu.prefetch_tiles, kNoPrefetch);
  ctx->geo.pdl = tu.programmatic;
  if (tu.tile_h != 0 && tu.tile_h != ctx->geo.tiles.th) ctx->tab.n_tiles = retile(&ctx->geo.tiles, tu.tile_h);
}

// Coordinate descent over the launch geometry, timing whole frames on one stream.
struct Autotuner {
  fuseflow_ctx* ctx;
  FramePtrs fp;
  int reps;
  cudaStream_t s;
  void* flush = nullptr;
  size_t flush_bytes = 0;
  std::vector<cudaEvent_t> ev;
  double start_us = 0.0, best_us = 0.0;

  Autotuner(fuseflow_ctx* c, const FramePtrs& f, int r, cudaStream_t st) : ctx(c), fp(f), reps(r), s(st) {}
  ~Autotuner() {
    if (flush) cudaFree(flush);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }

  // Median frame time (us) of the context's current geometry.
  int measure(double* us) {
    std::vector<float> t((size_t)reps);
    for (int r = -1; r < reps; ++r) {                 // one untimed frame first
      if (cudaMemsetAsync(flush, r & 0xff, flush_bytes, s) != cudaSuccess ||
          cudaEventRecord(ev[2 * std::max(r, 0)], s) != cudaSuccess ||
          launch_frame(ctx->d_rig, ctx->d_rays, fp, ctx->tab, TraceDev{}, ctx->out, ctx->geo, s, nullptr) !=
              cudaSuccess ||
          cudaEventRecord(ev[2 * std::max(r, 0) + 1], s) != cudaSuccess)
        return FUSEFLOW_ERR_CUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return FUSEFLOW_ERR_CUDA;
    for (int r = 0; r < reps; ++r)
      if (cudaEventElapsedTime(&t[(size_t)r], ev[2 * r], ev[2 * r + 1]) != cudaSuccess) return FUSEFLOW_ERR_CUDA;
    std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
    *us = 1e3 * t[(size_t)(reps / 2)];
    return FUSEFLOW_OK;
  }

  int time_setting(const fuseflow_tuning& tu, double* us) {
    apply_tuning(ctx, tu);
    return measure(us);
  }

  int run() {
    int dev = 0, l2 = 0, sms = 0;
    // the tile height goes first: it moves the assign step most, and the prefetch distance
    // below counts its tiles
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return FUSEFLOW_ERR_CUDA;
    flush_bytes = 2 * (size_t)std::max(l2, 1 << 20);
    if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
      flush = nullptr;
      cudaGetLastError();
      return FUSEFLOW_ERR_OUT_OF_MEMORY;
    }
    ev.resize(2 * (size_t)reps);
    for (cudaEvent_t& e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) { e = nullptr; return FUSEFLOW_ERR_CUDA; }

    fuseflow_tuning start{};
    fuseflow_get_tuning(ctx, &start);
    fuseflow_tuning best = start;
    int st = time_setting(best, &best_us);
    if (st != FUSEFLOW_OK) return st;
    auto consider = [&](fuseflow_tuning cand) -> int {
      if (std::memcmp(&cand, &best, sizeof cand) == 0) return FUSEFLOW_OK;
      double us = 0.0;
      const int r = time_setting(cand, &us);
      if (r == FUSEFLOW_OK && us < 0.99 * best_us) { best = cand; best_us = us; }
      return r;
    };
    for (int h : {8, 16, 32}) {
      fuseflow_tuning c = best;
      c.tile_h = h;
      if (h != best.tile_h) {          // the prefetch distance scaled to the same wave of pixels
        const long long a = best.prefetch_tiles;
        c.prefetch_tiles = (int)std::min<long long>(kNoPrefetch - 1, a * best.tile_h / h);
      }
      if ((st = consider(c)) != FUSEFLOW_OK) return st;
    }
    // count_chunks: one wave of b count blocks per SM, for b in 1..8
    long long total_chunks = 0;
    for (int i = 0; i < ctx->n_cams; ++i)
      total_chunks += ((long long)ctx->intr[i].width * ctx->intr[i].height + 2047) / 2048;
    std::vector<int> chunks = {2, 4, 6, 8, 16};
    for (int b : {1, 2, 3, 4, 6, 8}) {
      const long long per = (total_chunks + (long long)b * sms - 1) / ((long long)b * sms);
      chunks.push_back((int)std::max<long long>(1, std::min<long long>(64, per)));
    }
    for (int k : chunks) {
      fuseflow_tuning c = best;
      c.count_chunks = k;
      if ((st = consider(c)) != FUSEFLOW_OK) return st;
    }
    for (int b : {1, 2, 4, 8, 16}) {
      fuseflow_tuning c = best;
      c.emit_blocks = b * sms;
      if ((st = consider(c)) != FUSEFLOW_OK) return st;
    }
    const int wave = assign_resident_blocks(best.tile_h, ctx->k1) * sms;
    for (int a : {0, wave / 2, wave, 2 * wave}) {
      fuseflow_tuning c = best;
      c.prefetch_tiles = a;
      if ((st = consider(c)) != FUSEFLOW_OK) return st;
    }
    for (int pg : {0, 1, 2}) {
      fuseflow_tuning c = best;
      c.programmatic = pg;
      if ((st = consider(c)) != FUSEFLOW_OK) return st;
    }
    // both settings timed again back to back, so that clocks drift into neither
    if ((st = time_setting(start, &start_us)) != FUSEFLOW_OK) return st;
    if ((st = time_setting(best, &best_us)) != FUSEFLOW_OK) return st;
    if (start_us <= best_us) {             // no gain after all: keep the caller's setting
      apply_tuning(ctx, start);
      best_us = start_us;
    }
    return FUSEFLOW_OK;
  }
};

int fuseflow_get_tuning(const fuseflow_ctx* ctx, fuseflow_tuning* out) {
  if (!ctx || !out) return FUSEFLOW_ERR_INVALID_ARG;
  out->count_chunks = ctx->geo.count_chunks;
  out->emit_blocks = ctx->geo.emit_blocks;
  out->prefetch_tiles = ctx->geo.tiles.ahead >= kNoPrefetch ? 0 : ctx->geo.tiles.ahead;
  out->programmatic = ctx->geo.pdl;
  out->tile_h = ctx->geo.tiles.th;
  return FUSEFLOW_OK;
}

int fuseflow_set_tuning(fuseflow_ctx* ctx, const fuseflow_tuning* in) {
  if (!ctx || !in || in->count_chunks < 1 || in->count_chunks > 64 || in->emit_blocks < 1 ||
      in->emit_blocks > 65536 || in->prefetch_tiles < 0 || in->programmatic < 0 || in->programmatic > 2 ||
      (in->tile_h != 0 && in->tile_h != 8 && in->tile_h != 16 && in->tile_h != 32))
    return FUSEFLOW_ERR_INVALID_ARG;
  apply_tuning(ctx, *in);
  return FUSEFLOW_OK;
}

int fuseflow_autotune(fuseflow_ctx* ctx, const void* const* depth, const float* const* conf,
                      const uint8_t* const* rgb, int32_t reps, fuseflow_tuning* chosen,
                      double* frame_us, void* stream) {
  if (!ctx || reps < 3 || reps > 101) return FUSEFLOW_ERR_INVALID_ARG;
  int ok = 0;
  const FramePtrs fp = frame_ptrs(ctx, depth, conf, rgb, &ok);
  if (!ok) return FUSEFLOW_ERR_INVALID_ARG;
  Autotuner at(ctx, fp, reps, static_cast<cudaStream_t>(stream));
  const int st = at.run();
  if (st != FUSEFLOW_OK) return st;
  if (chosen) fuseflow_get_tuning(ctx, chosen);
  if (frame_us) { frame_us[0] = at.start_us; frame_us[1] = at.best_us; }
  return FUSEFLOW_OK;
}

const char* fuseflow_stage_name(int stage) {
  static const char* names[FUSEFLOW_N_STAGES] = {"clear", "count", "assign", "reduce", "scan",
                                                 "emit"};
  return (stage >= 0 && stage < FUSEFLOW_N_STAGES) ? names[stage] : "unknown";
}

int64_t fuseflow_num_pixels(const fuseflow_ctx* ctx) { return ctx ? ctx->n_px : 0; }
int64_t fuseflow_capacity(const fuseflow_ctx* ctx) { return ctx ? ctx->max_cells : 0; }
int64_t fuseflow_device_bytes(const fuseflow_ctx* ctx) {
  return ctx ? (int64_t)(ctx->table_bytes + ctx->out_bytes + ctx->stage_bytes + ctx->screen_bytes +
                         sizeof(RigDev))
             : 0;
}

}  // extern "C"

// ----------------------------------------------------------------------------------------
// Allocation-free variant of fuseflow_fuse_frame.
//
// All scratch (rig constants, ray tables, hash tables, per-pixel records, scan buffers)
// lives in one file-scope device array of kStaticBytes (about 23 MiB), held by every GPU
// that loads this library until the process exits.  Host code never dereferences the
// array's name: the device address comes from cudaGetSymbolAddress, taken once per device
// on that device's first call (which also clears the hash tables and synchronizes the
// stream).  Later calls reuse the array; the frame's own clear and emit steps leave the
// tables empty again, so calls in a row need no set-up.  Calls whose GPU work overlaps
// (several streams, or several host threads) race on the array.
namespace {

constexpr long long kStaticMaxPixels = 1ll << 19;      // 524,288 pixels per frame
constexpr unsigned kStaticMaxPartials = 1u << 17;      // (tile, cell) partial records
constexpr long long kStaticMaxCells = 1ll << 15;       // 32,768 output cells
constexpr unsigned kStaticSlots = 1u << 18;            // dense cell slots
constexpr unsigned kStaticCoarse = 1u << 16;           // coarse hash slots
constexpr int kStaticMaxRays = 1 << 16;                // sum over cameras of W + H
constexpr int kStaticMaxPairRays = 6 * kStaticMaxRays;  // float4: 2 (K - 1) sum(W + H)
constexpr long long kStaticWords = kStaticMaxPixels / 32;
constexpr int kStaticWBlocks = (int)((kStaticWords + 1023) / 1024);
constexpr int kStaticBStats = kMaxCams * (int)(kStaticMaxPixels / 2048 + 1);   // chunks = 1
constexpr int kStaticMaxDevices = 64;

constexpr size_t al256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kSRig = 0;
constexpr size_t kSRays = al256(kSRig + sizeof(RigDev));
constexpr size_t kSBConst = al256(kSRays + sizeof(float2) * kStaticMaxRays);
constexpr size_t kSPRay = al256(kSBConst + sizeof(BlockConst) * kMaxCams);
constexpr size_t kSFRec = al256(kSPRay + sizeof(float4) * kStaticMaxPairRays);
constexpr size_t kSFused = al256(kSFRec + sizeof(SlotRec) * kStaticSlots);
constexpr size_t kSCoarse = al256(kSFused + sizeof(unsigned) * kStaticSlots);
constexpr size_t kSCUsed = al256(kSCoarse + sizeof(CoarseEntry) * kStaticCoarse);
constexpr size_t kSCnt = al256(kSCUsed + sizeof(unsigned) * kStaticCoarse);
constexpr size_t kSBStats = al256(kSCnt + sizeof(FrameCounters) + sizeof(unsigned) * kStaticWords);
constexpr size_t kSPart = al256(kSBStats + sizeof(BlockStats) * kStaticBStats);
constexpr size_t kSStaged = al256(kSPart + sizeof(Partial) * kStaticMaxPartials);
constexpr size_t kSWPre = al256(kSStaged + sizeof(CellOut) * kStaticMaxCells);
constexpr size_t kSBSum = al256(kSWPre + sizeof(unsigned) * kStaticWords);
constexpr size_t kStaticBytes = al256(kSBSum + sizeof(unsigned) * kStaticWBlocks);
static_assert(kStaticBytes <= (32u << 20), "static scratch must stay modest");

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_static_mutex;                             // guards the host staging below
unsigned char* g_static_dev[kStaticMaxDevices] = {};   // device address per device
RigDev g_static_rig;                                   // host staging of the rig constants
float2 g_static_rays[kStaticMaxRays];                  // host staging of the ray tables
float4 g_static_pray[kStaticMaxPairRays];              // host staging of the pair rays
BlockConst g_static_bconst[kMaxCams];                  // host staging of the block constants

// The neighbour rule of neighbour_table() above (Sec. II.5(2)b: optical-axis angle, then
// centre distance, then index, 1e-9 tolerance) on fixed-size arrays: no heap use.
void neighbour_table_fixed(const fuseflow_extrinsics* ex, int n, int k1, int32_t* out) {
  struct Cand { double angle, dist; int j; };
  Cand cand[kMaxCams];
  for (int i = 0; i < n; ++i) {
    double ci[3], ai[3];
    centre_axis(ex[i], ci, ai);
    const double ni = std::sqrt(ai[0] * ai[0] + ai[1] * ai[1] + ai[2] * ai[2]);
    int m = 0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double cj[3], aj[3];
      centre_axis(ex[j], cj, aj);
      const double nj = std::sqrt(aj[0] * aj[0] + aj[1] * aj[1] + aj[2] * aj[2]);
      double cs = (ai[0] * aj[0] + ai[1] * aj[1] + ai[2] * aj[2]) / (ni * nj);
      cs = std::max(-1.0, std::min(1.0, cs));
      const double dx = ci[0] - cj[0], dy = ci[1] - cj[1], dz = ci[2] - cj[2];
      cand[m++] = {std::acos(cs), std::sqrt(dx * dx + dy * dy + dz * dz), j};
    }
    for (int a = 1; a < m; ++a) {
      const Cand v = cand[a];
      int b = a;
      auto before = [](const Cand& x, const Cand& y) {
        if (std::fabs(x.angle - y.angle) > 1e-9) return x.angle < y.angle;
        if (std::fabs(x.dist - y.dist) > 1e-9) return x.dist < y.dist;
        return x.j < y.j;
      };
      while (b > 0 && before(v, cand[b - 1])) { cand[b] = cand[b - 1]; --b; }
      cand[b] = v;
    }
    for (int q = 0; q < k1; ++q) out[i * k1 + q] = cand[q].j;
  }
}

Tables static_tables(unsigned char* base, long long n_px, int n_bstats) {
  Tables t{};
  t.frec = reinterpret_cast<SlotRec*>(base + kSFRec);
  t.fused = reinterpret_cast<unsigned*>(base + kSFused);
  t.max_slots = kStaticSlots;
  t.coarse = reinterpret_cast<CoarseEntry*>(base + kSCoarse);
  t.cused = reinterpret_cast<unsigned*>(base + kSCUsed);
  t.cmask = kStaticCoarse - 1;
  t.cnt = reinterpret_cast<FrameCounters*>(base + kSCnt);
  t.bitmap = reinterpret_cast<unsigned*>(t.cnt + 1);
  t.bstats = reinterpret_cast<BlockStats*>(base + kSBStats);
  t.n_bstats = n_bstats;
  t.part = reinterpret_cast<Partial*>(base + kSPart);
  t.max_partials = kStaticMaxPartials;
  t.staged = reinterpret_cast<CellOut*>(base + kSStaged);
  t.wprefix = reinterpret_cast<unsigned*>(base + kSWPre);
  t.bsum = reinterpret_cast<unsigned*>(base + kSBSum);
  t.n_words = (n_px + 31) / 32;
  t.n_wblocks = (int)((t.n_words + 1023) / 1024);
  return t;
}

// Device address of the scratch array on the current device; the first call on a device
// looks it up and empties its hash tables.
int static_scratch(int dev, cudaStream_t s, unsigned char** out) {
  if (dev < 0 || dev >= kStaticMaxDevices) return FUSEFLOW_ERR_INVALID_ARG;
  if (!g_static_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return FUSEFLOW_ERR_CUDA;
    unsigned char* base = static_cast<unsigned char*>(p);
    const Tables t = static_tables(base, kStaticMaxPixels, kStaticBStats);
    if (launch_init_tables(t, kStaticSlots, kStaticCoarse, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return FUSEFLOW_ERR_CUDA;
    g_static_dev[dev] = base;
  }
  *out = g_static_dev[dev];
  return FUSEFLOW_OK;
}

}  // namespace

extern "C" int fuseflow_fuse_frame_static(const fuseflow_intrinsics* intr,
                                          const fuseflow_extrinsics* extr, int32_t n_cams,
                                          const fuseflow_params* params, const void* const* depth,
                                          const float* const* conf, const uint8_t* const* rgb,
                                          float* pos, float* rgb_out, float* weight,
                                          uint32_t* count, uint32_t* rep, uint64_t* key,
                                          fuseflow_stats* stats, void* stream) {
  const int v = validate(intr, extr, n_cams, params);
  if (v != FUSEFLOW_OK) return v;
  if (!depth || !conf || !rgb || !pos || !rgb_out || !weight || !count || !rep || !key || !stats)
    return FUSEFLOW_ERR_INVALID_ARG;
  if (screen_set(params)) return FUSEFLOW_ERR_INVALID_ARG;     // no D^r buffer in the arena
  long long n_px = 0, max_px = 0, n_rays = 0;
  for (int i = 0; i < n_cams; ++i) {
    const long long px = (long long)intr[i].width * intr[i].height;
    n_px += px;
    max_px = std::max(max_px, px);
    n_rays += intr[i].width + intr[i].height;
    if (!depth[i] || !conf[i] || !rgb[i]) return FUSEFLOW_ERR_INVALID_ARG;
  }
  const long long max_cells = params->max_cells > 0 ? params->max_cells : kStaticMaxCells;
  const int K = std::min<int>(params->k_views, n_cams);
  const int k1 = K - 1;
  if (n_px > kStaticMaxPixels || n_rays > kStaticMaxRays || max_cells > kStaticMaxCells ||
      2ll * k1 * n_rays > kStaticMaxPairRays)
    return FUSEFLOW_ERR_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the rig constants go through host staging arrays that the next call overwrites, so a
  // captured call would replay another call's constants: capture is refused
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return FUSEFLOW_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return FUSEFLOW_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FUSEFLOW_ERR_CUDA;

  std::lock_guard<std::mutex> lock(g_static_mutex);
  unsigned char* base = nullptr;
  int st = static_scratch(dev, s, &base);
  if (st != FUSEFLOW_OK) return st;

  // rig constants, the same quantities fuseflow_create derives (Eq. 4 relative poses,
  // Sec. II.5(2)b neighbour table, ray tables), staged in host statics
  int32_t nbr[kMaxCams * kMaxK1];
  neighbour_table_fixed(extr, n_cams, k1, nbr);
  const double unit = params->depth_scale;
  RigDev& rig = g_static_rig;
  build_rig(intr, extr, n_cams, params, nbr, k1, rig, g_static_rays, g_static_pray);
  const int nr = (int)n_rays;
  const int np = (int)(2ll * k1 * n_rays);
  Geometry geo{};
  const int n_tiles = fill_tile_index(rig, &geo.tiles, 16);
  {
    int sm_count = 152;
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    geo.tiles.ahead = assign_resident_blocks(16, rig.k1) * sm_count;
  }
  fill_block_consts(rig, g_static_bconst);
  // pageable host -> device copies return once the host buffers have been read
  if (cudaMemcpyAsync(base + kSBConst, g_static_bconst, sizeof(BlockConst) * (size_t)n_cams,
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + kSRig, &rig, sizeof(RigDev), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + kSRays, g_static_rays, sizeof(float2) * (size_t)nr, cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      (np > 0 && cudaMemcpyAsync(base + kSPRay, g_static_pray, sizeof(float4) * (size_t)np,
                                 cudaMemcpyHostToDevice, s) != cudaSuccess))
    return FUSEFLOW_ERR_CUDA;

  geo.n_cams = n_cams;
  geo.top_k = params->top_k;
  geo.depth_f32 = rig.depth_f32;
  geo.count_blocks_x = (int)((max_px + 2047) / 2048);
  geo.count_chunks = 1;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  geo.emit_blocks = std::max(1, sms * 8);
  geo.pdl = 2;                                         // at most 2^19 pixels: small frames
  Tables t = static_tables(base, n_px, geo.count_blocks_x * n_cams);
  t.n_min = params->n_min;
  t.max_level = params->max_level;
  t.bconst = reinterpret_cast<const BlockConst*>(base + kSBConst);
  t.pray = reinterpret_cast<const float4*>(base + kSPRay);
  t.n_tiles = n_tiles;
  OutDev od{};
  od.stats = stats;
  od.pos = pos;
  od.rgb = rgb_out;
  od.weight = weight;
  od.count = count;
  od.rep = rep;
  od.key = reinterpret_cast<unsigned long long*>(key);
  od.max_cells = max_cells;
  od.s0_m = params->coarse_cell_m;
  od.unit_m = unit;
  od.unit_f = (float)unit;
  FramePtrs fp{};
  for (int i = 0; i < n_cams; ++i) {
    fp.depth[i] = depth[i];
    fp.conf[i] = conf[i];
    fp.rgb[i] = rgb[i];
  }
  const cudaError_t e = launch_frame(reinterpret_cast<const RigDev*>(base + kSRig),
                                     reinterpret_cast<const float2*>(base + kSRays), fp, t,
                                     TraceDev{}, od, geo, s, nullptr);
  return e == cudaSuccess ? FUSEFLOW_OK : FUSEFLOW_ERR_CUDA;
}
