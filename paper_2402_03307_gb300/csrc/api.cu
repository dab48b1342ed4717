// C ABI of libr4g: argument checks, frame layout and the launch sequence of
// the render (preprocess -> scan + key build -> radix sort -> tile ranges ->
// blend) and of its backward (blend backward -> preprocess backward).
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "r4g.h"
#include "r4g_internal.cuh"

struct r4g_ctx {
  r4g_config cfg;
  char err[512];
  // side stream of a render: the tile counts run there while the depth sort
  // and the binning run on the caller's stream (made on first use, on the
  // device current then)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  int device = -1;  // the device the side stream belongs to
  bool timing = false;
  struct Pending {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  double ms[R4G_NSTAGES] = {};
  int64_t launches[R4G_NSTAGES] = {};
};

namespace {

thread_local char g_err[512] = "";

r4g_status fail(r4g_ctx* ctx, r4g_status st, const char* msg) {
  char* dst = ctx ? ctx->err : g_err;
  std::snprintf(dst, 512, "%s", msg);
  return st;
}

r4g_status cuda_fail(r4g_ctx* ctx, cudaError_t e, const char* where) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  return fail(ctx, R4G_ECUDA, buf);
}

size_t align_up(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

bool tile_ok(int tw, int th) {
  return (tw == 16 && th == 16) || (tw == 8 && th == 8) || (tw == 16 && th == 32);
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

r4g_status check_gaussians(r4g_ctx* ctx, const r4g_gaussians* g) {
  if (!g) return fail(ctx, R4G_EINVAL, "gaussians is NULL");
  if (g->n < 0 || g->n > (int64_t(1) << 31) - 1) return fail(ctx, R4G_EINVAL, "n out of range");
  if ((g->scale_dtype != R4G_F32 && g->scale_dtype != R4G_BF16) ||
      (g->sh_dtype != R4G_F32 && g->sh_dtype != R4G_BF16))
    return fail(ctx, R4G_EINVAL, "unknown dtype");
  if (g->n == 0) return R4G_OK;
  if (!g->mean || !g->rotor || !g->logscale || !g->logit || !g->sh)
    return fail(ctx, R4G_EINVAL, "a parameter pointer is NULL");
  if (!aligned(g->mean, 16) || !aligned(g->rotor, 16) || !aligned(g->sh, 16) ||
      !aligned(g->logscale, g->scale_dtype == R4G_BF16 ? 8 : 16) || !aligned(g->logit, 4))
    return fail(ctx, R4G_EINVAL, "parameter buffers must be 16-byte aligned");
  return R4G_OK;
}

r4g_status check_camera(r4g_ctx* ctx, const r4g_camera* c) {
  if (!c) return fail(ctx, R4G_EINVAL, "camera is NULL");
  if (c->width <= 0 || c->height <= 0 || c->width > 32768 || c->height > 32768)
    return fail(ctx, R4G_EINVAL, "image size out of range (1..32768)");
  if (!(c->fx > 0) || !(c->fy > 0) || !std::isfinite(c->cx) || !std::isfinite(c->cy))
    return fail(ctx, R4G_EINVAL, "bad intrinsics");
  return R4G_OK;
}

cudaEvent_t take_event(r4g_ctx* ctx) {
  if (!ctx->pool.empty()) {
    cudaEvent_t e = ctx->pool.back();
    ctx->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Brackets one stage of a call: records an event pair around it when timing
// is enabled and counts the stage's kernel launches.
struct StageScope {
  r4g_ctx* ctx;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageScope(r4g_ctx* c, int st, cudaStream_t str, int nlaunch) : ctx(c), stage(st), s(str) {
    ctx->launches[stage] += nlaunch;
    if (ctx->timing) {
      a = take_event(ctx);
      if (a) cudaEventRecord(a, s);
    }
  }
  ~StageScope() {
    if (a) {
      cudaEvent_t b = take_event(ctx);
      if (b) {
        cudaEventRecord(b, s);
        ctx->pending.push_back({stage, a, b});
      } else {
        ctx->pool.push_back(a);
      }
    }
  }
};

}  // namespace

namespace r4g {

void set_last_error(const char* msg) { std::snprintf(g_err, sizeof(g_err), "%s", msg); }

FrameLayout make_layout(int64_t n, const int* widths, const int* heights, int nviews, int64_t cap, int tile_w,
                        int tile_h) {
  FrameLayout L{};
  L.n = n;
  L.cap = cap;
  L.nviews = nviews;
  L.m = n * nviews;
  L.tile_w = tile_w;
  L.tile_h = tile_h;
  int64_t tiles = 0, pix = 0, td = 0;
  int maxvt = 0;
  for (int v = 0; v < nviews; ++v) {
    ViewGeom& G = L.geom[v];
    G.width = widths[v];
    G.height = heights[v];
    G.tiles_x = (G.width + tile_w - 1) / tile_w;
    G.tiles_y = (G.height + tile_h - 1) / tile_h;
    G.tile_off = static_cast<uint32_t>(tiles);
    G.pix_off = static_cast<uint32_t>(pix);
    G.tdiff_off = static_cast<uint32_t>(td);
    tiles += static_cast<int64_t>(G.tiles_x) * G.tiles_y;
    pix += static_cast<int64_t>(G.width) * G.height;
    td += static_cast<int64_t>(G.tiles_x + 1) * (G.tiles_y + 1);
    if (G.tiles_x * G.tiles_y > maxvt) maxvt = G.tiles_x * G.tiles_y;
  }
  L.ntiles = static_cast<int>(tiles);
  L.npix = pix;
  L.tdiff_words = static_cast<int>(td);
  L.max_view_tiles = maxvt;
  L.width = L.geom[0].width;
  L.height = L.geom[0].height;
  L.tiles_x = L.geom[0].tiles_x;
  L.tiles_y = L.geom[0].tiles_y;
  const int64_t m = L.m;
  L.nblocks = static_cast<int>((m + kPreBlock - 1) / kPreBlock);
  L.sort_ctas = sort_ctas_for(cap);
  L.depth_ctas = sort_ctas_for(m);
  int tb = 0;
  while ((int64_t(1) << tb) < L.ntiles) ++tb;
  L.tile_bits = tb;
  const int tpasses = (tb + kSortRadixBits - 1) / kSortRadixBits;
  L.keys_in_1 = tpasses % 2 == 1;
  const int cnt_ctas = L.sort_ctas > L.depth_ctas ? L.sort_ctas : L.depth_ctas;
  const size_t npix = static_cast<size_t>(pix);
  size_t o = 0;
  // the header, the tile-count difference array and the depth sort's scratch
  // first: one memset at the start of a render clears all three, and the sort
  // needs no clearing kernel
  L.header = o;   o = align_up(o + sizeof(FrameHeader));
  L.tdiff = o;    o = align_up(o + sizeof(uint32_t) * td);
  L.onesweep = o; o = align_up(o + onesweep_scratch_bytes(m, 32));
  L.views = o;    o = align_up(o + sizeof(ViewDev) * nviews);
  L.rec = o;      o = align_up(o + 3 * sizeof(float4) * m);
  L.rect = o;     o = align_up(o + sizeof(uint2) * m);
  L.spans = o;    o = align_up(o + 2 * sizeof(uint4) * m);  // per item: 16 tile rows' (offset, width) bytes
  L.touched = o;  o = align_up(o + sizeof(uint32_t) * m);
  L.dkey0 = o;    o = align_up(o + sizeof(uint32_t) * m);
  L.dkey1 = o;    o = align_up(o + sizeof(uint32_t) * m);
  L.ord0 = o;     o = align_up(o + sizeof(uint32_t) * m);
  L.ord1 = o;     o = align_up(o + sizeof(uint32_t) * m);
  L.offs = o;     o = align_up(o + sizeof(uint32_t) * (m + 1));
  L.ioffs = o;    o = align_up(o + sizeof(uint32_t) * m);
  L.srect = o;    o = align_up(o + sizeof(uint4) * m);
  L.chunks = o;   o = align_up(o + sizeof(uint32_t) * ((cap + 2047) / 2048 + 1));
  L.blocksum = o; o = align_up(o + sizeof(uint32_t) * (L.nblocks + 1));
  L.glist = o;    o = align_up(o + sizeof(uint32_t) * n);
  L.keys0 = o;    o = align_up(o + sizeof(uint32_t) * cap);
  L.vals0 = o;    o = align_up(o + sizeof(uint32_t) * cap);
  L.keys1 = o;    o = align_up(o + sizeof(uint32_t) * cap);
  L.vals1 = o;    o = align_up(o + sizeof(uint32_t) * cap);
  L.egid = o;     o = align_up(o + sizeof(uint32_t) * cap);
  L.gbuf = o;     o = align_up(o + 12 * sizeof(float) * cap);
  L.reach = o;    o = align_up(o + static_cast<size_t>(cap));  // 1 when a pair's gradient slot holds a value
  L.ranges = o;   o = align_up(o + sizeof(uint2) * L.ntiles);
  L.torder = o;   o = align_up(o + sizeof(uint32_t) * L.ntiles);  // the blends' tile order
  L.tfinal = o;   o = align_up(o + sizeof(float) * npix);
  L.last = o;     o = align_up(o + sizeof(uint32_t) * npix);
  L.sortcnt = o;  o = align_up(o + sizeof(uint32_t) * kSortRadix * cnt_ctas);
  // the two sorts' scratch apart: the tile sort's is cleared and filled with
  // its histograms on a side stream while the depth sort runs
  L.tsort = o;    o = align_up(o + onesweep_scratch_bytes(cap + kChainSlack, tb));
  // multi-view backward: the visible items and their partial gradients (96 B each)
  const int64_t mi = nviews > 1 ? m : 0;
  L.ilist = o;    o = align_up(o + sizeof(uint32_t) * mi);
  L.ipart = o;    o = align_up(o + 96 * static_cast<size_t>(mi));
  L.total = o;
  return L;
}

FrameLayout make_layout1(int64_t n, int width, int height, int64_t cap, int tile_w, int tile_h) {
  return make_layout(n, &width, &height, 1, cap, tile_w, tile_h);
}

// Sorted tile keys / values of a frame (which buffer depends on the number
// of radix passes: pass p writes buffer 1 when p is even, buffer 0 when odd).
static const uint32_t* sorted_tile_keys(const FrameLayout& L, void* f) {
  return at<uint32_t>(f, L.keys_in_1 ? L.keys1 : L.keys0);
}
static const uint32_t* sorted_vals(const FrameLayout& L, void* f) {
  return at<uint32_t>(f, L.keys_in_1 ? L.vals1 : L.vals0);
}

}  // namespace r4g

using namespace r4g;

namespace {

// Host-side layout of a call; checks the views.
r4g_status batch_layout(r4g_ctx* ctx, int64_t n, const r4g_view* views, int32_t nviews, int64_t cap, int tile_w,
                        int tile_h, FrameLayout* L) {
  if (!views) return fail(ctx, R4G_EINVAL, "views is NULL");
  if (nviews < 1 || nviews > kMaxViews) return fail(ctx, R4G_EINVAL, "nviews must be 1..64");
  if (n * nviews > (int64_t(1) << 31) - 1) return fail(ctx, R4G_EINVAL, "n * nviews out of range (< 2^31)");
  int w[kMaxViews], h[kMaxViews];
  int64_t pix = 0, tiles = 0;
  for (int v = 0; v < nviews; ++v) {
    r4g_status st = check_camera(ctx, &views[v].cam);
    if (st != R4G_OK) return st;
    if (!std::isfinite(views[v].t)) return fail(ctx, R4G_EINVAL, "t is not finite");
    w[v] = views[v].cam.width;
    h[v] = views[v].cam.height;
    const int64_t vt = static_cast<int64_t>((w[v] + tile_w - 1) / tile_w) * ((h[v] + tile_h - 1) / tile_h);
    if (vt > kMaxTiles) return fail(ctx, R4G_EINVAL, "too many tiles (> 51200) in a view for this tile shape");
    pix += static_cast<int64_t>(w[v]) * h[v];
    tiles += vt;
  }
  if (pix > (int64_t(1) << 31) - 1) return fail(ctx, R4G_EINVAL, "too many pixels in the call (>= 2^31)");
  if (tiles > (int64_t(1) << 24)) return fail(ctx, R4G_EINVAL, "too many tiles in the call (> 2^24)");
  *L = make_layout(n, w, h, nviews, cap, tile_w, tile_h);
  return R4G_OK;
}

r4g_status render_impl(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_view* views, int32_t nviews,
                       const r4g_view* views_dev, float* out_rgb, float* out_T, uint32_t* out_last, void* frame,
                       size_t frame_bytes, int64_t key_capacity, void* stream) {
  r4g_status st = check_gaussians(ctx, g);
  if (st != R4G_OK) return st;
  if (!out_rgb || !frame) return fail(ctx, R4G_EINVAL, "out_rgb / frame is NULL");
  if (key_capacity < 0 || key_capacity >= int64_t(1) << 30) return fail(ctx, R4G_EINVAL, "key_capacity out of range (< 2^30)");
  if (!aligned(frame, 256)) return fail(ctx, R4G_EINVAL, "frame must be 256-byte aligned");
  if (views_dev && !aligned(views_dev, 4)) return fail(ctx, R4G_EINVAL, "views_dev must be 4-byte aligned");
  FrameLayout L;
  if ((st = batch_layout(ctx, g->n, views, nviews, key_capacity, ctx->cfg.tile_w, ctx->cfg.tile_h, &L)) != R4G_OK)
    return st;
  if (frame_bytes < L.total) return fail(ctx, R4G_EWORKSPACE, "frame smaller than r4g_frame_bytes");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the header, the difference array and the depth sort's scratch (adjacent)
  cudaError_t e = cudaMemsetAsync(at<char>(frame, L.header), 0,
                                  L.onesweep + onesweep_scratch_bytes(L.m, 32) - L.header, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  const bool has = L.n > 0;
  const int dpasses = 32 / kSortRadixBits;
  const int tpasses = (L.tile_bits + kSortRadixBits - 1) / kSortRadixBits;
  {
    StageScope sc(ctx, R4G_STAGE_PREPROCESS, s, (L.nviews > 1 || !has) ? (has ? 2 : 1) : 1);
    if ((e = launch_preprocess_fwd(*g, L, frame, ctx->cfg.sh_degree, ctx->cfg.flags, views, views_dev, s)) !=
        cudaSuccess)
      return cuda_fail(ctx, e, "preprocess");
  }
  uint32_t* err = &at<FrameHeader>(frame, L.header)->status;
  // fork: the tile counts (ranges and the tile sort's histograms) and the
  // clearing of the tile sort's scratch need only the preprocess's output
  {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(ctx, e, "cudaGetDevice");
    if (!ctx->side) {
      if ((e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(ctx, e, "side stream");
      ctx->device = dev;
    } else if (dev != ctx->device) {
      return fail(ctx, R4G_EINVAL, "a context renders on the device current at its first render; use one per device");
    }
  }
  if ((e = cudaEventRecord(ctx->fork, s)) != cudaSuccess || (e = cudaStreamWaitEvent(ctx->side, ctx->fork, 0)) != cudaSuccess)
    return cuda_fail(ctx, e, "fork");
  {
    StageScope sc(ctx, R4G_STAGE_RANGES, ctx->side, 1);
    uint32_t* hist = at<uint32_t>(frame, L.tsort);
    e = tpasses > 0 ? cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kSortRadix * tpasses, ctx->side) : cudaSuccess;
    if (e == cudaSuccess) e = launch_tile_counts(L, frame, hist, tpasses, ctx->side);
    if (e == cudaSuccess && has && tpasses > 0)
      e = prepare_onesweep(hist, L.cap + kChainSlack, L.tile_bits, true, ctx->side);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->join, ctx->side);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tile counts");
  }
  int which = 0;
  if (has) {
    // depth order of the items: stable sort of the depth bits, values = item index
    // (items without tiles dropped by the first pass; as many passes as the
    // frame's depth-key range needs, the others exit at once; the scratch is
    // cleared with the difference array)
    StageScope sc(ctx, R4G_STAGE_SORT, s, 1 + dpasses);
    e = launch_depth_sort(at<uint32_t>(frame, L.dkey0), at<uint32_t>(frame, L.dkey1), at<uint32_t>(frame, L.ord1),
                          at<uint32_t>(frame, L.dkey0), at<uint32_t>(frame, L.ord0), L.m,
                          at<FrameHeader>(frame, L.header), at<void>(frame, L.onesweep), err, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "depth sort");
  }
  {
    // depth-order offsets (and, for a one-tile image, the pair emission)
    StageScope sc(ctx, R4G_STAGE_BINNING, s,
                  has ? (L.nblocks <= kSelfScanBlocks ? 2 : 3) + (tpasses == 0 ? 1 : 0) : 0);
    if ((e = launch_binning(L, frame, s)) != cudaSuccess) return cuda_fail(ctx, e, "binning");
  }
  const uint32_t* count = &at<FrameHeader>(frame, L.header)->key_count;
  // join: the tile sort and the blend need the side stream's work
  if ((e = cudaStreamWaitEvent(s, ctx->join, 0)) != cudaSuccess) return cuda_fail(ctx, e, "join");
  if (has && tpasses > 0) {
    // stable sort of the depth-ordered pairs by tile id: the first pass runs in
    // the pair emission (values: the emission index of each pair), the others
    // here
    StageScope sc(ctx, R4G_STAGE_SORT, s, tpasses);
    void* ts = at<void>(frame, L.tsort);
    e = launch_emit_sort(L, frame, at<uint32_t>(frame, L.keys1), at<uint32_t>(frame, L.vals1),
                         static_cast<const uint32_t*>(ts), onesweep_status(ts, L.tile_bits),
                         onesweep_tickets(ts, L.tile_bits), s);
    if (e == cudaSuccess && tpasses == 2)  // the second pass, its look-back chained within low-digit groups
      e = launch_tile_chain_pass(L, frame, at<uint32_t>(frame, L.keys1), at<uint32_t>(frame, L.vals1),
                                 at<uint32_t>(frame, L.keys0), at<uint32_t>(frame, L.vals0), ts, s);
    else if (e == cudaSuccess)
      e = launch_onesweep(at<uint32_t>(frame, L.keys0), nullptr, at<uint32_t>(frame, L.keys1),
                          at<uint32_t>(frame, L.vals1), at<uint32_t>(frame, L.keys0), at<uint32_t>(frame, L.vals0),
                          count, 0, L.cap, L.tile_bits, ts, err, s, &which, true, true, 0xffffffffu, 0u, 1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tile sort");
  }
  const uint32_t* vals = sorted_vals(L, frame);
  {
    StageScope sc(ctx, R4G_STAGE_BLEND, s, 1);
    static const float kZero[3] = {0.0f, 0.0f, 0.0f};  // the flow has no background
    const float* bg = (ctx->cfg.flags & R4G_FLAG_FLOW) ? kZero : ctx->cfg.bg;
    if ((e = launch_blend_fwd(L, frame, vals, bg, out_rgb, out_T, out_last,
                              (ctx->cfg.flags & R4G_FLAG_COUNT_PAIRS) != 0, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "blend");
  }
  return R4G_OK;
}

r4g_status backward_impl(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_view* views, int32_t nviews,
                         const float* grad_rgb, r4g_grads* grads, void* frame, size_t frame_bytes,
                         int64_t key_capacity, void* stream) {
  r4g_status st = check_gaussians(ctx, g);
  if (st != R4G_OK) return st;
  if (ctx->cfg.flags & R4G_FLAG_FLOW) return fail(ctx, R4G_EINVAL, "the flow render has no backward");
  if (!grad_rgb || !grads || !frame) return fail(ctx, R4G_EINVAL, "NULL argument");
  if (g->n > 0 && (!grads->mean || !grads->rotor || !grads->logscale || !grads->logit || !grads->sh))
    return fail(ctx, R4G_EINVAL, "a gradient pointer is NULL");
  if (g->n > 0 && (!aligned(grads->mean, 16) || !aligned(grads->rotor, 16) || !aligned(grads->logscale, 16) ||
                   !aligned(grads->sh, 16) || !aligned(grads->logit, 4)))
    return fail(ctx, R4G_EINVAL, "gradient buffers must be 16-byte aligned");
  if (key_capacity < 0 || key_capacity >= int64_t(1) << 30) return fail(ctx, R4G_EINVAL, "key_capacity out of range");
  if (!aligned(frame, 256)) return fail(ctx, R4G_EINVAL, "frame must be 256-byte aligned");
  FrameLayout L;
  if ((st = batch_layout(ctx, g->n, views, nviews, key_capacity, ctx->cfg.tile_w, ctx->cfg.tile_h, &L)) != R4G_OK)
    return st;
  if (frame_bytes < L.total) return fail(ctx, R4G_EWORKSPACE, "frame smaller than r4g_frame_bytes");
  if (L.n == 0) return R4G_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  const uint32_t* vals = sorted_vals(L, frame);
  {
    StageScope sc(ctx, R4G_STAGE_BLEND_BWD, s, 1);
    if ((e = launch_blend_bwd(L, frame, vals, ctx->cfg.bg, grad_rgb, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "blend backward");
  }
  {
    // a multi-view FP32 call lists its items, gathers their pair gradients, then
    // runs the item and Gaussian passes
    const bool two_pass = L.nviews > 1 && !(ctx->cfg.flags & R4G_FLAG_FP64_SLICE);
    StageScope sc(ctx, R4G_STAGE_PREPROCESS_BWD, s, two_pass ? 4 : 1);
    if ((e = launch_preprocess_bwd(*g, L, frame, ctx->cfg.sh_degree, ctx->cfg.flags, *grads, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "preprocess backward");
  }
  return R4G_OK;
}

}  // namespace

extern "C" {

int32_t r4g_version(void) { return 1 * 10000 + 0 * 100 + 0; }

r4g_status r4g_create(r4g_ctx** out, const r4g_config* cfg) {
  if (!out) return fail(nullptr, R4G_EINVAL, "out is NULL");
  *out = nullptr;
  r4g_config c;
  if (cfg) {
    c = *cfg;
  } else {
    std::memset(&c, 0, sizeof(c));
    c.tile_w = 16;
    c.tile_h = 16;
    c.sh_degree = 3;
  }
  if (!tile_ok(c.tile_w, c.tile_h)) return fail(nullptr, R4G_EINVAL, "tile shape must be 8x8, 16x16 or 16x32");
  if (c.sh_degree < 0 || c.sh_degree > 3) return fail(nullptr, R4G_EINVAL, "sh_degree must be 0..3");
  if (c.flags & ~(R4G_FLAG_FP64_SLICE | R4G_FLAG_NO_TEMPORAL_CULL | R4G_FLAG_COUNT_PAIRS | R4G_FLAG_FLOW))
    return fail(nullptr, R4G_EINVAL, "unknown flag");
  r4g_ctx* ctx = new (std::nothrow) r4g_ctx;
  if (!ctx) return fail(nullptr, R4G_ENOMEM, "out of host memory");
  ctx->cfg = c;
  ctx->err[0] = 0;
  *out = ctx;
  return R4G_OK;
}

void r4g_destroy(r4g_ctx* ctx) {
  if (!ctx) return;
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  if (ctx->join) cudaEventDestroy(ctx->join);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  for (auto& p : ctx->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  delete ctx;
}

r4g_status r4g_set_timing(r4g_ctx* ctx, int32_t enable) {
  if (!ctx) return fail(nullptr, R4G_EINVAL, "ctx is NULL");
  ctx->timing = enable != 0;
  return R4G_OK;
}

r4g_status r4g_stage_times(r4g_ctx* ctx, double* ms, int64_t* launches, int32_t reset) {
  if (!ctx) return fail(nullptr, R4G_EINVAL, "ctx is NULL");
  for (auto& p : ctx->pending) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.a, p.b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "r4g_stage_times");
    ctx->ms[p.stage] += t;
    ctx->pool.push_back(p.a);
    ctx->pool.push_back(p.b);
  }
  ctx->pending.clear();
  for (int k = 0; k < R4G_NSTAGES; ++k) {
    if (ms) ms[k] = ctx->ms[k];
    if (launches) launches[k] = ctx->launches[k];
    if (reset) {
      ctx->ms[k] = 0;
      ctx->launches[k] = 0;
    }
  }
  return R4G_OK;
}

const char* r4g_last_error(const r4g_ctx* ctx) { return ctx ? ctx->err : g_err; }

r4g_status r4g_frame_bytes(const r4g_ctx* ctx, int64_t n, int32_t width, int32_t height,
                           int64_t key_capacity, size_t* bytes) {
  r4g_ctx* c = const_cast<r4g_ctx*>(ctx);
  if (!ctx || !bytes) return fail(c, R4G_EINVAL, "NULL argument");
  if (n < 0 || n > (int64_t(1) << 31) - 1) return fail(c, R4G_EINVAL, "n out of range");
  if (width <= 0 || height <= 0 || width > 32768 || height > 32768) return fail(c, R4G_EINVAL, "bad image size");
  if (key_capacity < 0 || key_capacity >= int64_t(1) << 30) return fail(c, R4G_EINVAL, "key_capacity out of range (< 2^30)");
  *bytes = make_layout1(n, width, height, key_capacity, ctx->cfg.tile_w, ctx->cfg.tile_h).total;
  return R4G_OK;
}

r4g_status r4g_frame_status(r4g_ctx* ctx, const void* frame, size_t frame_bytes,
                            int64_t* keys_needed, void* stream) {
  if (!ctx || !frame) return fail(ctx, R4G_EINVAL, "NULL argument");
  if (frame_bytes < sizeof(FrameHeader)) return fail(ctx, R4G_EWORKSPACE, "frame too small");
  FrameHeader h;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&h, frame, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "r4g_frame_status");
  if (keys_needed) *keys_needed = h.key_needed;
  if (h.status & 1u) return fail(ctx, R4G_EOVERFLOW, "key capacity exceeded: re-render with a larger frame");
  if (h.status & 2u) return fail(ctx, R4G_ETIMEOUT, "a radix-sort look-back wait hit its iteration limit");
  if (h.status & 4u) return fail(ctx, R4G_EDEVICE, "device views differ in image size from the host views");
  return R4G_OK;
}

r4g_status r4g_frame_status_async(const void* frame, size_t frame_bytes, uint32_t* host_out, void* stream) {
  if (!frame || !host_out) return fail(nullptr, R4G_EINVAL, "NULL argument");
  if (frame_bytes < sizeof(FrameHeader)) return fail(nullptr, R4G_EWORKSPACE, "frame too small");
  static_assert(offsetof(FrameHeader, status) == 0 && offsetof(FrameHeader, key_count) == 4 &&
                    offsetof(FrameHeader, key_needed) == 8,
                "the status words lead the frame header");
  const cudaError_t e = cudaMemcpyAsync(host_out, frame, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                        static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "r4g_frame_status_async");
  return R4G_OK;
}

r4g_status r4g_frame_status_decode(const uint32_t* words, int64_t* keys_needed) {
  if (!words) return fail(nullptr, R4G_EINVAL, "NULL argument");
  if (keys_needed) *keys_needed = words[2];
  if (words[0] & 1u) return fail(nullptr, R4G_EOVERFLOW, "key capacity exceeded: re-render with a larger frame");
  if (words[0] & 2u) return fail(nullptr, R4G_ETIMEOUT, "a radix-sort look-back wait hit its iteration limit");
  if (words[0] & 4u) return fail(nullptr, R4G_EDEVICE, "device views differ in image size from the host views");
  return R4G_OK;
}

r4g_status r4g_frame_stats(r4g_ctx* ctx, const void* frame, size_t frame_bytes, r4g_frame_info* out,
                           void* stream) {
  if (!ctx || !frame || !out) return fail(ctx, R4G_EINVAL, "NULL argument");
  if (frame_bytes < sizeof(FrameHeader)) return fail(ctx, R4G_EWORKSPACE, "frame too small");
  FrameHeader h;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&h, frame, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "r4g_frame_stats");
  out->n_visible = h.n_visible;
  out->key_count = h.key_count;
  out->key_needed = h.key_needed;
  out->composited_pairs = (ctx->cfg.flags & R4G_FLAG_COUNT_PAIRS) ? static_cast<int64_t>(h.composited) : -1;
  out->status = (h.status & 1u)   ? R4G_EOVERFLOW
                : (h.status & 2u) ? R4G_ETIMEOUT
                : (h.status & 4u) ? R4G_EDEVICE
                                  : R4G_OK;
  out->reserved = 0;
  out->reached_pairs = h.n_reached;
  out->visible_gaussians = h.n_glist;
  return R4G_OK;
}

r4g_status r4g_frame_export(r4g_ctx* ctx, const void* frame, size_t frame_bytes, int64_t n,
                            int32_t width, int32_t height, uint32_t* key_count, uint64_t* keys,
                            uint32_t* values, uint32_t* ranges, float* records, void* stream) {
  if (!ctx || !frame) return fail(ctx, R4G_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FrameHeader h;
  cudaError_t e = cudaMemcpyAsync(&h, frame, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "r4g_frame_export");
  // The key capacity is not stored in the frame; the largest one that fits is
  // recovered from the frame size, which is how the layout was made.
  int64_t lo = 0, hi = int64_t(0xffffffffu);
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo + 1) / 2;
    if (make_layout1(n, width, height, mid, ctx->cfg.tile_w, ctx->cfg.tile_h).total <= frame_bytes) lo = mid;
    else hi = mid - 1;
  }
  const FrameLayout L = make_layout1(n, width, height, lo, ctx->cfg.tile_w, ctx->cfg.tile_h);
  if (L.total > frame_bytes || h.key_count > L.cap) return fail(ctx, R4G_EWORKSPACE, "frame size does not match");
  void* f = const_cast<void*>(frame);
  const uint32_t K = h.key_count;
  if (key_count) e = cudaMemcpyAsync(key_count, &at<FrameHeader>(f, L.header)->key_count, 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && keys && K) e = launch_export_keys(L, f, sorted_tile_keys(L, f), sorted_vals(L, f), keys, s);
  if (e == cudaSuccess && values && K) e = launch_export_values(L, f, sorted_vals(L, f), values, s);
  if (e == cudaSuccess && ranges)
    e = cudaMemcpyAsync(ranges, at<uint2>(f, L.ranges), 8ull * L.ntiles, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && records && n) {
    const char* rec = at<char>(f, L.rec);
    for (int part = 0; part < 3 && e == cudaSuccess; ++part)
      e = cudaMemcpy2DAsync(records + 4 * part, 48, rec + part * 16 * n, 16, 16, n, cudaMemcpyDeviceToDevice, s);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "r4g_frame_export");
  return R4G_OK;
}

r4g_status r4g_render(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_camera* cam, float t,
                      float* out_rgb, float* out_T, uint32_t* out_last, void* frame,
                      size_t frame_bytes, int64_t key_capacity, void* stream) {
  if (!ctx) return fail(nullptr, R4G_EINVAL, "ctx is NULL");
  r4g_status st = check_camera(ctx, cam);
  if (st != R4G_OK) return st;
  if (!std::isfinite(t)) return fail(ctx, R4G_EINVAL, "t is not finite");
  r4g_view v;
  v.cam = *cam;
  v.t = t;
  return render_impl(ctx, g, &v, 1, nullptr, out_rgb, out_T, out_last, frame, frame_bytes, key_capacity, stream);
}

r4g_status r4g_render_backward(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_camera* cam, float t,
                               const float* grad_rgb, r4g_grads* grads, void* frame,
                               size_t frame_bytes, int64_t key_capacity, void* stream) {
  if (!ctx) return fail(nullptr, R4G_EINVAL, "ctx is NULL");
  r4g_status st = check_camera(ctx, cam);
  if (st != R4G_OK) return st;
  r4g_view v;
  v.cam = *cam;
  v.t = t;
  return backward_impl(ctx, g, &v, 1, grad_rgb, grads, frame, frame_bytes, key_capacity, stream);
}

r4g_status r4g_batch_frame_bytes(const r4g_ctx* ctx, int64_t n, const r4g_view* views, int32_t nviews,
                                 int64_t key_capacity, int32_t tile_w, int32_t tile_h, size_t* bytes) {
  r4g_ctx* c = const_cast<r4g_ctx*>(ctx);
  if (!ctx || !bytes) return fail(c, R4G_EINVAL, "NULL argument");
  if (n < 0 || n > (int64_t(1) << 31) - 1) return fail(c, R4G_EINVAL, "n out of range");
  if (key_capacity < 0 || key_capacity >= int64_t(1) << 30) return fail(c, R4G_EINVAL, "key_capacity out of range");
  if (tile_w == 0 && tile_h == 0) {
    tile_w = ctx->cfg.tile_w;
    tile_h = ctx->cfg.tile_h;
  }
  if (!tile_ok(tile_w, tile_h)) return fail(c, R4G_EINVAL, "tile shape must be 8x8, 16x16 or 16x32");
  FrameLayout L;
  r4g_status st = batch_layout(c, n, views, nviews, key_capacity, tile_w, tile_h, &L);
  if (st != R4G_OK) return st;
  *bytes = L.total;
  return R4G_OK;
}

r4g_status r4g_render_batch(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_view* views, int32_t nviews,
                            const r4g_view* views_dev, float* out_rgb, float* out_T, void* frame,
                            size_t frame_bytes, int64_t key_capacity, void* stream) {
  if (!ctx) return fail(nullptr, R4G_EINVAL, "ctx is NULL");
  return render_impl(ctx, g, views, nviews, views_dev, out_rgb, out_T, nullptr, frame, frame_bytes, key_capacity,
                     stream);
}

r4g_status r4g_render_batch_backward(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_view* views,
                                     int32_t nviews, const float* grad_rgb, r4g_grads* grads, void* frame,
                                     size_t frame_bytes, int64_t key_capacity, void* stream) {
  if (!ctx) return fail(nullptr, R4G_EINVAL, "ctx is NULL");
  return backward_impl(ctx, g, views, nviews, grad_rgb, grads, frame, frame_bytes, key_capacity, stream);
}

r4g_status r4g_autotune_batch(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_view* views, int32_t nviews,
                              float* out_rgb, const float* grad_rgb, r4g_grads* grads, void* frame,
                              size_t frame_bytes, int64_t key_capacity, int32_t reps, void* stream,
                              r4g_tune_result* out) {
  if (!ctx || !out) return fail(ctx, R4G_EINVAL, "NULL argument");
  if (reps < 1 || reps > 1000) return fail(ctx, R4G_EINVAL, "reps must be 1..1000");
  if (ctx->timing) return fail(ctx, R4G_EINVAL, "disable stage timing while tuning");
  static const int kShapes[3][2] = {{8, 8}, {16, 16}, {16, 32}};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int32_t tw0 = ctx->cfg.tile_w, th0 = ctx->cfg.tile_h;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(ctx, R4G_ECUDA, "cudaEventCreate");
  }
  int best = -1;
  r4g_status result = R4G_OK;
  for (int k = 0; k < 3; ++k) {
    out->ms[k] = -1.0f;
    out->keys_needed[k] = -1;
    ctx->cfg.tile_w = kShapes[k][0];
    ctx->cfg.tile_h = kShapes[k][1];
    FrameLayout L;
    if (batch_layout(ctx, g ? g->n : 0, views, nviews, key_capacity, kShapes[k][0], kShapes[k][1], &L) != R4G_OK ||
        L.total > frame_bytes)
      continue;  // this shape does not fit the frame or the tile limit
    float ms = 0.0f;
    cudaError_t e = cudaSuccess;
    r4g_status st = R4G_OK;
    for (int r = -1; r < reps && st == R4G_OK && e == cudaSuccess; ++r) {  // r = -1: warm-up
      if (r == 0) e = cudaEventRecord(e0, s);
      st = render_impl(ctx, g, views, nviews, nullptr, out_rgb, nullptr, nullptr, frame, frame_bytes, key_capacity,
                       stream);
      if (st == R4G_OK && grad_rgb)
        st = backward_impl(ctx, g, views, nviews, grad_rgb, grads, frame, frame_bytes, key_capacity, stream);
    }
    if (st != R4G_OK) {
      result = st;
      break;
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    FrameHeader h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, frame, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      result = cuda_fail(ctx, e, "r4g_autotune_batch");
      break;
    }
    out->keys_needed[k] = h.key_needed;
    if (h.status & 3u) continue;  // overflow or a sort wait gave up: not a valid timing
    out->ms[k] = ms / reps;
    if (best < 0 || out->ms[k] < out->ms[best]) best = k;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != R4G_OK || best < 0) {
    ctx->cfg.tile_w = tw0;
    ctx->cfg.tile_h = th0;
    if (result != R4G_OK) return result;
    return fail(ctx, R4G_EOVERFLOW, "no tile shape rendered within the frame and key capacity");
  }
  ctx->cfg.tile_w = kShapes[best][0];
  ctx->cfg.tile_h = kShapes[best][1];
  out->tile_w = ctx->cfg.tile_w;
  out->tile_h = ctx->cfg.tile_h;
  return R4G_OK;
}

r4g_status r4g_set_tile(r4g_ctx* ctx, int32_t tile_w, int32_t tile_h) {
  if (!ctx) return fail(nullptr, R4G_EINVAL, "ctx is NULL");
  if (!tile_ok(tile_w, tile_h)) return fail(ctx, R4G_EINVAL, "tile shape must be 8x8, 16x16 or 16x32");
  ctx->cfg.tile_w = tile_w;
  ctx->cfg.tile_h = tile_h;
  return R4G_OK;
}

r4g_status r4g_get_config(const r4g_ctx* ctx, r4g_config* out) {
  if (!ctx || !out) return fail(const_cast<r4g_ctx*>(ctx), R4G_EINVAL, "NULL argument");
  *out = ctx->cfg;
  return R4G_OK;
}

r4g_status r4g_sort_scratch_bytes(int64_t n, size_t* bytes) {
  if (!bytes || n < 0 || n > int64_t(0xffffffffu)) return fail(nullptr, R4G_EINVAL, "bad argument");
  const int ctas = sort_ctas_for(n);
  *bytes = align_up(sizeof(uint64_t) * n) + align_up(sizeof(uint32_t) * n) +
           align_up(sizeof(uint32_t) * kSortRadix * ctas);
  return R4G_OK;
}

r4g_status r4g_sort_pairs(const uint64_t* keys_in, const uint32_t* values_in, uint64_t* keys_out,
                          uint32_t* values_out, int64_t n, int32_t begin_bit, int32_t end_bit,
                          void* scratch, size_t scratch_bytes, void* stream) {
  if (n < 0 || n > int64_t(0xffffffffu)) return fail(nullptr, R4G_EINVAL, "n out of range");
  if (begin_bit < 0 || end_bit > 64 || begin_bit >= end_bit) return fail(nullptr, R4G_EINVAL, "bad bit range");
  size_t need = 0;
  r4g_sort_scratch_bytes(n, &need);
  if (n == 0) return R4G_OK;
  if (!keys_in || !values_in || !keys_out || !values_out || !scratch) return fail(nullptr, R4G_EINVAL, "NULL argument");
  if (scratch_bytes < need) return fail(nullptr, R4G_EWORKSPACE, "scratch smaller than r4g_sort_scratch_bytes");
  if (!aligned(scratch, 256) || !aligned(keys_in, 8) || !aligned(keys_out, 8))
    return fail(nullptr, R4G_EINVAL, "misaligned buffer");
  if (keys_in == keys_out || values_in == values_out) return fail(nullptr, R4G_EINVAL, "outputs alias inputs");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint64_t* tk = at<uint64_t>(scratch, 0);
  uint32_t* tv = at<uint32_t>(scratch, align_up(sizeof(uint64_t) * n));
  uint32_t* cnt = at<uint32_t>(scratch, align_up(sizeof(uint64_t) * n) + align_up(sizeof(uint32_t) * n));
  const int passes = (end_bit - begin_bit + kSortRadixBits - 1) / kSortRadixBits;
  // the last pass (index passes-1) writes buffer 1 when its index is even
  const bool last_even = (passes - 1) % 2 == 0;
  uint64_t* k1 = last_even ? keys_out : tk;
  uint32_t* v1 = last_even ? values_out : tv;
  uint64_t* k2 = last_even ? tk : keys_out;
  uint32_t* v2 = last_even ? tv : values_out;
  int which = 0;
  const cudaError_t e = launch_sort(keys_in, values_in, k1, v1, k2, v2, nullptr, static_cast<uint32_t>(n), n,
                                    begin_bit, end_bit, cnt, sort_ctas_for(n), s, &which);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "sort");
  return R4G_OK;
}

}  // extern "C"
