// Per-Gaussian preprocess of the render (forward). One thread per Gaussian
// for all the views of a call: the view-independent part (parameters,
// rotor, R, Sigma4) is computed once, the slice and projection once per
// view. Coalesced 16-byte loads of the SoA parameters; the SH row is read
// only for survivors.
//
// This file is compiled without floating-point contraction (-fmad=false):
// every multiply and add rounds as written, so the one-view and the
// multi-view kernels (which the compiler schedules differently) produce the
// same bits, and a view of a batch equals its single-view render.
#include <cuda_runtime.h>

#include "preprocess_common.cuh"
#include "tile_rows.cuh"

namespace r4g {

// ---- view table ---------------------------------------------------------------
struct HostViews {
  r4g_view v[kMaxViews];
};
struct GeomTable {
  ViewGeom g[kMaxViews];
};

// The camera as the kernels use it (rotation, centre -R^T t, focal lengths
// and the 1.3 tan(fov/2) clamp of J) and the view's place in the batch. A
// device view whose image size differs from the host layout sets status
// bit 2 and is rendered with the layout's size.
__device__ __forceinline__ ViewDev make_view(const r4g_view& V, const ViewGeom& G, FrameHeader* hdr) {
  ViewDev d;
  CamDev& c = d.cam;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int j = 0; j < 3; ++j) c.R[3 * k + j] = V.cam.world_to_cam[4 * k + j];
    c.t[k] = V.cam.world_to_cam[4 * k + 3];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {  // centre = -R^T t
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) acc = __fsub_rn(acc, __fmul_rn(c.R[3 * k + j], c.t[k]));
    c.pos[j] = acc;
  }
  c.fx = V.cam.fx;
  c.fy = V.cam.fy;
  c.cx = V.cam.cx;
  c.cy = V.cam.cy;
  c.limx = __fmul_rn(kClampFov, __fdiv_rn(static_cast<float>(G.width), __fmul_rn(2.0f, c.fx)));
  c.limy = __fmul_rn(kClampFov, __fdiv_rn(static_cast<float>(G.height), __fmul_rn(2.0f, c.fy)));
  c.width = G.width;
  c.height = G.height;
  d.t = V.t;
  d.tiles_x = G.tiles_x;
  d.tiles_y = G.tiles_y;
  d.tile_off = G.tile_off;
  d.pix_off = G.pix_off;
  d.tdiff_off = G.tdiff_off;
  d.pad[0] = d.pad[1] = d.pad[2] = 0u;
  if (hdr && (V.cam.width != G.width || V.cam.height != G.height)) atomicOr(&hdr->status, 4u);
  return d;
}

// Multi-view calls: one thread per view writes the frame's view table, from
// the host views (a kernel parameter) or from device views.
__global__ void setup_views_kernel(HostViews hv, GeomTable gt, const r4g_view* __restrict__ vdev, int nviews,
                                   ViewDev* __restrict__ out, FrameHeader* hdr) {
  const int v = threadIdx.x;
  if (v >= nviews) return;
  const r4g_view V = vdev ? vdev[v] : hv.v[v];
  out[v] = make_view(V, gt.g[v], hdr);
}

cudaError_t launch_setup_views(const FrameLayout& L, void* frame, const r4g_view* views_host,
                               const r4g_view* views_dev, cudaStream_t s) {
  HostViews hv;
  GeomTable gt;
  for (int v = 0; v < L.nviews; ++v) {
    hv.v[v] = views_host ? views_host[v] : r4g_view{};
    gt.g[v] = L.geom[v];
  }
  setup_views_kernel<<<1, kMaxViews, 0, s>>>(hv, gt, views_dev, L.nviews, at<ViewDev>(frame, L.views),
                                             at<FrameHeader>(frame, L.header));
  return cudaGetLastError();
}

// ---- forward ------------------------------------------------------------------
// kMulti: several views (a loop keeping the view-independent values live);
// otherwise exactly one, with a smaller register footprint.
// One view (kMulti false) needs no setup launch: every block builds the
// view's table entry from the host view (or the device view) itself, and
// block 0 stores it in the frame for the later kernels.
struct OneView {
  r4g_view v;
  ViewGeom g;
  const r4g_view* vdev;
};

template <typename S, bool kScaleBF16, bool kShBF16, bool kMulti>
__global__ void __launch_bounds__(kPreFwdBlock, kMulti ? 4 : 7)
    preprocess_fwd_kernel(r4g_gaussians g, ViewDev* __restrict__ views, int nviews, OneView one, PreOut out,
                          int sh_degree, bool temporal_cull, bool flow) {
  // the next kernel of the render (the depth sort's) may launch now and wait
  griddep_launch_dependents();
  if constexpr (!kMulti) nviews = 1;
  __shared__ uint32_t s_pairs[kMaxViews];
  __shared__ uint32_t s_wcnt[kPreFwdBlock / 32];
  __shared__ uint32_t s_vis, s_base, s_kminc, s_kmax;
  __shared__ uint32_t s_cnt[kPreFwdBlock];  // each thread's pair count in the current view
  __shared__ __align__(16) ViewDev s_views[kMaxViews];  // the view table (copied as 16-byte words)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = threadIdx.x; v < kMaxViews; v += kPreFwdBlock) s_pairs[v] = 0;
  // the view-independent part first: its loads and Sigma4 overlap the
  // building of the view table
  const int i = blockIdx.x * kPreFwdBlock + threadIdx.x;
  const bool live = i < g.n;
  Sig4<S> G;
  if (live) gauss_sigma<S, kScaleBF16>(g, i, G);
  if constexpr (kMulti) {
    for (int k = threadIdx.x; k < nviews * 8; k += kPreFwdBlock)
      reinterpret_cast<uint4*>(s_views)[k] = reinterpret_cast<const uint4*>(views)[k];
  } else if (threadIdx.x == 0) {
    const ViewDev d = make_view(one.vdev ? one.vdev[0] : one.v, one.g, blockIdx.x == 0 ? out.header : nullptr);
    s_views[0] = d;
    if (blockIdx.x == 0) views[0] = d;
  }
  if (threadIdx.x == 0) s_vis = s_kminc = s_kmax = 0;
  __syncthreads();
  uint32_t nvis = 0;
  uint32_t kminc = 0, kmax = 0;  // range of this thread's depth keys (complemented minimum)
  const size_t M = static_cast<size_t>(g.n) * nviews;
  for (int v = 0; v < (kMulti ? nviews : 1); ++v) {
    uint32_t ntiles = 0;
    const ViewDev& V = s_views[v];
    const size_t item = static_cast<size_t>(v) * g.n + i;
    bool vis = false;
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    TileEllipse E{};
    uint32_t key = 0xffffffffu;
    if (live) {
      const CamDev& cam = V.cam;
      Fwd f;
      S invW, dt;
      view_geometry<S>(G, cam, V.t, temporal_cull, f, invW, dt);
      int i0 = 0, i1 = -1, j0 = 0, j1 = -1;
      vis = f.visible && pixel_box(f, cam, i0, i1, j0, j1);
      key = __float_as_uint(f.pc[2]);
      if (vis) {
        if (flow) {  // the colour slot carries d(mean2d)/dt (channel 2 zero)
          image_velocity<S>(G, invW, cam, f);
        } else {
          forward_color<kShBF16>(g, i, cam, sh_degree, f);
        }
        x0 = i0 / out.tile_w;
        x1 = i1 / out.tile_w + 1;
        y0 = j0 / out.tile_h;
        y1 = j1 / out.tile_h + 1;
        // with the opacity's logarithms the blends' staging needs
        const float l255 = __log2f(255.0f * f.o_t);
        out.recA[item] = make_float4(f.mean2d[0], f.mean2d[1], f.conic[0], f.conic[1]);
        out.recA[M + item] = make_float4(f.conic[2], f.o_t, f.pc[2], l255);
        out.recA[2 * M + item] = make_float4(f.rgb[0], f.rgb[1], f.rgb[2], fmaxf(__log2f(f.o_t), -126.0f));
        out.rect[item] = make_uint2(static_cast<uint32_t>(x0) | (static_cast<uint32_t>(y0) << 16),
                                    static_cast<uint32_t>(x1) | (static_cast<uint32_t>(y1) << 16));
        if (span_mode(x0, x1, y0, y1))
          E = tile_ellipse(f.mean2d[0], f.mean2d[1], f.conic[0], f.conic[1], f.conic[2], l255);
      } else {
        out.recA[item] = make_float4(0.f, 0.f, 0.f, 0.f);
        out.recA[M + item] = make_float4(0.f, 0.f, 0.f, 0.f);
        out.recA[2 * M + item] = make_float4(0.f, 0.f, 0.f, 0.f);
        out.rect[item] = make_uint2(0u, 0u);
      }
    }
    {
      // The tiles of each tile row the contributing ellipse meets (an
      // interval; every tile of the row for a rectangle too large to store
      // spans for), +1 on each as two updates of the row's difference array,
      // the spans kept for the pair emission. The warp shares the rows of its
      // lanes' Gaussians out 32 at a time (lanes' row counts differ widely).
      {
        const int R = vis ? y1 - y0 : 0;
        int pre = R;  // inclusive scan of the row counts over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, pre, o);
          if (lane >= o) pre += y;
        }
        const int excl = pre - R;
        const int total = __shfl_sync(0xffffffffu, pre, 31);
        s_cnt[threadIdx.x] = 0u;
        __syncwarp();
        uint32_t* td = out.tdiff + V.tdiff_off;
        const int st = V.tiles_x + 1;
        uint16_t* sp16 = reinterpret_cast<uint16_t*>(out.spans);
        for (int f0 = 0; f0 < total; f0 += 32) {
          const int fi = f0 + lane;
          int j = 0;  // the lane whose rows hold flattened row fi: the last with excl <= fi
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const int cand = j + step;
            const int ec = __shfl_sync(0xffffffffu, excl, cand & 31);
            if (cand < 32 && ec <= fi) j = cand;
          }
          TileEllipse Ej;
          Ej.mx = __shfl_sync(0xffffffffu, E.mx, j);
          Ej.my = __shfl_sync(0xffffffffu, E.my, j);
          Ej.a = __shfl_sync(0xffffffffu, E.a, j);
          Ej.b = __shfl_sync(0xffffffffu, E.b, j);
          Ej.c = __shfl_sync(0xffffffffu, E.c, j);
          Ej.thr = __shfl_sync(0xffffffffu, E.thr, j);
          Ej.det = __shfl_sync(0xffffffffu, E.det, j);
          Ej.ia = __shfl_sync(0xffffffffu, E.ia, j);
          Ej.rx = __shfl_sync(0xffffffffu, E.rx, j);
          Ej.ry = __shfl_sync(0xffffffffu, E.ry, j);
          Ej.dyl = __shfl_sync(0xffffffffu, E.dyl, j);
          Ej.dyr = __shfl_sync(0xffffffffu, E.dyr, j);
          Ej.exact = __shfl_sync(0xffffffffu, E.exact ? 1 : 0, j) != 0;
          const int jx0 = __shfl_sync(0xffffffffu, x0, j), jx1 = __shfl_sync(0xffffffffu, x1, j);
          const int jy0 = __shfl_sync(0xffffffffu, y0, j), jy1 = __shfl_sync(0xffffffffu, y1, j);
          const int jex = __shfl_sync(0xffffffffu, excl, j);
          if (fi >= total) continue;
          const int k = fi - jex, ty = jy0 + k;
          const bool spanned = span_mode(jx0, jx1, jy0, jy1);
          int c0 = jx0, c1 = jx1 - 1;
          const bool ok = spanned ? tile_row_span(Ej, ty, out.tws, out.ths, jx0, jx1, c0, c1) : true;
          uint32_t w = 0;
          if (ok) {
            atomicAdd(td + ty * st + c0, 1u);
            atomicAdd(td + ty * st + c1 + 1, 0xffffffffu);
            w = static_cast<uint32_t>(c1 - c0 + 1);
            atomicAdd(&s_cnt[(threadIdx.x & ~31) + j], w);
          }
          if (spanned) {
            const size_t jitem = static_cast<size_t>(v) * g.n + (i - lane + j);
            sp16[jitem * kSpanRows + k] = static_cast<uint16_t>(ok ? (static_cast<uint32_t>(c0 - jx0) | (w << 8)) : 0u);
          }
        }
        __syncwarp();
        ntiles = s_cnt[threadIdx.x];
      }
    }
    if (live) {
      out.touched[item] = ntiles;
      out.dkey[item] = ntiles ? key : 0xffffffffu;
      if (ntiles) {
        kminc = max(kminc, ~key);
        kmax = max(kmax, key);
      }
    }
    const uint32_t ws = __reduce_add_sync(0xffffffffu, ntiles);
    if (lane == 0 && ws) atomicAdd(&s_pairs[v], ws);
    nvis += ntiles > 0 ? 1u : 0u;
  }
  // visible items, pairs per view, and the list of Gaussians visible in some
  // view (appended per block, in index order within the block)
  const uint32_t wv = __reduce_add_sync(0xffffffffu, nvis);
  const uint32_t lm = __ballot_sync(0xffffffffu, nvis > 0);
  kminc = __reduce_max_sync(0xffffffffu, kminc);
  kmax = __reduce_max_sync(0xffffffffu, kmax);
  if (lane == 0) {
    s_wcnt[warp] = __popc(lm);
    if (wv) {
      atomicAdd(&s_vis, wv);
      atomicMax(&s_kminc, kminc);
      atomicMax(&s_kmax, kmax);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kPreFwdBlock / 32; ++w) {
      const uint32_t c = s_wcnt[w];
      s_wcnt[w] = tot;
      tot += c;
    }
    s_base = tot ? atomicAdd(&out.header->n_glist, tot) : 0u;
    if (s_vis) {
      atomicAdd(&out.header->n_visible, s_vis);
      atomicMax(&out.header->dkey_minc, s_kminc);
      atomicMax(&out.header->dkey_max, s_kmax);
    }
  }
  for (int v = threadIdx.x; v < nviews; v += kPreFwdBlock)
    if (s_pairs[v]) atomicAdd(&out.header->view_pairs[v], s_pairs[v]);
  __syncthreads();
  if (nvis > 0) out.glist[s_base + s_wcnt[warp] + __popc(lm & ((1u << lane) - 1u))] = static_cast<uint32_t>(i);
}

template <typename S, bool A, bool B>
static void launch_pre_t(const r4g_gaussians& g, ViewDev* views, int nviews, const OneView& one, const PreOut& o,
                         int nblocks, int sh_degree, bool tc, bool fl, cudaStream_t s) {
  if (nviews > 1)
    preprocess_fwd_kernel<S, A, B, true><<<nblocks, kPreFwdBlock, 0, s>>>(g, views, nviews, one, o, sh_degree, tc, fl);
  else
    preprocess_fwd_kernel<S, A, B, false><<<nblocks, kPreFwdBlock, 0, s>>>(g, views, nviews, one, o, sh_degree, tc,
                                                                         fl);
}

cudaError_t launch_preprocess_fwd(const r4g_gaussians& g, const FrameLayout& L, void* frame, int sh_degree,
                                  uint32_t flags, const r4g_view* views_host, const r4g_view* views_dev,
                                  cudaStream_t s) {
  OneView one{};
  if (L.nviews > 1) {
    cudaError_t e = launch_setup_views(L, frame, views_host, views_dev, s);
    if (e != cudaSuccess) return e;
  } else {
    one.v = views_host[0];
    one.g = L.geom[0];
    one.vdev = views_dev;
    if (L.n == 0) {  // no preprocess blocks: the table still has to be written
      cudaError_t e = launch_setup_views(L, frame, views_host, views_dev, s);
      if (e != cudaSuccess) return e;
    }
  }
  if (L.n == 0) return cudaSuccess;
  PreOut o;
  o.recA = at<float4>(frame, L.rec);
  o.rect = at<uint2>(frame, L.rect);
  o.spans = at<uint4>(frame, L.spans);
  o.touched = at<uint32_t>(frame, L.touched);
  o.dkey = at<uint32_t>(frame, L.dkey0);
  o.tdiff = at<uint32_t>(frame, L.tdiff);
  o.glist = at<uint32_t>(frame, L.glist);
  o.header = at<FrameHeader>(frame, L.header);
  o.tile_w = L.tile_w;
  o.tile_h = L.tile_h;
  o.tws = log2_pow2(L.tile_w);
  o.ths = log2_pow2(L.tile_h);
  ViewDev* views = at<ViewDev>(frame, L.views);
  const bool tc = !(flags & R4G_FLAG_NO_TEMPORAL_CULL);
  const bool fl = (flags & R4G_FLAG_FLOW) != 0;
  const bool f64 = flags & R4G_FLAG_FP64_SLICE;
  const bool sb = g.scale_dtype == R4G_BF16, hb = g.sh_dtype == R4G_BF16;
  const int nb = static_cast<int>((L.n + kPreFwdBlock - 1) / kPreFwdBlock);
#define R4G_PF(S_, A_, B_) launch_pre_t<S_, A_, B_>(g, views, L.nviews, one, o, nb, sh_degree, tc, fl, s)
  if (f64) {
    if (sb && hb) R4G_PF(double, true, true);
    else if (sb) R4G_PF(double, true, false);
    else if (hb) R4G_PF(double, false, true);
    else R4G_PF(double, false, false);
  } else {
    if (sb && hb) R4G_PF(float, true, true);
    else if (sb) R4G_PF(float, true, false);
    else if (hb) R4G_PF(float, false, true);
    else R4G_PF(float, false, false);
  }
#undef R4G_PF
  return cudaGetLastError();
}


}  // namespace r4g
