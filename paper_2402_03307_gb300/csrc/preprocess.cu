// Per-Gaussian preprocess of the render (forward): activations, rotor
// normalisation and rotation (appendix A.1/A.2), Sigma4 (Sec. 3.2.1), the
// temporal slice and visibility cull (Sec. 3.2.2, appendix A.3), EWA
// projection (Sec. 3.1), SH colour, and the tile rectangle each Gaussian's
// contributing pixels can lie in. One thread per Gaussian for all the views
// of a call: the view-independent part (parameters, rotor, R, Sigma4) is
// computed once, the slice and projection once per view. Coalesced 16-byte
// loads of the SoA parameters; the SH row is read only for survivors.
#include <cuda_runtime.h>

#include "r4g_internal.cuh"
#include "r4g_math.cuh"

namespace r4g {

// Per-item outputs (item = view * N + Gaussian).
struct PreOut {
  float4* recA;  // [3][M] records: (mean2d.x, mean2d.y, conic a, conic b),
                 // (conic c, opacity_t, depth, 0), (r, g, b, 0)
  uint2* rect;   // tile rect: (x0 | y0 << 16, x1 | y1 << 16), [x0, x1) x [y0, y1)
  uint32_t* touched;
  uint32_t* dkey;  // float bits of the depth for items with tiles, else 0xffffffff
  uint32_t* tdiff; // per view, 2D difference array of the tile counts, (tiles_y + 1) x (tiles_x + 1)
  uint32_t* glist; // Gaussians visible in some view
  FrameHeader* header;
  int tile_w, tile_h;
};

// Everything the forward computes for one Gaussian, kept so the backward can
// reuse the same code path.
struct Fwd {
  bool visible;
  float opacity, o_t, temporal;
  float mu3[3], sig3[6];  // xx, xy, xz, yy, yz, zz
  float pc[3];
  float mean2d[2];
  float cov[3];  // dilated 2D covariance a, b, c
  float conic[3];
  float rgb[3];
  bool rgb_pos[3];  // colour channel not clamped at 0
  float dir[3];     // unit view direction
  float dist;       // |mu3 - campos|
  bool clampx, clampy;
};

// View-independent intermediates of one Gaussian (rotor, R, Sigma4) in the
// slice precision S, kept for the backward.
template <typename S>
struct Geo {
  Params p;
  RotorNorm<S> rn;
  S R[16];
  S sc2[4];
  S C[10];  // Sigma4 upper triangle: xx xy xz xt yy yz yt zz zt tt
  float opacity;
};

template <typename S, bool kScaleBF16>
__device__ __forceinline__ void gauss_setup(const r4g_gaussians& g, int i, Geo<S>& G) {
  load_params<kScaleBF16>(g, i, G.p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float s = expf(G.p.ls[k]);
    G.sc2[k] = static_cast<S>(s) * static_cast<S>(s);
  }
  G.opacity = 1.0f / (1.0f + expf(-G.p.logit));
  rotor_normalize<S>(G.p.rot, G.rn);
  rotor_matrix<S>(G.rn.r, G.R);
  cov4<S>(G.R, G.sc2, G.C);
}

// What the per-view steps need of a Gaussian: Sigma4, the 4D mean, opacity.
template <typename S>
struct Sig4 {
  S C[10];
  float mean[4];
  float opacity;
};

template <typename S, bool kScaleBF16>
__device__ __forceinline__ void gauss_sigma(const r4g_gaussians& g, int i, Sig4<S>& Q) {
  Geo<S> G;
  gauss_setup<S, kScaleBF16>(g, i, G);
#pragma unroll
  for (int k = 0; k < 10; ++k) Q.C[k] = G.C[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) Q.mean[k] = G.p.mean[k];
  Q.opacity = G.opacity;
}

// Slice at t, cull, and EWA projection for one view; invW = 1 / Sigma_tt and
// dt = t - mu_t are returned for the backward.
template <typename S>
__device__ __forceinline__ void view_geometry(const Sig4<S>& Q, const CamDev& cam, float t, bool temporal_cull,
                                              Fwd& f, S& invW, S& dt) {
  const S* C = Q.C;
  const float* pm = Q.mean;
  f.opacity = Q.opacity;
  // Sigma4 = [[U, V], [V^T, W]]: U = C[0,1,2; 1,4,5; 2,5,7], V = (C3, C6, C8), W = C9
  const S W = C[9];
  invW = S(1) / W;
  dt = static_cast<S>(t) - static_cast<S>(pm[3]);
  const S lam_dt2 = dt * dt * invW;
  const S V0 = C[3], V1 = C[6], V2 = C[8];
  const S mv = dt * invW;
  f.mu3[0] = static_cast<float>(static_cast<S>(pm[0]) + mv * V0);
  f.mu3[1] = static_cast<float>(static_cast<S>(pm[1]) + mv * V1);
  f.mu3[2] = static_cast<float>(static_cast<S>(pm[2]) + mv * V2);
  f.sig3[0] = static_cast<float>(C[0] - V0 * V0 * invW);
  f.sig3[1] = static_cast<float>(C[1] - V0 * V1 * invW);
  f.sig3[2] = static_cast<float>(C[2] - V0 * V2 * invW);
  f.sig3[3] = static_cast<float>(C[4] - V1 * V1 * invW);
  f.sig3[4] = static_cast<float>(C[5] - V1 * V2 * invW);
  f.sig3[5] = static_cast<float>(C[7] - V2 * V2 * invW);
  const float lam = static_cast<float>(lam_dt2);
  f.temporal = expf(-0.5f * lam);
  f.o_t = f.opacity * f.temporal;
  bool vis = !(temporal_cull && lam > kTemporalCut);

  // world -> camera
  const float* Rc = cam.R;
  const float x = Rc[0] * f.mu3[0] + Rc[1] * f.mu3[1] + Rc[2] * f.mu3[2] + cam.t[0];
  const float y = Rc[3] * f.mu3[0] + Rc[4] * f.mu3[1] + Rc[5] * f.mu3[2] + cam.t[1];
  const float z = Rc[6] * f.mu3[0] + Rc[7] * f.mu3[1] + Rc[8] * f.mu3[2] + cam.t[2];
  f.pc[0] = x; f.pc[1] = y; f.pc[2] = z;
  vis = vis && (z > kNear);
  const float iz = 1.0f / z;
  // Jacobian of (fx x/z + cx, fy y/z + cy) at the clamped position
  const float rx = x * iz, ry = y * iz;
  const float crx = fminf(fmaxf(rx, -cam.limx), cam.limx);
  const float cry = fminf(fmaxf(ry, -cam.limy), cam.limy);
  f.clampx = crx != rx;
  f.clampy = cry != ry;
  const float j00 = cam.fx * iz, j02 = -cam.fx * crx * iz;
  const float j11 = cam.fy * iz, j12 = -cam.fy * cry * iz;
  // T = J Rc (2x3)
  const float T0[3] = {j00 * Rc[0] + j02 * Rc[6], j00 * Rc[1] + j02 * Rc[7], j00 * Rc[2] + j02 * Rc[8]};
  const float T1[3] = {j11 * Rc[3] + j12 * Rc[6], j11 * Rc[4] + j12 * Rc[7], j11 * Rc[5] + j12 * Rc[8]};
  const float* s3 = f.sig3;
  // M = T Sigma3
  const float M0[3] = {T0[0] * s3[0] + T0[1] * s3[1] + T0[2] * s3[2],
                       T0[0] * s3[1] + T0[1] * s3[3] + T0[2] * s3[4],
                       T0[0] * s3[2] + T0[1] * s3[4] + T0[2] * s3[5]};
  const float M1[3] = {T1[0] * s3[0] + T1[1] * s3[1] + T1[2] * s3[2],
                       T1[0] * s3[1] + T1[1] * s3[3] + T1[2] * s3[4],
                       T1[0] * s3[2] + T1[1] * s3[4] + T1[2] * s3[5]};
  f.cov[0] = M0[0] * T0[0] + M0[1] * T0[1] + M0[2] * T0[2] + kDilation;
  f.cov[1] = M0[0] * T1[0] + M0[1] * T1[1] + M0[2] * T1[2];
  f.cov[2] = M1[0] * T1[0] + M1[1] * T1[1] + M1[2] * T1[2] + kDilation;
  const float det = f.cov[0] * f.cov[2] - f.cov[1] * f.cov[1];
  vis = vis && (det > 0.0f);
  const float idet = 1.0f / det;
  f.conic[0] = f.cov[2] * idet;
  f.conic[1] = -f.cov[1] * idet;
  f.conic[2] = f.cov[0] * idet;
  f.mean2d[0] = cam.fx * rx + cam.cx;
  f.mean2d[1] = cam.fy * ry + cam.cy;
  // alpha <= opacity_t, so below 1/255 nothing is ever composited
  vis = vis && (f.o_t >= kAlphaMin);
  f.visible = vis;
}

template <bool kShBF16>
__device__ __forceinline__ void forward_color(const r4g_gaussians& g, int i, const CamDev& cam,
                                              int sh_degree, Fwd& f, float (*keep_c)[3] = nullptr,
                                              float* keep_Y = nullptr) {
  float d0 = f.mu3[0] - cam.pos[0], d1 = f.mu3[1] - cam.pos[1], d2 = f.mu3[2] - cam.pos[2];
  const float dist = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  const float idist = 1.0f / dist;
  f.dist = dist;
  f.dir[0] = d0 * idist; f.dir[1] = d1 * idist; f.dir[2] = d2 * idist;
  float Y[16];
  sh_basis(f.dir[0], f.dir[1], f.dir[2], Y);
  const int nb = (sh_degree + 1) * (sh_degree + 1);
  float c[16][3];
  load_sh<kShBF16>(g.sh, i, nb, c);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float acc = 0.5f;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k < nb) acc += Y[k] * c[k][ch];
    f.rgb_pos[ch] = acc > 0.0f;
    f.rgb[ch] = fmaxf(acc, 0.0f);
  }
  if (keep_c) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      keep_Y[k] = k < nb ? Y[k] : 0.0f;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) keep_c[k][ch] = k < nb ? c[k][ch] : 0.0f;
    }
  }
}

// Pixel-column range whose centres can lie inside the region where
// alpha >= 1/255 and power >= -4.5, i.e. d^T conic d <= min(9, 2 ln(255 o_t)).
// The axis-aligned box of that ellipse has half-widths sqrt(k2 Sigma'_xx) and
// sqrt(k2 Sigma'_yy); a relative and an absolute slack keep the box a
// superset under FP32 rounding. The box only selects tiles: each pixel still
// applies the exact tests, so the image does not depend on the tile shape.
__device__ __forceinline__ bool pixel_box(const Fwd& f, const CamDev& cam, int& i0, int& i1,
                                          int& j0, int& j1) {
  const float k2 = 1.01f * fminf(9.0f, 2.0f * logf(255.0f * f.o_t));
  const float hx = sqrtf(k2 * f.cov[0]) + 0.5f;
  const float hy = sqrtf(k2 * f.cov[2]) + 0.5f;
  const float lim = 1e7f;
  const float xa = fminf(fmaxf(f.mean2d[0] - hx - 0.5f, -lim), lim);
  const float xb = fminf(fmaxf(f.mean2d[0] + hx - 0.5f, -lim), lim);
  const float ya = fminf(fmaxf(f.mean2d[1] - hy - 0.5f, -lim), lim);
  const float yb = fminf(fmaxf(f.mean2d[1] + hy - 0.5f, -lim), lim);
  i0 = max(static_cast<int>(ceilf(xa)), 0);
  i1 = min(static_cast<int>(floorf(xb)), cam.width - 1);
  j0 = max(static_cast<int>(ceilf(ya)), 0);
  j1 = min(static_cast<int>(floorf(yb)), cam.height - 1);
  return i0 <= i1 && j0 <= j1;
}

// ---- view table ---------------------------------------------------------------
struct HostViews {
  r4g_view v[kMaxViews];
};
struct GeomTable {
  ViewGeom g[kMaxViews];
};

// One thread per view: the camera as the kernels use it (rotation, centre
// -R^T t, focal lengths and the 1.3 tan(fov/2) clamp of J) from the host
// views (a kernel parameter) or from device views, and the view's place in
// the batch. A device view whose image size differs from the host layout
// sets status bit 2 and is rendered with the layout's size.
__global__ void setup_views_kernel(HostViews hv, GeomTable gt, const r4g_view* __restrict__ vdev, int nviews,
                                   ViewDev* __restrict__ out, FrameHeader* hdr) {
  const int v = threadIdx.x;
  if (v >= nviews) return;
  const r4g_view V = vdev ? vdev[v] : hv.v[v];
  const ViewGeom& G = gt.g[v];
  ViewDev d;
  CamDev& c = d.cam;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int j = 0; j < 3; ++j) c.R[3 * k + j] = V.cam.world_to_cam[4 * k + j];
    c.t[k] = V.cam.world_to_cam[4 * k + 3];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {  // centre = -R^T t, in double
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) acc = __dadd_rn(acc, -__dmul_rn(static_cast<double>(c.R[3 * k + j]), c.t[k]));
    c.pos[j] = static_cast<float>(acc);
  }
  c.fx = V.cam.fx;
  c.fy = V.cam.fy;
  c.cx = V.cam.cx;
  c.cy = V.cam.cy;
  c.limx = static_cast<float>(static_cast<double>(kClampFov) * (G.width / (2.0 * static_cast<double>(c.fx))));
  c.limy = static_cast<float>(static_cast<double>(kClampFov) * (G.height / (2.0 * static_cast<double>(c.fy))));
  c.width = G.width;
  c.height = G.height;
  d.t = V.t;
  d.tiles_x = G.tiles_x;
  d.tiles_y = G.tiles_y;
  d.tile_off = G.tile_off;
  d.pix_off = G.pix_off;
  d.tdiff_off = G.tdiff_off;
  d.pad[0] = d.pad[1] = d.pad[2] = 0u;
  if (V.cam.width != G.width || V.cam.height != G.height) atomicOr(&hdr->status, 4u);
  out[v] = d;
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
template <typename S, bool kScaleBF16, bool kShBF16>
__global__ void __launch_bounds__(kPreBlock)
    preprocess_fwd_kernel(r4g_gaussians g, const ViewDev* __restrict__ views, int nviews, PreOut out,
                          int sh_degree, bool temporal_cull) {
  __shared__ uint32_t s_pairs[kMaxViews];
  __shared__ uint32_t s_wcnt[kPreBlock / 32];
  __shared__ uint32_t s_vis, s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = threadIdx.x; v < kMaxViews; v += kPreBlock) s_pairs[v] = 0;
  if (threadIdx.x == 0) s_vis = 0;
  __syncthreads();
  const int i = blockIdx.x * kPreBlock + threadIdx.x;
  const bool live = i < g.n;
  Sig4<S> G;
  if (live) gauss_sigma<S, kScaleBF16>(g, i, G);
  uint32_t nvis = 0;
  const size_t M = static_cast<size_t>(g.n) * nviews;
  for (int v = 0; v < nviews; ++v) {
    uint32_t ntiles = 0;
    if (live) {
      const ViewDev& V = views[v];
      const CamDev& cam = V.cam;
      const size_t item = static_cast<size_t>(v) * g.n + i;
      Fwd f;
      S invW, dt;
      view_geometry<S>(G, cam, V.t, temporal_cull, f, invW, dt);
      int i0 = 0, i1 = -1, j0 = 0, j1 = -1;
      const bool vis = f.visible && pixel_box(f, cam, i0, i1, j0, j1);
      if (vis) {
        forward_color<kShBF16>(g, i, cam, sh_degree, f);
        const int x0 = i0 / out.tile_w, x1 = i1 / out.tile_w + 1;
        const int y0 = j0 / out.tile_h, y1 = j1 / out.tile_h + 1;
        ntiles = static_cast<uint32_t>((x1 - x0) * (y1 - y0));
        out.recA[item] = make_float4(f.mean2d[0], f.mean2d[1], f.conic[0], f.conic[1]);
        out.recA[M + item] = make_float4(f.conic[2], f.o_t, f.pc[2], 0.0f);
        out.recA[2 * M + item] = make_float4(f.rgb[0], f.rgb[1], f.rgb[2], 0.0f);
        out.rect[item] = make_uint2(static_cast<uint32_t>(x0) | (static_cast<uint32_t>(y0) << 16),
                                    static_cast<uint32_t>(x1) | (static_cast<uint32_t>(y1) << 16));
        // +1 on every tile of the rectangle, as four corner updates
        uint32_t* td = out.tdiff + V.tdiff_off;
        const int st = V.tiles_x + 1;
        atomicAdd(td + y0 * st + x0, 1u);
        atomicAdd(td + y0 * st + x1, 0xffffffffu);
        atomicAdd(td + y1 * st + x0, 0xffffffffu);
        atomicAdd(td + y1 * st + x1, 1u);
      } else {
        out.recA[item] = make_float4(0.f, 0.f, 0.f, 0.f);
        out.recA[M + item] = make_float4(0.f, 0.f, 0.f, 0.f);
        out.recA[2 * M + item] = make_float4(0.f, 0.f, 0.f, 0.f);
        out.rect[item] = make_uint2(0u, 0u);
      }
      out.touched[item] = ntiles;
      out.dkey[item] = ntiles ? __float_as_uint(f.pc[2]) : 0xffffffffu;
    }
    const uint32_t ws = __reduce_add_sync(0xffffffffu, ntiles);
    if (lane == 0 && ws) atomicAdd(&s_pairs[v], ws);
    nvis += ntiles > 0 ? 1u : 0u;
  }
  // visible items, pairs per view, and the list of Gaussians visible in some
  // view (appended per block, in index order within the block)
  const uint32_t wv = __reduce_add_sync(0xffffffffu, nvis);
  const uint32_t lm = __ballot_sync(0xffffffffu, nvis > 0);
  if (lane == 0) {
    s_wcnt[warp] = __popc(lm);
    if (wv) atomicAdd(&s_vis, wv);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kPreBlock / 32; ++w) {
      const uint32_t c = s_wcnt[w];
      s_wcnt[w] = tot;
      tot += c;
    }
    s_base = tot ? atomicAdd(&out.header->n_glist, tot) : 0u;
    if (s_vis) atomicAdd(&out.header->n_visible, s_vis);
  }
  for (int v = threadIdx.x; v < nviews; v += kPreBlock)
    if (s_pairs[v]) atomicAdd(&out.header->view_pairs[v], s_pairs[v]);
  __syncthreads();
  if (nvis > 0) out.glist[s_base + s_wcnt[warp] + __popc(lm & ((1u << lane) - 1u))] = static_cast<uint32_t>(i);
}

template <typename S, bool A, bool B>
static void launch_pre_t(const r4g_gaussians& g, const ViewDev* views, int nviews, const PreOut& o, int nblocks,
                         int sh_degree, bool tc, cudaStream_t s) {
  preprocess_fwd_kernel<S, A, B><<<nblocks, kPreBlock, 0, s>>>(g, views, nviews, o, sh_degree, tc);
}

cudaError_t launch_preprocess_fwd(const r4g_gaussians& g, const FrameLayout& L, void* frame, int sh_degree,
                                  uint32_t flags, cudaStream_t s) {
  if (L.n == 0) return cudaSuccess;
  PreOut o;
  o.recA = at<float4>(frame, L.rec);
  o.rect = at<uint2>(frame, L.rect);
  o.touched = at<uint32_t>(frame, L.touched);
  o.dkey = at<uint32_t>(frame, L.dkey0);
  o.tdiff = at<uint32_t>(frame, L.tdiff);
  o.glist = at<uint32_t>(frame, L.glist);
  o.header = at<FrameHeader>(frame, L.header);
  o.tile_w = L.tile_w;
  o.tile_h = L.tile_h;
  const ViewDev* views = at<ViewDev>(frame, L.views);
  const bool tc = !(flags & R4G_FLAG_NO_TEMPORAL_CULL);
  const bool f64 = flags & R4G_FLAG_FP64_SLICE;
  const bool sb = g.scale_dtype == R4G_BF16, hb = g.sh_dtype == R4G_BF16;
  const int nb = static_cast<int>((L.n + kPreBlock - 1) / kPreBlock);
#define R4G_PF(S_, A_, B_) launch_pre_t<S_, A_, B_>(g, views, L.nviews, o, nb, sh_degree, tc, s)
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


// ---- backward ---------------------------------------------------------------
// Gradient of the rotor -> matrix map (appendix A.2): every entry of R is a
// quadratic form of the normalised rotor, so dR_e / dr is linear in r.
// Off-diagonal entries are 2 * sum of signed products r_a r_b.
template <typename S>
__device__ __forceinline__ void prod_term(S w, const S r[8], S g[8], int a, int b) {
  g[a] += w * r[b];
  g[b] += w * r[a];
}

template <typename S>
__device__ __forceinline__ void rotor_matrix_bwd(const S r[8], const S gR[16], S g[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) g[k] = S(0);
  // diagonal entries: sums of +-r_k^2; signs over (s, b01, b02, b12, b03, b13, b23, p)
  const int dsg[4][8] = {{1, -1, -1, 1, -1, 1, 1, -1},
                         {1, -1, 1, -1, 1, -1, 1, -1},
                         {1, 1, -1, -1, 1, 1, -1, -1},
                         {1, 1, 1, 1, -1, -1, -1, -1}};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const S w = S(2) * gR[5 * d];
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] += dsg[d][k] > 0 ? w * r[k] : -w * r[k];
  }
  // indices: s 0, b01 1, b02 2, b12 3, b03 4, b13 5, b23 6, p 7
  S w;
  w = S(2) * gR[1];   // R01 = 2(b01 s - b02 b12 - b03 b13 + b23 p)
  prod_term(w, r, g, 1, 0); prod_term(-w, r, g, 2, 3); prod_term(-w, r, g, 4, 5); prod_term(w, r, g, 6, 7);
  w = S(2) * gR[2];   // R02 = 2(b01 b12 + b02 s - b03 b23 - b13 p)
  prod_term(w, r, g, 1, 3); prod_term(w, r, g, 2, 0); prod_term(-w, r, g, 4, 6); prod_term(-w, r, g, 5, 7);
  w = S(2) * gR[3];   // R03 = 2(b01 b13 + b02 b23 + b03 s + b12 p)
  prod_term(w, r, g, 1, 5); prod_term(w, r, g, 2, 6); prod_term(w, r, g, 4, 0); prod_term(w, r, g, 3, 7);
  w = S(2) * gR[4];   // R10 = 2(-b01 s - b02 b12 - b03 b13 - b23 p)
  prod_term(-w, r, g, 1, 0); prod_term(-w, r, g, 2, 3); prod_term(-w, r, g, 4, 5); prod_term(-w, r, g, 6, 7);
  w = S(2) * gR[6];   // R12 = 2(-b01 b02 + b03 p + b12 s - b13 b23)
  prod_term(-w, r, g, 1, 2); prod_term(w, r, g, 4, 7); prod_term(w, r, g, 3, 0); prod_term(-w, r, g, 5, 6);
  w = S(2) * gR[7];   // R13 = 2(-b01 b03 - b02 p + b12 b23 + b13 s)
  prod_term(-w, r, g, 1, 4); prod_term(-w, r, g, 2, 7); prod_term(w, r, g, 3, 6); prod_term(w, r, g, 5, 0);
  w = S(2) * gR[8];   // R20 = 2(b01 b12 - b02 s - b03 b23 + b13 p)
  prod_term(w, r, g, 1, 3); prod_term(-w, r, g, 2, 0); prod_term(-w, r, g, 4, 6); prod_term(w, r, g, 5, 7);
  w = S(2) * gR[9];   // R21 = 2(-b01 b02 - b03 p - b12 s - b13 b23)
  prod_term(-w, r, g, 1, 2); prod_term(-w, r, g, 4, 7); prod_term(-w, r, g, 3, 0); prod_term(-w, r, g, 5, 6);
  w = S(2) * gR[11];  // R23 = 2(b01 p - b02 b03 - b12 b13 + b23 s)
  prod_term(w, r, g, 1, 7); prod_term(-w, r, g, 2, 4); prod_term(-w, r, g, 3, 5); prod_term(w, r, g, 6, 0);
  w = S(2) * gR[12];  // R30 = 2(b01 b13 + b02 b23 - b03 s - b12 p)
  prod_term(w, r, g, 1, 5); prod_term(w, r, g, 2, 6); prod_term(-w, r, g, 4, 0); prod_term(-w, r, g, 3, 7);
  w = S(2) * gR[13];  // R31 = 2(-b01 b03 + b02 p + b12 b23 - b13 s)
  prod_term(-w, r, g, 1, 4); prod_term(w, r, g, 2, 7); prod_term(w, r, g, 3, 6); prod_term(-w, r, g, 5, 0);
  w = S(2) * gR[14];  // R32 = 2(-b01 p - b02 b03 - b12 b13 - b23 s)
  prod_term(-w, r, g, 1, 7); prod_term(-w, r, g, 2, 4); prod_term(-w, r, g, 3, 5); prod_term(-w, r, g, 6, 0);
}

// Gradient of F_norm (appendix A.1): r1 = r + delta(r) P r with P r = grad eps
// (P symmetric, P^2 = I), r_hat = r1 / |r1|; delta depends on eps and l^2.
template <typename S>
__device__ __forceinline__ void rotor_normalize_bwd(const float rin[8], const RotorNorm<S>& rn,
                                                    const S gh[8], S gr[8]) {
  if (rn.ident) {
#pragma unroll
    for (int k = 0; k < 8; ++k) gr[k] = S(0);
    return;
  }
  const S invn = S(1) / sqrt(rn.n2);
  S dot = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) dot += rn.r[k] * gh[k];
  S g1[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) g1[k] = (gh[k] - rn.r[k] * dot) * invn;
  S r[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) r[k] = static_cast<S>(rin[k]);
  S Pr[8], Pg[8];
  eps_grad(r, Pr);
  eps_grad(g1, Pg);
  S gdot = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) gdot += g1[k] * Pr[k];
  S dd_de = 0, dd_dl2 = 0;
  if (rn.l2 > S(0)) {
    S disc = rn.l2 * rn.l2 - S(4) * rn.eps * rn.eps;
    disc = disc > S(0) ? disc : S(0);
    const S sq = sqrt(disc);
    const S D = rn.l2 + sq;
    dd_de = S(-2) / D;
    dd_dl2 = S(2) * rn.eps / (D * D);
    if (sq > S(0)) {
      dd_de -= S(8) * rn.eps * rn.eps / (D * D * sq);
      dd_dl2 *= S(1) + rn.l2 / sq;
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k)
    gr[k] = g1[k] + rn.delta * Pg[k] + gdot * (dd_de * Pr[k] + dd_dl2 * S(2) * r[k]);
}

constexpr int kBwdBlock = 128;

// Gradient sums over the views of one Gaussian, in the slice precision S.
template <typename S>
struct BwdAcc {
  S G4[10];   // symmetric d Sigma4, upper triangle (xx xy xz xt yy yz yt zz zt tt)
  S gmean[4];
  S gop;      // d opacity
};

// One view's part of the backward of one Gaussian: from the summed per-pair
// gradients (ga = d mean2d.x, d mean2d.y, d conic a, d conic b; gb.x = d conic
// c, gb.y = d opacity_t; gc = d rgb) through the colour, the conic, the EWA
// projection and the temporal slice, down to d Sigma4, d mean and d opacity
// (accumulated in acc) and d SH (added to the SH gradient row).
template <typename S, bool kShBF16>
__device__ __forceinline__ void view_backward(const r4g_gaussians& g, int i, const Sig4<S>& G, const CamDev& cam,
                                              float t, int sh_degree, bool temporal_cull, float4 ga, float4 gb,
                                              float4 gc, float* __restrict__ gsh, BwdAcc<S>& acc) {
  Fwd f;
  S invW, dt;
  view_geometry<S>(G, cam, t, temporal_cull, f, invW, dt);
  float shc[16][3], Y[16];
  forward_color<kShBF16>(g, i, cam, sh_degree, f, shc, Y);

  // ---- colour: rgb = max(0, sum_k Y_k(dir) c_k + 0.5)
  const float grgb[3] = {f.rgb_pos[0] ? gc.x : 0.f, f.rgb_pos[1] ? gc.y : 0.f, f.rgb_pos[2] ? gc.z : 0.f};
  const int nb = (sh_degree + 1) * (sh_degree + 1);
  float wk[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) wk[k] = shc[k][0] * grgb[0] + shc[k][1] * grgb[1] + shc[k][2] * grgb[2];
  {
    // d c_k = Y_k d rgb, accumulated as 16-byte vectors over the 48-float row
    float4* gsh4 = reinterpret_cast<float4*>(gsh + static_cast<size_t>(i) * 48);
    const int nvec = (nb * 3 + 3) / 4;
#pragma unroll
    for (int v = 0; v < 12; ++v) {
      if (v < nvec) {
        float4 a = gsh4[v];
        float* ap = reinterpret_cast<float*>(&a);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int e = 4 * v + h;
          if (e < nb * 3) ap[h] += Y[e / 3] * grgb[e % 3];
        }
        gsh4[v] = a;
      }
    }
  }
  float gmu[3];
  {
    const float x = f.dir[0], y = f.dir[1], z = f.dir[2];
    const float xx = x * x, yy = y * y, zz = z * z;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    // d Y_k / d(x, y, z) of the degree-3 polynomials
    gy += wk[1] * -kY1;
    gz += wk[2] * kY1;
    gx += wk[3] * -kY1;
    gx += wk[4] * kY2a * y;                 gy += wk[4] * kY2a * x;
    gy += wk[5] * -kY2a * z;                gz += wk[5] * -kY2a * y;
    gx += wk[6] * -2.f * kY2b * x;          gy += wk[6] * -2.f * kY2b * y;  gz += wk[6] * 4.f * kY2b * z;
    gx += wk[7] * -kY2a * z;                gz += wk[7] * -kY2a * x;
    gx += wk[8] * 2.f * kY2c * x;           gy += wk[8] * -2.f * kY2c * y;
    gx += wk[9] * -6.f * kY3a * x * y;      gy += wk[9] * -3.f * kY3a * (xx - yy);
    gx += wk[10] * kY3b * y * z;            gy += wk[10] * kY3b * x * z;    gz += wk[10] * kY3b * x * y;
    gx += wk[11] * 2.f * kY3c * x * y;      gy += wk[11] * -kY3c * (4.f * zz - xx - 3.f * yy);
    gz += wk[11] * -8.f * kY3c * y * z;
    gx += wk[12] * -6.f * kY3d * x * z;     gy += wk[12] * -6.f * kY3d * y * z;
    gz += wk[12] * kY3d * (6.f * zz - 3.f * xx - 3.f * yy);
    gx += wk[13] * -kY3c * (4.f * zz - 3.f * xx - yy);  gy += wk[13] * 2.f * kY3c * x * y;
    gz += wk[13] * -8.f * kY3c * x * z;
    gx += wk[14] * 2.f * kY3e * x * z;      gy += wk[14] * -2.f * kY3e * y * z;  gz += wk[14] * kY3e * (xx - yy);
    gx += wk[15] * -3.f * kY3a * (xx - yy); gy += wk[15] * 6.f * kY3a * x * y;
    // dir = v / |v|
    const float dd = x * gx + y * gy + z * gz;
    const float idist = 1.0f / f.dist;
    gmu[0] = (gx - x * dd) * idist;
    gmu[1] = (gy - y * dd) * idist;
    gmu[2] = (gz - z * dd) * idist;
  }

  // ---- conic = inverse of the dilated 2D covariance (A, B; B, C)
  const float A = f.cov[0], B = f.cov[1], Cc = f.cov[2];
  const float det = A * Cc - B * B;
  const float idet = 1.0f / det, id2 = idet * idet;
  const float gA = ga.z * (-Cc * Cc * id2) + ga.w * (B * Cc * id2) + gb.x * (idet - A * Cc * id2);
  const float gB = ga.z * (2.f * B * Cc * id2) + ga.w * (-idet - 2.f * B * B * id2) + gb.x * (2.f * A * B * id2);
  const float gC = ga.z * (idet - Cc * A * id2) + ga.w * (B * A * id2) + gb.x * (-A * A * id2);
  const float P00 = gA, P01 = 0.5f * gB, P11 = gC;  // symmetric gradient of Sigma'

  // ---- Sigma' = T Sigma3 T^T + 0.3 I with T = J Rc
  const float* Rc = cam.R;
  const float x = f.pc[0], y = f.pc[1], z = f.pc[2];
  const float iz = 1.0f / z, iz2 = iz * iz;
  const float rx = x * iz, ry = y * iz;
  const float crx = fminf(fmaxf(rx, -cam.limx), cam.limx);
  const float cry = fminf(fmaxf(ry, -cam.limy), cam.limy);
  const float j00 = cam.fx * iz, j02 = -cam.fx * crx * iz;
  const float j11 = cam.fy * iz, j12 = -cam.fy * cry * iz;
  const float T0[3] = {j00 * Rc[0] + j02 * Rc[6], j00 * Rc[1] + j02 * Rc[7], j00 * Rc[2] + j02 * Rc[8]};
  const float T1[3] = {j11 * Rc[3] + j12 * Rc[6], j11 * Rc[4] + j12 * Rc[7], j11 * Rc[5] + j12 * Rc[8]};
  const float* s3 = f.sig3;
  const float ST0[3] = {s3[0] * T0[0] + s3[1] * T0[1] + s3[2] * T0[2],
                        s3[1] * T0[0] + s3[3] * T0[1] + s3[4] * T0[2],
                        s3[2] * T0[0] + s3[4] * T0[1] + s3[5] * T0[2]};
  const float ST1[3] = {s3[0] * T1[0] + s3[1] * T1[1] + s3[2] * T1[2],
                        s3[1] * T1[0] + s3[3] * T1[1] + s3[4] * T1[2],
                        s3[2] * T1[0] + s3[4] * T1[1] + s3[5] * T1[2]};
  // d Sigma3 (symmetric, all nine entries) = T^T P T
  float GS[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      GS[a][b] = T0[a] * (P00 * T0[b] + P01 * T1[b]) + T1[a] * (P01 * T0[b] + P11 * T1[b]);
  // d T = 2 P T Sigma3
  float gT0[3], gT1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gT0[a] = 2.f * (P00 * ST0[a] + P01 * ST1[a]);
    gT1[a] = 2.f * (P01 * ST0[a] + P11 * ST1[a]);
  }
  const float gj00 = gT0[0] * Rc[0] + gT0[1] * Rc[1] + gT0[2] * Rc[2];
  const float gj02 = gT0[0] * Rc[6] + gT0[1] * Rc[7] + gT0[2] * Rc[8];
  const float gj11 = gT1[0] * Rc[3] + gT1[1] * Rc[4] + gT1[2] * Rc[5];
  const float gj12 = gT1[0] * Rc[6] + gT1[1] * Rc[7] + gT1[2] * Rc[8];
  const float dj02_dx = f.clampx ? 0.f : -cam.fx * iz2;
  const float dj02_dz = cam.fx * crx * iz2 + (f.clampx ? 0.f : cam.fx * x * iz2 * iz);
  const float dj12_dy = f.clampy ? 0.f : -cam.fy * iz2;
  const float dj12_dz = cam.fy * cry * iz2 + (f.clampy ? 0.f : cam.fy * y * iz2 * iz);
  const float gpx = gj02 * dj02_dx + ga.x * cam.fx * iz;
  const float gpy = gj12 * dj12_dy + ga.y * cam.fy * iz;
  const float gpz = gj00 * (-cam.fx * iz2) + gj02 * dj02_dz + gj11 * (-cam.fy * iz2) + gj12 * dj12_dz -
                    ga.x * cam.fx * x * iz2 - ga.y * cam.fy * y * iz2;
  gmu[0] += Rc[0] * gpx + Rc[3] * gpy + Rc[6] * gpz;
  gmu[1] += Rc[1] * gpx + Rc[4] * gpy + Rc[7] * gpz;
  gmu[2] += Rc[2] * gpx + Rc[5] * gpy + Rc[8] * gpz;

  // ---- temporal slice (slice precision S)
  const S* C = G.C;
  const S V[3] = {C[3], C[6], C[8]};
  const S got = static_cast<S>(gb.y);
  const S g_o = got * static_cast<S>(f.temporal);
  const S g_lam = S(-0.5) * got * static_cast<S>(f.o_t);
  S gV[3], gmxyz[3];
  S gdt = 0, ginvW = 0;
  const S mv = dt * invW;
  S gmuV = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gmxyz[a] = static_cast<S>(gmu[a]);
    gV[a] = mv * gmxyz[a];
    gmuV += gmxyz[a] * V[a];
  }
  gdt += invW * gmuV;
  ginvW += dt * gmuV;
  S GSV[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    GSV[a] = static_cast<S>(GS[a][0]) * V[0] + static_cast<S>(GS[a][1]) * V[1] + static_cast<S>(GS[a][2]) * V[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) gV[a] -= S(2) * invW * GSV[a];
  ginvW -= V[0] * GSV[0] + V[1] * GSV[1] + V[2] * GSV[2];
  gdt += S(2) * dt * invW * g_lam;
  ginvW += dt * dt * g_lam;
  const S gW = -invW * invW * ginvW;
  acc.G4[0] += static_cast<S>(GS[0][0]);
  acc.G4[1] += static_cast<S>(GS[0][1]);
  acc.G4[2] += static_cast<S>(GS[0][2]);
  acc.G4[3] += S(0.5) * gV[0];
  acc.G4[4] += static_cast<S>(GS[1][1]);
  acc.G4[5] += static_cast<S>(GS[1][2]);
  acc.G4[6] += S(0.5) * gV[1];
  acc.G4[7] += static_cast<S>(GS[2][2]);
  acc.G4[8] += S(0.5) * gV[2];
  acc.G4[9] += gW;
  acc.gmean[0] += gmxyz[0];
  acc.gmean[1] += gmxyz[1];
  acc.gmean[2] += gmxyz[2];
  acc.gmean[3] -= gdt;
  acc.gop += g_o;
}

// Backward of the preprocess over the Gaussians visible in some view (the
// list the forward built). For each view, each warp first sums, for each of
// its 32 Gaussians in turn, the per-pair gradients the blend backward wrote
// (an item's pairs are contiguous, [ioffs[item], ioffs[item] + touched[item])),
// reading them coalesced; then every thread runs its Gaussian's view
// backward. After the views, the Sigma4 -> R -> rotor and scale backward runs
// once per Gaussian and the gradients are added to the caller's buffers.
// Every Gaussian is one thread's: the gradient is deterministic.
template <typename S, bool kScaleBF16, bool kShBF16>
__global__ void __launch_bounds__(kBwdBlock, 3)
    preprocess_bwd_kernel(r4g_gaussians g, const ViewDev* __restrict__ views, int nviews,
                          const uint32_t* __restrict__ glist, const uint32_t* __restrict__ ioffs,
                          const uint32_t* __restrict__ touched, const float4* __restrict__ gbuf,
                          const FrameHeader* hdr, int sh_degree, bool temporal_cull, r4g_grads out) {
  const int j = blockIdx.x * kBwdBlock + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int nlist = static_cast<int>(hdr->n_glist);
  if ((hdr->status & 1u) || (j - lane) >= nlist) return;  // warp-uniform (overflowed frame: no gradient)
  const bool mine = j < nlist;
  const int i = mine ? static_cast<int>(glist[j]) : 0;
  Sig4<S> Q;
  if (mine) gauss_sigma<S, kScaleBF16>(g, i, Q);
  BwdAcc<S> acc;
#pragma unroll
  for (int k = 0; k < 10; ++k) acc.G4[k] = S(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) acc.gmean[k] = S(0);
  acc.gop = S(0);
  for (int v = 0; v < nviews; ++v) {
    const size_t item = static_cast<size_t>(v) * g.n + i;
    const uint32_t cnt = mine ? touched[item] : 0u;
    if (__ballot_sync(0xffffffffu, cnt != 0u) == 0u) continue;
    const uint32_t o = cnt ? ioffs[item] : 0u;
    // warp-cooperative gather of the pair gradients: lane l adds pairs l, l+32, ...
    float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga, gc = ga;
    for (int q = 0; q < 32; ++q) {
      const uint32_t qc = __shfl_sync(0xffffffffu, cnt, q);
      if (qc < 2) continue;  // warp-uniform; a single pair is read by its owner below
      const uint32_t qo = __shfl_sync(0xffffffffu, o, q);
      float v9[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (uint32_t k = lane; k < qc; k += 32) {
        const float4* pr = gbuf + 3 * static_cast<size_t>(qo + k);
        const float4 x = pr[0], y = pr[1], z = pr[2];
        v9[0] += x.x; v9[1] += x.y; v9[2] += x.z; v9[3] += x.w;
        v9[4] += y.x; v9[5] += y.y;
        v9[6] += z.x; v9[7] += z.y; v9[8] += z.z;
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) {
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) v9[k] += __shfl_xor_sync(0xffffffffu, v9[k], sh);
      }
      if (lane == q) {
        ga = make_float4(v9[0], v9[1], v9[2], v9[3]);
        gb = make_float4(v9[4], v9[5], 0.f, 0.f);
        gc = make_float4(v9[6], v9[7], v9[8], 0.f);
      }
    }
    if (cnt == 1) {
      const float4* pr = gbuf + 3 * static_cast<size_t>(o);
      ga = pr[0];
      gb = pr[1];
      gc = pr[2];
    }
    if (cnt) view_backward<S, kShBF16>(g, i, Q, views[v].cam, views[v].t, sh_degree, temporal_cull, ga, gb, gc,
                                       out.sh, acc);
  }
  if (!mine) return;
  Geo<S> G;  // the rotor and scale intermediates, recomputed rather than kept through the views
  gauss_setup<S, kScaleBF16>(g, i, G);
  // symmetric gradient of Sigma4
  S G4[4][4];
  G4[0][0] = acc.G4[0]; G4[0][1] = G4[1][0] = acc.G4[1]; G4[0][2] = G4[2][0] = acc.G4[2];
  G4[0][3] = G4[3][0] = acc.G4[3]; G4[1][1] = acc.G4[4]; G4[1][2] = G4[2][1] = acc.G4[5];
  G4[1][3] = G4[3][1] = acc.G4[6]; G4[2][2] = acc.G4[7]; G4[2][3] = G4[3][2] = acc.G4[8];
  G4[3][3] = acc.G4[9];
  // ---- Sigma4 = R diag(sc2) R^T
  const S* R = G.R;
  S gR[16], gsc2[4];
  S G4R[4][4];  // G4 R
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      G4R[a][k] = G4[a][0] * R[k] + G4[a][1] * R[4 + k] + G4[a][2] * R[8 + k] + G4[a][3] * R[12 + k];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 4; ++k) gR[4 * a + k] = S(2) * G4R[a][k] * G.sc2[k];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    gsc2[k] = R[k] * G4R[0][k] + R[4 + k] * G4R[1][k] + R[8 + k] * G4R[2][k] + R[12 + k] * G4R[3][k];
  // ---- rotor
  S grh[8], grot[8];
  rotor_matrix_bwd<S>(G.rn.r, gR, grh);
  rotor_normalize_bwd<S>(G.p.rot, G.rn, grh, grot);

  // ---- write (accumulate)
  // accumulate (+=) with 16-byte vector accesses
  float4* gm = reinterpret_cast<float4*>(out.mean) + i;
  float4 vm = *gm;
  vm.x += static_cast<float>(acc.gmean[0]);
  vm.y += static_cast<float>(acc.gmean[1]);
  vm.z += static_cast<float>(acc.gmean[2]);
  vm.w += static_cast<float>(acc.gmean[3]);
  *gm = vm;
  float4* gr = reinterpret_cast<float4*>(out.rotor) + 2 * static_cast<size_t>(i);
  float4 r0 = gr[0], r1 = gr[1];
  r0.x += static_cast<float>(grot[0]); r0.y += static_cast<float>(grot[1]);
  r0.z += static_cast<float>(grot[2]); r0.w += static_cast<float>(grot[3]);
  r1.x += static_cast<float>(grot[4]); r1.y += static_cast<float>(grot[5]);
  r1.z += static_cast<float>(grot[6]); r1.w += static_cast<float>(grot[7]);
  gr[0] = r0;
  gr[1] = r1;
  float4* gl = reinterpret_cast<float4*>(out.logscale) + i;
  float4 vl = *gl;
  vl.x += static_cast<float>(gsc2[0] * S(2) * G.sc2[0]);
  vl.y += static_cast<float>(gsc2[1] * S(2) * G.sc2[1]);
  vl.z += static_cast<float>(gsc2[2] * S(2) * G.sc2[2]);
  vl.w += static_cast<float>(gsc2[3] * S(2) * G.sc2[3]);
  *gl = vl;
  out.logit[i] += static_cast<float>(acc.gop) * G.opacity * (1.0f - G.opacity);
}

template <typename S, bool A, bool B>
static void launch_pre_bwd_t(const r4g_gaussians& g, const FrameLayout& L, void* frame, int sh_degree, bool tc,
                             const r4g_grads& out, cudaStream_t s) {
  const int nb = static_cast<int>((L.n + kBwdBlock - 1) / kBwdBlock);
  preprocess_bwd_kernel<S, A, B><<<nb, kBwdBlock, 0, s>>>(
      g, at<ViewDev>(frame, L.views), L.nviews, at<uint32_t>(frame, L.glist), at<uint32_t>(frame, L.ioffs),
      at<uint32_t>(frame, L.touched), at<float4>(frame, L.gbuf), at<FrameHeader>(frame, L.header), sh_degree, tc,
      out);
}

cudaError_t launch_preprocess_bwd(const r4g_gaussians& g, const FrameLayout& L, void* frame, int sh_degree,
                                  uint32_t flags, r4g_grads grads, cudaStream_t s) {
  if (L.n == 0) return cudaSuccess;
  const bool tc = !(flags & R4G_FLAG_NO_TEMPORAL_CULL);
  const bool f64 = flags & R4G_FLAG_FP64_SLICE;
  const bool sb = g.scale_dtype == R4G_BF16, hb = g.sh_dtype == R4G_BF16;
#define R4G_PB(S_, A_, B_) launch_pre_bwd_t<S_, A_, B_>(g, L, frame, sh_degree, tc, grads, s)
  if (f64) {
    if (sb && hb) R4G_PB(double, true, true);
    else if (sb) R4G_PB(double, true, false);
    else if (hb) R4G_PB(double, false, true);
    else R4G_PB(double, false, false);
  } else {
    if (sb && hb) R4G_PB(float, true, true);
    else if (sb) R4G_PB(float, true, false);
    else if (hb) R4G_PB(float, false, true);
    else R4G_PB(float, false, false);
  }
#undef R4G_PB
  return cudaGetLastError();
}

}  // namespace r4g
