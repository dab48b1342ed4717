// Per-Gaussian preprocess of the render (forward): activations, rotor
// normalisation and rotation (appendix A.1/A.2), Sigma4 (Sec. 3.2.1), the
// temporal slice and visibility cull (Sec. 3.2.2, appendix A.3), EWA
// projection (Sec. 3.1), SH colour, and the tile rectangle each Gaussian's
// contributing pixels can lie in. One thread per Gaussian; coalesced 16-byte
// loads of the SoA parameters; the SH row is read only for survivors.
#include <cuda_runtime.h>

#include "r4g_internal.cuh"
#include "r4g_math.cuh"

namespace r4g {

struct PreOut {
  float4* recA;  // (mean2d.x, mean2d.y, conic a, conic b)
  float4* recB;  // (conic c, opacity_t, depth, 0)
  float4* recC;  // (r, g, b, 0)
  uint2* rect;   // tile rect: (x0 | y0 << 16, x1 | y1 << 16), [x0, x1) x [y0, y1)
  uint32_t* touched;
  uint32_t* dkey;  // float bits of the depth for Gaussians with tiles, else 0xffffffff
  uint32_t* tdiff; // 2D difference array of the tile counts, (tiles_y + 1) x (tiles_x + 1)
  uint32_t* blocksum;
  FrameHeader* header;
  int tile_w, tile_h, tiles_x, tiles_y;
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

// Intermediates of the rotor / Sigma4 / slice steps in the slice precision S,
// kept for the backward.
template <typename S>
struct Geo {
  Params p;
  RotorNorm<S> rn;
  S R[16];
  S sc2[4];
  S C[10];
  S invW, dt;
};

template <typename S, bool kScaleBF16>
__device__ __forceinline__ void forward_geometry(const r4g_gaussians& g, int i, const CamDev& cam,
                                                 float t, bool temporal_cull, Fwd& f,
                                                 Geo<S>* keep = nullptr) {
  Params p;
  load_params<kScaleBF16>(g, i, p);
  S sc2[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float s = expf(p.ls[k]);
    sc2[k] = static_cast<S>(s) * static_cast<S>(s);
  }
  f.opacity = 1.0f / (1.0f + expf(-p.logit));
  RotorNorm<S> rn;
  rotor_normalize<S>(p.rot, rn);
  S R[16];
  rotor_matrix<S>(rn.r, R);
  S C[10];
  cov4<S>(R, sc2, C);
  // Sigma4 = [[U, V], [V^T, W]]: U = C[0,1,2; 1,4,5; 2,5,7], V = (C3, C6, C8), W = C9
  const S W = C[9];
  const S invW = S(1) / W;
  const S dt = static_cast<S>(t) - static_cast<S>(p.mean[3]);
  const S lam_dt2 = dt * dt * invW;
  const S V0 = C[3], V1 = C[6], V2 = C[8];
  const S mv = dt * invW;
  f.mu3[0] = static_cast<float>(static_cast<S>(p.mean[0]) + mv * V0);
  f.mu3[1] = static_cast<float>(static_cast<S>(p.mean[1]) + mv * V1);
  f.mu3[2] = static_cast<float>(static_cast<S>(p.mean[2]) + mv * V2);
  f.sig3[0] = static_cast<float>(C[0] - V0 * V0 * invW);
  f.sig3[1] = static_cast<float>(C[1] - V0 * V1 * invW);
  f.sig3[2] = static_cast<float>(C[2] - V0 * V2 * invW);
  f.sig3[3] = static_cast<float>(C[4] - V1 * V1 * invW);
  f.sig3[4] = static_cast<float>(C[5] - V1 * V2 * invW);
  f.sig3[5] = static_cast<float>(C[7] - V2 * V2 * invW);
  if (keep) {
    keep->p = p;
    keep->rn = rn;
#pragma unroll
    for (int k = 0; k < 16; ++k) keep->R[k] = R[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) keep->sc2[k] = sc2[k];
#pragma unroll
    for (int k = 0; k < 10; ++k) keep->C[k] = C[k];
    keep->invW = invW;
    keep->dt = dt;
  }
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

template <typename S, bool kScaleBF16, bool kShBF16>
__global__ void __launch_bounds__(kPreBlock)
    preprocess_fwd_kernel(r4g_gaussians g, CamDev cam, float t, PreOut out, int sh_degree,
                          bool temporal_cull) {
  const int i = blockIdx.x * kPreBlock + threadIdx.x;
  uint32_t ntiles = 0;
  if (i < g.n) {
    Fwd f;
    forward_geometry<S, kScaleBF16>(g, i, cam, t, temporal_cull, f);
    int i0 = 0, i1 = -1, j0 = 0, j1 = -1;
    bool vis = f.visible && pixel_box(f, cam, i0, i1, j0, j1);
    if (vis) {
      forward_color<kShBF16>(g, i, cam, sh_degree, f);
      const int x0 = i0 / out.tile_w, x1 = i1 / out.tile_w + 1;
      const int y0 = j0 / out.tile_h, y1 = j1 / out.tile_h + 1;
      ntiles = static_cast<uint32_t>((x1 - x0) * (y1 - y0));
      out.recA[i] = make_float4(f.mean2d[0], f.mean2d[1], f.conic[0], f.conic[1]);
      out.recB[i] = make_float4(f.conic[2], f.o_t, f.pc[2], 0.0f);
      out.recC[i] = make_float4(f.rgb[0], f.rgb[1], f.rgb[2], 0.0f);
      out.rect[i] = make_uint2(static_cast<uint32_t>(x0) | (static_cast<uint32_t>(y0) << 16),
                               static_cast<uint32_t>(x1) | (static_cast<uint32_t>(y1) << 16));
      // +1 on every tile of the rectangle, as four corner updates
      const int st = out.tiles_x + 1;
      atomicAdd(out.tdiff + y0 * st + x0, 1u);
      atomicAdd(out.tdiff + y0 * st + x1, 0xffffffffu);
      atomicAdd(out.tdiff + y1 * st + x0, 0xffffffffu);
      atomicAdd(out.tdiff + y1 * st + x1, 1u);
    } else {
      out.recA[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      out.recB[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      out.recC[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      out.rect[i] = make_uint2(0u, 0u);
    }
    out.touched[i] = ntiles;
    out.dkey[i] = ntiles ? __float_as_uint(f.pc[2]) : 0xffffffffu;
  }
  // per-block totals of the tile counts and of the visible Gaussians
  __shared__ uint32_t s_sum[kPreBlock / 32], s_vis[kPreBlock / 32];
  const uint32_t ws = __reduce_add_sync(0xffffffffu, ntiles);
  const uint32_t wv = __reduce_add_sync(0xffffffffu, ntiles > 0 ? 1u : 0u);
  if ((threadIdx.x & 31) == 0) {
    s_sum[threadIdx.x >> 5] = ws;
    s_vis[threadIdx.x >> 5] = wv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0, b = 0;
#pragma unroll
    for (int w = 0; w < kPreBlock / 32; ++w) {
      a += s_sum[w];
      b += s_vis[w];
    }
    out.blocksum[blockIdx.x] = a;
    if (b) atomicAdd(&out.header->n_visible, b);
  }
}

template <typename S, bool A, bool B>
static void launch_pre_t(const r4g_gaussians& g, const CamDev& cam, float t, const PreOut& o,
                         int nblocks, int sh_degree, bool tc, cudaStream_t s) {
  preprocess_fwd_kernel<S, A, B><<<nblocks, kPreBlock, 0, s>>>(g, cam, t, o, sh_degree, tc);
}

cudaError_t launch_preprocess_fwd(const r4g_gaussians& g, const CamDev& cam, float t,
                                  const FrameLayout& L, void* frame, int sh_degree,
                                  uint32_t flags, cudaStream_t s) {
  if (L.n == 0) return cudaSuccess;
  PreOut o;
  o.recA = at<float4>(frame, L.rec);
  o.recB = o.recA + L.n;
  o.recC = o.recB + L.n;
  o.rect = at<uint2>(frame, L.rect);
  o.touched = at<uint32_t>(frame, L.touched);
  o.dkey = at<uint32_t>(frame, L.dkey0);
  o.tdiff = at<uint32_t>(frame, L.tdiff);
  o.blocksum = at<uint32_t>(frame, L.blocksum);
  o.header = at<FrameHeader>(frame, L.header);
  o.tile_w = L.tile_w; o.tile_h = L.tile_h; o.tiles_x = L.tiles_x; o.tiles_y = L.tiles_y;
  const bool tc = !(flags & R4G_FLAG_NO_TEMPORAL_CULL);
  const bool f64 = flags & R4G_FLAG_FP64_SLICE;
  const bool sb = g.scale_dtype == R4G_BF16, hb = g.sh_dtype == R4G_BF16;
  const int nb = L.nblocks;
  if (f64) {
    if (sb && hb) launch_pre_t<double, true, true>(g, cam, t, o, nb, sh_degree, tc, s);
    else if (sb) launch_pre_t<double, true, false>(g, cam, t, o, nb, sh_degree, tc, s);
    else if (hb) launch_pre_t<double, false, true>(g, cam, t, o, nb, sh_degree, tc, s);
    else launch_pre_t<double, false, false>(g, cam, t, o, nb, sh_degree, tc, s);
  } else {
    if (sb && hb) launch_pre_t<float, true, true>(g, cam, t, o, nb, sh_degree, tc, s);
    else if (sb) launch_pre_t<float, true, false>(g, cam, t, o, nb, sh_degree, tc, s);
    else if (hb) launch_pre_t<float, false, true>(g, cam, t, o, nb, sh_degree, tc, s);
    else launch_pre_t<float, false, false>(g, cam, t, o, nb, sh_degree, tc, s);
  }
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

// The backward runs over the depth order, whose first n_visible entries are
// the Gaussians with tiles, so every warp is full. Each warp first sums, for
// each of its 32 Gaussians in turn, the per-pair gradients the blend
// backward wrote (a Gaussian's pairs are contiguous, [offs[j], offs[j] + cnt)),
// reading them coalesced; then every thread runs its Gaussian's chain rule.
template <typename S, bool kScaleBF16, bool kShBF16>
__global__ void __launch_bounds__(kBwdBlock, 4)
    preprocess_bwd_kernel(r4g_gaussians g, CamDev cam, float t, const uint32_t* __restrict__ order,
                          const uint32_t* __restrict__ offs, const uint32_t* __restrict__ touched,
                          const float4* __restrict__ gbuf, const FrameHeader* hdr, int sh_degree,
                          bool temporal_cull, r4g_grads out) {
  const int j = blockIdx.x * kBwdBlock + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int nvis = static_cast<int>(hdr->n_visible);
  if ((hdr->status & 1u) || (j - lane) >= nvis) return;  // warp-uniform (overflowed frame: no gradient)
  const bool mine = j < nvis;
  const uint32_t gi = mine ? order[j] : 0u;
  const uint32_t o = mine ? offs[j] : 0u;
  const uint32_t cnt = mine ? touched[gi] : 0u;
  // warp-cooperative gather of the pair gradients: lane l adds pairs l, l+32, ...
  float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga, gc = ga;
  for (int q = 0; q < 32; ++q) {
    const uint32_t qc = __shfl_sync(0xffffffffu, cnt, q);
    if (qc < 2) continue;  // warp-uniform; a single pair is read by its owner below
    const uint32_t qo = __shfl_sync(0xffffffffu, o, q);
    float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (uint32_t k = lane; k < qc; k += 32) {
      const float4* pr = gbuf + 3 * static_cast<size_t>(qo + k);
      const float4 x = pr[0], y = pr[1], z = pr[2];
      v[0] += x.x; v[1] += x.y; v[2] += x.z; v[3] += x.w;
      v[4] += y.x; v[5] += y.y;
      v[6] += z.x; v[7] += z.y; v[8] += z.z;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], sh);
    }
    if (lane == q) {
      ga = make_float4(v[0], v[1], v[2], v[3]);
      gb = make_float4(v[4], v[5], 0.f, 0.f);
      gc = make_float4(v[6], v[7], v[8], 0.f);
    }
  }
  if (cnt == 1) {
    const float4* pr = gbuf + 3 * static_cast<size_t>(o);
    ga = pr[0];
    gb = pr[1];
    gc = pr[2];
  }
  if (!mine) return;
  const int i = static_cast<int>(gi);
  Fwd f;
  Geo<S> G;
  forward_geometry<S, kScaleBF16>(g, i, cam, t, temporal_cull, f, &G);
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
    float4* gsh4 = reinterpret_cast<float4*>(out.sh + static_cast<size_t>(i) * 48);
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
  const S invW = G.invW, dt = G.dt;
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
  // symmetric gradient of Sigma4
  S G4[4][4];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) G4[a][b] = static_cast<S>(GS[a][b]);
    G4[a][3] = G4[3][a] = S(0.5) * gV[a];
  }
  G4[3][3] = gW;
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
  vm.x += static_cast<float>(gmxyz[0]);
  vm.y += static_cast<float>(gmxyz[1]);
  vm.z += static_cast<float>(gmxyz[2]);
  vm.w += static_cast<float>(-gdt);
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
  out.logit[i] += static_cast<float>(g_o) * f.opacity * (1.0f - f.opacity);
}

struct BwdIn {
  const uint32_t *order, *offs, *touched;
  const float4* gbuf;
  const FrameHeader* hdr;
};

template <typename S, bool A, bool B>
static void launch_pre_bwd_t(const r4g_gaussians& g, const CamDev& cam, float t, const BwdIn& in, int nblocks,
                             int sh_degree, bool tc, const r4g_grads& out, cudaStream_t s) {
  preprocess_bwd_kernel<S, A, B><<<nblocks, kBwdBlock, 0, s>>>(g, cam, t, in.order, in.offs, in.touched, in.gbuf,
                                                               in.hdr, sh_degree, tc, out);
}

cudaError_t launch_preprocess_bwd(const r4g_gaussians& g, const CamDev& cam, float t,
                                  const FrameLayout& L, void* frame, int sh_degree,
                                  uint32_t flags, r4g_grads grads, cudaStream_t s) {
  if (L.n == 0) return cudaSuccess;
  BwdIn in;
  in.order = at<uint32_t>(frame, L.order_in_1 ? L.ord1 : L.ord0);
  in.offs = at<uint32_t>(frame, L.offs);
  in.touched = at<uint32_t>(frame, L.touched);
  in.gbuf = at<float4>(frame, L.gbuf);
  in.hdr = at<FrameHeader>(frame, L.header);
  const bool tc = !(flags & R4G_FLAG_NO_TEMPORAL_CULL);
  const bool f64 = flags & R4G_FLAG_FP64_SLICE;
  const bool sb = g.scale_dtype == R4G_BF16, hb = g.sh_dtype == R4G_BF16;
  const int nb = static_cast<int>((L.n + kBwdBlock - 1) / kBwdBlock);
#define R4G_PB(S_, A_, B_) launch_pre_bwd_t<S_, A_, B_>(g, cam, t, in, nb, sh_degree, tc, grads, s)
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
