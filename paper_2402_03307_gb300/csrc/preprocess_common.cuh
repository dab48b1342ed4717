// Device helpers of the per-Gaussian preprocess shared by the forward
// (preprocess_fwd.cu) and the backward (preprocess.cu): activations, rotor
// normalisation and rotation (appendix A.1/A.2), Sigma4 (Sec. 3.2.1), the
// temporal slice and visibility cull (Sec. 3.2.2, appendix A.3), EWA
// projection (Sec. 3.1), SH colour, and the tile rectangle each Gaussian's
// contributing pixels can lie in.
#pragma once
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

}  // namespace r4g
