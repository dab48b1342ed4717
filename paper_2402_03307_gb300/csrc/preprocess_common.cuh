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
                 // (conic c, opacity_t, depth, log2(255 o_t)), (r, g, b, max(log2 o_t, -126))
  uint2* rect;   // tile rect: (x0 | y0 << 16, x1 | y1 << 16), [x0, x1) x [y0, y1)
  uint4* spans;  // [2 per item] the tile rows' column spans (tile_rows.cuh)
  uint32_t* touched;
  uint32_t* dkey;  // float bits of the depth for items with tiles, else 0xffffffff
  uint32_t* tdiff; // per view, per-row difference arrays of the tile counts, (tiles_y + 1) x (tiles_x + 1)
  uint32_t* glist; // Gaussians visible in some view
  FrameHeader* header;
  int tile_w, tile_h;
  int tws, ths;  // log2 of the tile width and height
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
    const float s = __expf(G.p.ls[k]);  // the hardware exponential: ~1e-7 relative
    G.sc2[k] = static_cast<S>(s) * static_cast<S>(s);
  }
  G.opacity = __fdividef(1.0f, 1.0f + __expf(-G.p.logit));  // 0 once exp(-logit) overflows
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
      if (k < nb) acc = fma_s(Y[k], c[k][ch], acc);
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

// Image-plane velocity of the sliced centre (Sec. 3.2.2: slicing adds
// (t - mu_t) V / W to the centre, so V / W is its speed): with
// p_c = (x, y, z) and p_c' = R_cw V / W,
//   d(mean2d)/dt = (fx (x' z - x z') / z^2, fy (y' z - y z') / z^2),
// stored in f.rgb as (du/dt, dv/dt, 0) so the blend composites it with the
// colour's weights.
template <typename S>
__device__ __forceinline__ void image_velocity(const Sig4<S>& Q, S invW, const CamDev& cam, Fwd& f) {
  const float v0 = static_cast<float>(Q.C[3] * invW);
  const float v1 = static_cast<float>(Q.C[6] * invW);
  const float v2 = static_cast<float>(Q.C[8] * invW);
  const float* Rc = cam.R;
  const float xd = Rc[0] * v0 + Rc[1] * v1 + Rc[2] * v2;
  const float yd = Rc[3] * v0 + Rc[4] * v1 + Rc[5] * v2;
  const float zd = Rc[6] * v0 + Rc[7] * v1 + Rc[8] * v2;
  const float x = f.pc[0], y = f.pc[1], z = f.pc[2];
  const float iz2 = 1.0f / (z * z);
  f.rgb[0] = cam.fx * (xd * z - x * zd) * iz2;
  f.rgb[1] = cam.fy * (yd * z - y * zd) * iz2;
  f.rgb[2] = 0.0f;
}

// Pixel-column range whose centres can lie inside the region where
// alpha >= 1/255 and power >= -4.5, i.e. d^T conic d <= min(9, 2 ln(255 o_t)).
// The axis-aligned box of that ellipse has half-widths sqrt(k2 Sigma'_xx) and
// sqrt(k2 Sigma'_yy); a relative and an absolute slack keep the box a
// superset under FP32 rounding. The box only selects tiles: each pixel still
// applies the exact tests, so the image does not depend on the tile shape.
__device__ __forceinline__ bool pixel_box(const Fwd& f, const CamDev& cam, int& i0, int& i1,
                                          int& j0, int& j1) {
  const float k2 = 1.01f * fminf(9.0f, 2.0f * __logf(255.0f * f.o_t));
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

// Backward of Sigma4 = R diag(s^2) R^T, R = F_map(F_norm(rotor)), s =
// exp(log-scale): from the symmetric gradient G4 of Sigma4 to the gradients
// of the raw rotor (grot) and of the log-scales (gls).
template <typename S>
__device__ __forceinline__ void sigma4_backward(const Geo<S>& G, const S G4[4][4], S grot[8], S gls[4]) {
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
  S grh[8];
  rotor_matrix_bwd<S>(G.rn.r, gR, grh);
  rotor_normalize_bwd<S>(G.p.rot, G.rn, grh, grot);
#pragma unroll
  for (int k = 0; k < 4; ++k) gls[k] = gsc2[k] * S(2) * G.sc2[k];  // d s^2 / d log s = 2 s^2
}

}  // namespace r4g
