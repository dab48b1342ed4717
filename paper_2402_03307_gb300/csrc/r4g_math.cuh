// Per-Gaussian device arithmetic of the render: parameter loads, rotor
// normalisation (appendix A.1), rotor -> matrix (appendix A.2), Sigma4
// (Sec. 3.2.1), temporal slice (Sec. 3.2.2 / appendix A.3), projection (Sec. 3.1)
// and the degree-3 real SH basis. Shared by the forward and backward
// preprocess kernels.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

#include "r4g_internal.cuh"

namespace r4g {

__device__ __forceinline__ float bf16_to_f32(uint16_t h) {
  return __uint_as_float(static_cast<uint32_t>(h) << 16);
}

// Raw parameters of one Gaussian, loaded with 16-byte vector loads.
struct Params {
  float mean[4];
  float rot[8];
  float ls[4];
  float logit;
};

template <bool kScaleBF16>
__device__ __forceinline__ void load_params(const r4g_gaussians& g, int i, Params& p) {
  const float4 m = __ldg(reinterpret_cast<const float4*>(g.mean) + i);
  const float4 r0 = __ldg(reinterpret_cast<const float4*>(g.rotor) + 2 * i);
  const float4 r1 = __ldg(reinterpret_cast<const float4*>(g.rotor) + 2 * i + 1);
  p.mean[0] = m.x; p.mean[1] = m.y; p.mean[2] = m.z; p.mean[3] = m.w;
  p.rot[0] = r0.x; p.rot[1] = r0.y; p.rot[2] = r0.z; p.rot[3] = r0.w;
  p.rot[4] = r1.x; p.rot[5] = r1.y; p.rot[6] = r1.z; p.rot[7] = r1.w;
  if constexpr (kScaleBF16) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(g.logscale) + i);
    p.ls[0] = bf16_to_f32(v.x & 0xffffu); p.ls[1] = bf16_to_f32(v.x >> 16);
    p.ls[2] = bf16_to_f32(v.y & 0xffffu); p.ls[3] = bf16_to_f32(v.y >> 16);
  } else {
    const float4 v = __ldg(reinterpret_cast<const float4*>(g.logscale) + i);
    p.ls[0] = v.x; p.ls[1] = v.y; p.ls[2] = v.z; p.ls[3] = v.w;
  }
  p.logit = __ldg(g.logit + i);
}

// Read-only 16-byte loads the compiler must issue where they are written: a
// Gaussian's SH row is loop-invariant over the views of a call, and hoisting
// it out of the view loop (and out of the visibility test) would keep 48
// registers live throughout and read the rows of invisible Gaussians.
__device__ __forceinline__ float4 ld_nc_f4(const float4* p) {
  float4 r;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "l"(p));
  return r;
}

__device__ __forceinline__ uint4 ld_nc_u4(const uint4* p) {
  uint4 r;
  asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

// SH coefficients of one Gaussian: c[k][ch] for the first nb = (deg+1)^2 bands.
template <bool kShBF16>
__device__ __forceinline__ void load_sh(const void* sh, int i, int nb, float c[16][3]) {
  if constexpr (kShBF16) {
    const uint4* p = reinterpret_cast<const uint4*>(sh) + 6 * static_cast<int64_t>(i);
    const int nvec = (nb * 3 + 7) / 8;
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      if (v < nvec) {
        const uint4 w = ld_nc_u4(p + v);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int h = 0; h < 8; ++h) {
          const int e = v * 8 + h;
          const float f = bf16_to_f32((h & 1) ? (ws[h >> 1] >> 16) : (ws[h >> 1] & 0xffffu));
          c[e / 3][e % 3] = f;
        }
      }
    }
  } else {
    const float4* p = reinterpret_cast<const float4*>(sh) + 12 * static_cast<int64_t>(i);
    const int nvec = (nb * 3 + 3) / 4;
#pragma unroll
    for (int v = 0; v < 12; ++v) {
      if (v < nvec) {
        const float4 w = ld_nc_f4(p + v);
        const float ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int e = v * 4 + h;
          c[e / 3][e % 3] = ws[h];
        }
      }
    }
  }
}

// ---- rotor (appendix A.1, A.2) ----------------------------------------------
// Storage order (s, b01, b02, b12, b03, b13, b23, p).
template <typename S>
struct RotorNorm {
  S r[8];      // normalised rotor
  S eps, l2, delta, n2;
  S r1[8];     // rotor after the root step, before division by its norm
  bool ident;  // degenerate input mapped to the identity rotor
};

template <typename S>
__device__ __forceinline__ void eps_grad(const S r[8], S g[8]) {
  // d eps / d (s, b01, b02, b12, b03, b13, b23, p) for
  // eps = p s - b01 b23 + b02 b13 - b03 b12
  g[0] = r[7]; g[1] = -r[6]; g[2] = r[5]; g[3] = -r[4];
  g[4] = -r[3]; g[5] = r[2]; g[6] = -r[1]; g[7] = r[0];
}

template <typename S>
__device__ __forceinline__ void rotor_normalize(const float in[8], RotorNorm<S>& o) {
  S r[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) r[k] = static_cast<S>(in[k]);
  const S eps = r[7] * r[0] - r[1] * r[6] + r[2] * r[5] - r[4] * r[3];
  S l2 = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) l2 += r[k] * r[k];
  S disc = l2 * l2 - S(4) * eps * eps;
  disc = disc > S(0) ? disc : S(0);
  // root of (1 + d^2) eps + l^2 d = 0 that vanishes with eps, written as
  // -2 eps / (l^2 + sqrt(l^4 - 4 eps^2)) (finite at eps = 0)
  const S delta = l2 > S(0) ? S(-2) * eps / (l2 + sqrt(disc)) : S(0);
  S g[8];
  eps_grad(r, g);
  S n2 = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    o.r1[k] = r[k] + delta * g[k];
    n2 += o.r1[k] * o.r1[k];
  }
  o.eps = eps; o.l2 = l2; o.delta = delta; o.n2 = n2;
  o.ident = !(n2 > S(1e-20));
  if (o.ident) {
#pragma unroll
    for (int k = 0; k < 8; ++k) o.r[k] = S(0);
    o.r[0] = S(1);
  } else {
    const S inv = S(1) / sqrt(n2);
#pragma unroll
    for (int k = 0; k < 8; ++k) o.r[k] = o.r1[k] * inv;
  }
}

// a b + c rounded once, in the slice precision, whatever the translation
// unit's contraction flags: the forward preprocess (compiled without
// contraction, so that one-view and multi-view renders agree bit for bit) and
// the backward's recomputation take the same fused steps.
__device__ __forceinline__ float fma_s(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_s(double a, double b, double c) { return __fma_rn(a, b, c); }

// a0 b0 + a1 b1 + a2 b2 + a3 b3 as one product and three fused steps.
template <typename S>
__device__ __forceinline__ S dot4(S a0, S b0, S a1, S b1, S a2, S b2, S a3, S b3) {
  return fma_s(a3, b3, fma_s(a2, b2, fma_s(a1, b1, a0 * b0)));
}

// R (row-major 4x4) from a normalised rotor, the closed forms of appendix A.2
// (each diagonal entry a signed sum of the eight squares, each off-diagonal
// entry twice a signed sum of four products).
template <typename S>
__device__ __forceinline__ void rotor_matrix(const S r[8], S R[16]) {
  const S s = r[0], b01 = r[1], b02 = r[2], b12 = r[3], b03 = r[4], b13 = r[5], b23 = r[6], p = r[7];
  // sum of s^2 - p^2 and the squares of the bivector parts with the given signs
  auto diag = [&](S e01, S e02, S e03, S e12, S e13, S e23) {
    S x = fma_s(-p, p, s * s);
    x = fma_s(e01 * b01, b01, x);
    x = fma_s(e02 * b02, b02, x);
    x = fma_s(e03 * b03, b03, x);
    x = fma_s(e12 * b12, b12, x);
    x = fma_s(e13 * b13, b13, x);
    return fma_s(e23 * b23, b23, x);
  };
  const S one = S(1);
  R[0] = diag(-one, -one, -one, one, one, one);
  R[5] = diag(-one, one, one, -one, -one, one);
  R[10] = diag(one, -one, one, -one, one, -one);
  R[15] = diag(one, one, -one, one, -one, -one);
  R[1] = S(2) * dot4(b01, s, -b02, b12, -b03, b13, b23, p);
  R[2] = S(2) * dot4(b01, b12, b02, s, -b03, b23, -b13, p);
  R[3] = S(2) * dot4(b01, b13, b02, b23, b03, s, b12, p);
  R[4] = S(2) * dot4(-b01, s, -b02, b12, -b03, b13, -b23, p);
  R[6] = S(2) * dot4(-b01, b02, b03, p, b12, s, -b13, b23);
  R[7] = S(2) * dot4(-b01, b03, -b02, p, b12, b23, b13, s);
  R[8] = S(2) * dot4(b01, b12, -b02, s, -b03, b23, b13, p);
  R[9] = S(2) * dot4(-b01, b02, -b03, p, -b12, s, -b13, b23);
  R[11] = S(2) * dot4(b01, p, -b02, b03, -b12, b13, b23, s);
  R[12] = S(2) * dot4(b01, b13, b02, b23, -b03, s, -b12, p);
  R[13] = S(2) * dot4(-b01, b03, b02, p, b12, b23, -b13, s);
  R[14] = S(2) * dot4(-b01, p, -b02, b03, -b12, b13, -b23, s);
}

// Sigma4 = R diag(s^2) R^T; returned as its 10 unique entries
// (00, 01, 02, 03, 11, 12, 13, 22, 23, 33).
template <typename S>
__device__ __forceinline__ void cov4(const S R[16], const S sc2[4], S C[10]) {
  S Rs[16];  // R diag(s^2)
#pragma unroll
  for (int i = 0; i < 16; ++i) Rs[i] = R[i] * sc2[i & 3];
  int k = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = i; j < 4; ++j) {
      C[k++] = dot4(Rs[4 * i + 0], R[4 * j + 0], Rs[4 * i + 1], R[4 * j + 1], Rs[4 * i + 2], R[4 * j + 2],
                    Rs[4 * i + 3], R[4 * j + 3]);
    }
  }
}

// ---- degree-3 real SH basis --------------------------------------------------
// Y_{l,m} = sqrt2 Im Y_l^|m| (m<0), Y_l^0, sqrt2 Re Y_l^m (m>0) with the
// Condon-Shortley phase in Y_l^m; index l^2 + l + m. Constants (closed forms):
constexpr float kY00 = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
constexpr float kY2a = 1.0925484305920792f;   // sqrt(15 / pi) / 2
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5 / pi) / 4
constexpr float kY2c = 0.54627421529603959f;  // sqrt(15 / pi) / 4
constexpr float kY3a = 0.59004358992664352f;  // sqrt(35 / (2 pi)) / 4
constexpr float kY3b = 2.8906114426405538f;   // sqrt(105 / pi) / 2
constexpr float kY3c = 0.45704579946446572f;  // sqrt(21 / (2 pi)) / 4
constexpr float kY3d = 0.37317633259011546f;  // sqrt(7 / pi) / 4
constexpr float kY3e = 1.4453057213202769f;   // sqrt(105 / pi) / 4

__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = kY00;
  Y[1] = -kY1 * y;
  Y[2] = kY1 * z;
  Y[3] = -kY1 * x;
  Y[4] = kY2a * x * y;
  Y[5] = -kY2a * y * z;
  Y[6] = kY2b * (2.f * zz - xx - yy);
  Y[7] = -kY2a * x * z;
  Y[8] = kY2c * (xx - yy);
  Y[9] = -kY3a * y * (3.f * xx - yy);
  Y[10] = kY3b * x * y * z;
  Y[11] = -kY3c * y * (4.f * zz - xx - yy);
  Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kY3c * x * (4.f * zz - xx - yy);
  Y[14] = kY3e * z * (xx - yy);
  Y[15] = -kY3a * x * (xx - 3.f * yy);
}

}  // namespace r4g
