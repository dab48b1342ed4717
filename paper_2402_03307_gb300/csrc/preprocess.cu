// Backward of the per-Gaussian preprocess (Sec. 4.2 "CUDA Acceleration":
// the rotor -> rotation and slicing steps differentiated by hand): colour,
// conic, EWA projection, temporal slice per view, then Sigma4 -> R -> F_norm
// and the activations once per Gaussian.
#include <cuda_runtime.h>

#include "preprocess_common.cuh"

namespace r4g {

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
// With kShOut the SH gradient is added into the caller's row gsh; without
// it the unit view direction and the clamped colour gradient go to dirg[6]
// (the SH gradient being Y(dir) (x) d rgb, formed later).
template <typename S, bool kShBF16, bool kShOut = true>
__device__ __forceinline__ void view_backward(const r4g_gaussians& g, int i, const Sig4<S>& G, const CamDev& cam,
                                              float t, int sh_degree, bool temporal_cull, float4 ga, float4 gb,
                                              float4 gc, float* __restrict__ gsh, BwdAcc<S>& acc,
                                              float& radius, float* dirg = nullptr) {
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
  if constexpr (!kShOut) {
    dirg[0] = f.dir[0]; dirg[1] = f.dir[1]; dirg[2] = f.dir[2];
    dirg[3] = grgb[0]; dirg[4] = grgb[1]; dirg[5] = grgb[2];
  } else {
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
  {  // screen radius 3 sqrt(lambda_max(Sigma')) for the density-control statistics
    const float hm = 0.5f * (A - Cc);
    radius = 3.0f * sqrtf(0.5f * (A + Cc) + sqrtf(hm * hm + B * B));
  }
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

// Sum of an item's per-pair gradients (pairs [o, o + cnt) of the gradient
// buffer) for each lane's item. Only pairs whose reach flag is set hold a
// gradient (a pixel of their tile composited them); the others count as zero
// and are not read. Items of 2 .. kGroupPairs pairs (nearly all of them) are
// taken by groups of kGroupLanes lanes, 32 / kGroupLanes items per round: each
// lane reads up to kGroupPairs / kGroupLanes of its item's pairs (all loads
// issued together), the group sums them by a butterfly, and each item's owner
// takes its group's sums with one shuffle per value. Larger items are taken by
// the whole warp, U at a time (lane l adding pairs l, l + 32, ..., then a
// butterfly over the warp); a single pair is read by its owner. gc.w counts the
// tiles in which a pixel composited the item (summed only with kStats).
// Returns whether any pair of the lane's item holds a gradient (if none, the
// item's gradient is zero). The sums are in a fixed order.
constexpr int kGroupLanes = 8;
constexpr uint32_t kGroupPairs = 32;

template <bool kStats, int U>
__device__ __forceinline__ bool gather_pairs(uint32_t cnt, uint32_t o, int lane, const float4* __restrict__ gbuf,
                                             const uint8_t* __restrict__ reach, float4& ga, float4& gb,
                                             float4& gc) {
  constexpr int G = kGroupLanes, NG = 32 / G, PPL = kGroupPairs / G;  // pairs per lane
  constexpr int NV = kStats ? 10 : 9;
  ga = make_float4(0.f, 0.f, 0.f, 0.f);
  gb = ga;
  gc = ga;
  bool got = false;
  // ---- items of 2 .. kGroupPairs pairs: a group of G lanes each
  const bool grouped = cnt >= 2u && cnt <= kGroupPairs;
  const uint32_t gmask = __ballot_sync(0xffffffffu, grouped);
  const int grp = lane / G, gl = lane % G;
  for (int r0 = 0; r0 < 32 && (gmask >> r0); r0 += NG) {
    if (((gmask >> r0) & ((1u << NG) - 1u)) == 0u) continue;  // warp-uniform
    const uint32_t qc = __shfl_sync(0xffffffffu, grouped ? cnt : 0u, r0 + grp);
    const uint32_t qo = __shfl_sync(0xffffffffu, o, r0 + grp);
    bool f[PPL];
#pragma unroll
    for (int i = 0; i < PPL; ++i) {
      const uint32_t k = static_cast<uint32_t>(gl + i * G);
      f[i] = k < qc && reach[qo + k];
    }
    float v[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) v[k] = 0.f;
#pragma unroll
    for (int i = 0; i < PPL; ++i) {
      if (!f[i]) continue;
      const float4* pr = gbuf + 3 * static_cast<size_t>(qo + static_cast<uint32_t>(gl + i * G));
      const float4 x = pr[0], y = pr[1], z = pr[2];
      v[0] += x.x; v[1] += x.y; v[2] += x.z; v[3] += x.w;
      v[4] += y.x; v[5] += y.y;
      v[6] += z.x; v[7] += z.y; v[8] += z.z; v[9] += z.w;
    }
    bool found = false;
#pragma unroll
    for (int i = 0; i < PPL; ++i) found = found || f[i];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
      for (int sh = G / 2; sh > 0; sh >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], sh);
    }
    const uint32_t fb = __ballot_sync(0xffffffffu, found);
    // the owner of item r0 + g takes group g's sums (held by its first lane)
    const int src = ((lane - r0) & (NG - 1)) * G;
    float w[10];
#pragma unroll
    for (int k = 0; k < NV; ++k) w[k] = __shfl_sync(0xffffffffu, v[k], src);
    const bool any = ((fb >> src) & ((1u << G) - 1u)) != 0u;
    if (grouped && lane >= r0 && lane < r0 + NG && any) {
      got = true;
      ga = make_float4(w[0], w[1], w[2], w[3]);
      gb = make_float4(w[4], w[5], 0.f, 0.f);
      gc = make_float4(w[6], w[7], w[8], kStats ? w[9] : 0.f);
    }
  }
  // ---- larger items: the whole warp each, U at a time
  const uint32_t big = cnt > kGroupPairs ? cnt : 0u;
  if (__ballot_sync(0xffffffffu, big != 0u) == 0u) {
    if (cnt == 1 && reach[o]) {
      const float4* pr = gbuf + 3 * static_cast<size_t>(o);
      ga = pr[0];
      gb = pr[1];
      gc = pr[2];
      got = true;
    }
    return got;
  }
  for (int q0 = 0; q0 < 32; q0 += U) {
    uint32_t qc[U], qo[U], kmax = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      qc[u] = __shfl_sync(0xffffffffu, big, q0 + u);  // only the larger items (the others are done)
      qo[u] = __shfl_sync(0xffffffffu, o, q0 + u);
      kmax = max(kmax, qc[u]);
    }
    if (kmax == 0) continue;  // warp-uniform
    float v[U][10];
    bool found[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      found[u] = false;
#pragma unroll
      for (int k = 0; k < 10; ++k) v[u][k] = 0.f;
    }
    for (uint32_t k = lane; k < kmax; k += 32) {
      bool f[U];
#pragma unroll
      for (int u = 0; u < U; ++u) f[u] = k < qc[u] && reach[qo[u] + k];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!f[u]) continue;
        found[u] = true;
        const float4* pr = gbuf + 3 * static_cast<size_t>(qo[u] + k);
        const float4 x = pr[0], y = pr[1], z = pr[2];
        v[u][0] += x.x; v[u][1] += x.y; v[u][2] += x.z; v[u][3] += x.w;
        v[u][4] += y.x; v[u][5] += y.y;
        v[u][6] += z.x; v[u][7] += z.y; v[u][8] += z.z; v[u][9] += z.w;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!__any_sync(0xffffffffu, found[u])) continue;  // no pair of this item holds a gradient
      if (lane == q0 + u) got = true;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) v[u][k] += __shfl_xor_sync(0xffffffffu, v[u][k], sh);
      }
      if constexpr (kStats) {
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) v[u][9] += __shfl_xor_sync(0xffffffffu, v[u][9], sh);
      }
      if (lane == q0 + u) {
        ga = make_float4(v[u][0], v[u][1], v[u][2], v[u][3]);
        gb = make_float4(v[u][4], v[u][5], 0.f, 0.f);
        gc = make_float4(v[u][6], v[u][7], v[u][8], v[u][9]);
      }
    }
  }
  if (cnt == 1 && reach[o]) {
    const float4* pr = gbuf + 3 * static_cast<size_t>(o);
    ga = pr[0];
    gb = pr[1];
    gc = pr[2];
    got = true;
  }
  return got;
}

// Backward of the preprocess over the Gaussians visible in some view (the
// list the forward built). For each view, each warp first sums, for each of
// its 32 Gaussians in turn, the per-pair gradients the blend backward wrote
// (an item's pairs are contiguous, [ioffs[item], ioffs[item] + touched[item])),
// reading them coalesced; then every thread runs its Gaussian's view
// backward. After the views, the Sigma4 -> R -> rotor and scale backward runs
// once per Gaussian and the gradients are added to the caller's buffers.
// Every Gaussian is one thread's: the gradient is deterministic.
template <typename S, bool kScaleBF16, bool kShBF16, bool kMulti, bool kStats>
__global__ void __launch_bounds__(kBwdBlock, kMulti ? 3 : 4)
    preprocess_bwd_kernel(r4g_gaussians g, const ViewDev* __restrict__ views, int nviews,
                          const uint32_t* __restrict__ glist, const uint32_t* __restrict__ ioffs,
                          const uint32_t* __restrict__ touched, const float4* __restrict__ gbuf,
                          const uint8_t* __restrict__ reach, const FrameHeader* hdr, int sh_degree,
                          bool temporal_cull, r4g_grads out) {
  griddep_wait();
  griddep_launch_dependents();
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
  float vs_grad = 0.0f, vs_count = 0.0f, max_radius = 0.0f;  // density-control statistics
  for (int v = 0; v < (kMulti ? nviews : 1); ++v) {
    const size_t item = static_cast<size_t>(v) * g.n + i;
    const uint32_t cnt = mine ? touched[item] : 0u;
    if (__ballot_sync(0xffffffffu, cnt != 0u) == 0u) continue;
    const uint32_t o = cnt ? ioffs[item] : 0u;
    float4 ga, gb, gc;
    const bool got = gather_pairs<kStats, 2>(cnt, o, lane, gbuf, reach, ga, gb, gc);
    if (got) {  // an item no pixel composited has a zero gradient
      float radius;
      view_backward<S, kShBF16>(g, i, Q, views[v].cam, views[v].t, sh_degree, temporal_cull, ga, gb, gc, out.sh,
                                acc, radius);
      if (kStats && gc.w > 0.0f) {  // composited into a pixel of this view
        const float ux = ga.x * (0.5f * static_cast<float>(views[v].cam.width));
        const float uy = ga.y * (0.5f * static_cast<float>(views[v].cam.height));
        vs_grad += sqrtf(ux * ux + uy * uy);
        vs_count += 1.0f;
        max_radius = fmaxf(max_radius, radius);
      }
    }
  }
  if (!mine) return;
  if (kStats && vs_count > 0.0f) {
    if (out.vs_grad) out.vs_grad[i] += vs_grad;
    if (out.vs_count) out.vs_count[i] += vs_count;
    if (out.max_radius) out.max_radius[i] = fmaxf(out.max_radius[i], max_radius);
  }
  Geo<S> G;  // the rotor and scale intermediates, recomputed rather than kept through the views
  gauss_setup<S, kScaleBF16>(g, i, G);
  // symmetric gradient of Sigma4
  S G4[4][4];
  G4[0][0] = acc.G4[0]; G4[0][1] = G4[1][0] = acc.G4[1]; G4[0][2] = G4[2][0] = acc.G4[2];
  G4[0][3] = G4[3][0] = acc.G4[3]; G4[1][1] = acc.G4[4]; G4[1][2] = G4[2][1] = acc.G4[5];
  G4[1][3] = G4[3][1] = acc.G4[6]; G4[2][2] = acc.G4[7]; G4[2][3] = G4[3][2] = acc.G4[8];
  G4[3][3] = acc.G4[9];
  S grot[8], gls[4];
  sigma4_backward<S>(G, G4, grot, gls);

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
  vl.x += static_cast<float>(gls[0]);
  vl.y += static_cast<float>(gls[1]);
  vl.z += static_cast<float>(gls[2]);
  vl.w += static_cast<float>(gls[3]);
  *gl = vl;
  out.logit[i] += static_cast<float>(acc.gop) * G.opacity * (1.0f - G.opacity);
}

// ---- multi-view backward in two passes -------------------------------------
// With several views, a thread per Gaussian would idle in every view that does
// not see its Gaussian. Instead: (1) the visible (view, Gaussian) items are
// listed, (2) one thread per listed item runs that view's backward and keeps a
// partial gradient (96 B), (3) one thread per Gaussian sums its items'
// partials in view order (deterministic) and runs the Sigma4 -> rotor and
// scale backward once.
// float4s per partial: d Sigma4 (10), d mean (4), d opacity, dir (3), d rgb (3), statistics (3)
constexpr int kPartVec = 6;

__global__ void __launch_bounds__(1024)
    list_items_kernel(const uint32_t* __restrict__ touched, uint32_t m, uint32_t* __restrict__ ilist,
                      FrameHeader* hdr) {
  griddep_wait();
  griddep_launch_dependents();
  // one counter update per CTA (per warp, 16M items made the counter the bottleneck)
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_base;
  const uint32_t k = blockIdx.x * 1024 + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool vis = k < m && touched[k] != 0u;
  const uint32_t b = __ballot_sync(0xffffffffu, vis);
  if (lane == 0) s_warp[warp] = __popc(b);
  __syncthreads();
  if (warp == 0) {
    const uint32_t c = s_warp[lane];
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_warp[lane] = x - c;  // exclusive over the warps
    if (lane == 31) s_base = x ? atomicAdd(&hdr->n_ilist, x) : 0u;
  }
  __syncthreads();
  if (vis) ilist[s_base + s_warp[warp] + __popc(b & ((1u << lane) - 1u))] = k;
}

// First pass of the multi-view backward: each listed item's per-pair
// gradients summed (gather_pairs), written into the first three vectors of its
// partial slot (ga, gb with gb.z = 1 marking an item with a gradient, gc); an
// item without one gets its whole partial zeroed. A kernel of its own, lean
// in registers, so that many warps keep the gather's loads in flight.
constexpr int kGatherBlock = 256;
constexpr int kGatherItems = 2;  // items in flight per round of the gather

template <bool kStats>
__global__ void __launch_bounds__(kGatherBlock)
    preprocess_bwd_gather_kernel(const uint32_t* __restrict__ ilist, const uint32_t* __restrict__ ioffs,
                                 const uint32_t* __restrict__ touched, const float4* __restrict__ gbuf,
                                 const uint8_t* __restrict__ reach, const FrameHeader* hdr,
                                 float4* __restrict__ ipart) {
  griddep_wait();
  griddep_launch_dependents();
  const int j = blockIdx.x * kGatherBlock + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int nlist = static_cast<int>(hdr->n_ilist);
  if ((hdr->status & 1u) || (j - lane) >= nlist) return;  // warp-uniform
  const bool mine = j < nlist;
  const uint32_t item = mine ? ilist[j] : 0u;
  const uint32_t cnt = mine ? touched[item] : 0u;
  const uint32_t o = cnt ? ioffs[item] : 0u;
  float4 ga, gb, gc;
  const bool got = gather_pairs<kStats, kGatherItems>(cnt, o, lane, gbuf, reach, ga, gb, gc) && mine;
  if (!mine) return;
  float4* d = ipart + kPartVec * static_cast<size_t>(item);
  if (got) {
    gb.z = 1.0f;
    d[0] = ga;
    d[1] = gb;
    d[2] = gc;
  } else {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    d[0] = d[1] = d[2] = d[3] = d[4] = d[5] = z;
  }
}

template <bool kScaleBF16, bool kShBF16, bool kStats>
__global__ void __launch_bounds__(kBwdBlock, 4)
    preprocess_bwd_items_kernel(r4g_gaussians g, const ViewDev* __restrict__ views,
                                const uint32_t* __restrict__ ilist, const FrameHeader* hdr, int sh_degree,
                                bool temporal_cull, float4* __restrict__ ipart) {
  griddep_wait();
  griddep_launch_dependents();
  // Items without a gradient (no pixel composited them) have a zero partial
  // already (the gather pass); the others are packed to the front of the CTA
  // (their summed pair gradients through shared memory) so the chain rule
  // runs on full warps: in a scene whose pixels saturate early most items
  // have none.
  __shared__ float4 s_g[3][kBwdBlock];
  __shared__ uint32_t s_item[kBwdBlock];
  __shared__ uint32_t s_wcnt[kBwdBlock / 32];
  const int j = blockIdx.x * kBwdBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nlist = static_cast<int>(hdr->n_ilist);
  if ((hdr->status & 1u) || static_cast<int>(blockIdx.x) * kBwdBlock >= nlist) return;  // CTA-uniform
  const bool mine = j < nlist;
  uint32_t item = mine ? ilist[j] : 0u;
  float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga, gc = ga;
  if (mine) {
    const float4* src = ipart + kPartVec * static_cast<size_t>(item);
    gb = src[1];
    if (gb.z != 0.0f) {
      ga = src[0];
      gc = src[2];
    }
  }
  const bool got = mine && gb.z != 0.0f;
  const uint32_t b = __ballot_sync(0xffffffffu, got);
  if (lane == 0) s_wcnt[warp] = __popc(b);
  __syncthreads();
  uint32_t base = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kBwdBlock / 32; ++w) {
    base += w < warp ? s_wcnt[w] : 0u;
    total += s_wcnt[w];
  }
  if (got) {
    const uint32_t r = base + __popc(b & ((1u << lane) - 1u));
    s_item[r] = item;
    s_g[0][r] = ga;
    s_g[1][r] = gb;
    s_g[2][r] = gc;
  }
  __syncthreads();
  if (threadIdx.x >= total) return;
  item = s_item[threadIdx.x];
  ga = s_g[0][threadIdx.x];
  gb = s_g[1][threadIdx.x];
  gc = s_g[2][threadIdx.x];
  float4* d = ipart + kPartVec * static_cast<size_t>(item);
  const int v = static_cast<int>(item / static_cast<uint32_t>(g.n));
  const int i = static_cast<int>(item - static_cast<uint32_t>(v) * static_cast<uint32_t>(g.n));
  Sig4<float> Q;
  gauss_sigma<float, kScaleBF16>(g, i, Q);
  BwdAcc<float> acc;
#pragma unroll
  for (int k = 0; k < 10; ++k) acc.G4[k] = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) acc.gmean[k] = 0.0f;
  acc.gop = 0.0f;
  float radius, dirg[6];
  view_backward<float, kShBF16, false>(g, i, Q, views[v].cam, views[v].t, sh_degree, temporal_cull, ga, gb, gc,
                                       nullptr, acc, radius, dirg);
  float st[3] = {0.0f, 0.0f, 0.0f};
  if (kStats && gc.w > 0.0f) {  // composited into a pixel of this view
    const float ux = ga.x * (0.5f * static_cast<float>(views[v].cam.width));
    const float uy = ga.y * (0.5f * static_cast<float>(views[v].cam.height));
    st[0] = sqrtf(ux * ux + uy * uy);
    st[1] = 1.0f;
    st[2] = radius;
  }
  d[0] = make_float4(acc.G4[0], acc.G4[1], acc.G4[2], acc.G4[3]);
  d[1] = make_float4(acc.G4[4], acc.G4[5], acc.G4[6], acc.G4[7]);
  d[2] = make_float4(acc.G4[8], acc.G4[9], acc.gmean[0], acc.gmean[1]);
  d[3] = make_float4(acc.gmean[2], acc.gmean[3], acc.gop, dirg[0]);
  d[4] = make_float4(dirg[1], dirg[2], dirg[3], dirg[4]);
  d[5] = make_float4(dirg[5], st[0], st[1], st[2]);
}

template <bool kScaleBF16, bool kStats>
__global__ void __launch_bounds__(kBwdBlock)
    preprocess_bwd_gauss_kernel(r4g_gaussians g, int nviews, const uint32_t* __restrict__ glist,
                                const uint32_t* __restrict__ touched, const float4* __restrict__ ipart,
                                const FrameHeader* hdr, int sh_degree, r4g_grads out) {
  griddep_wait();
  griddep_launch_dependents();
  const int j = blockIdx.x * kBwdBlock + threadIdx.x;
  const int nlist = static_cast<int>(hdr->n_glist);
  if ((hdr->status & 1u) || j >= nlist) return;
  const int i = static_cast<int>(glist[j]);
  float G4s[10], gm[4], gop = 0.0f, vs_grad = 0.0f, vs_count = 0.0f, max_radius = 0.0f;
#pragma unroll
  for (int k = 0; k < 10; ++k) G4s[k] = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) gm[k] = 0.0f;
  const int nb = (sh_degree + 1) * (sh_degree + 1);
  // the SH gradient sum_v Y(dir_v) (x) d rgb_v in registers, added to the
  // caller's row once; the next view's visibility is loaded while this
  // view's partial is: one memory round trip per view
  float gsh[48];
#pragma unroll
  for (int k = 0; k < 48; ++k) gsh[k] = 0.0f;
  uint32_t tnext = touched[i];
  for (int v = 0; v < nviews; ++v) {
    const uint32_t tcur = tnext;
    if (v + 1 < nviews) tnext = touched[static_cast<size_t>(v + 1) * g.n + i];
    if (tcur == 0u) continue;
    const float4* p = ipart + kPartVec * (static_cast<size_t>(v) * g.n + i);
    const float4 a = p[0], b = p[1], c = p[2], d = p[3], e = p[4], f = p[5];
    G4s[0] += a.x; G4s[1] += a.y; G4s[2] += a.z; G4s[3] += a.w;
    G4s[4] += b.x; G4s[5] += b.y; G4s[6] += b.z; G4s[7] += b.w;
    G4s[8] += c.x; G4s[9] += c.y; gm[0] += c.z; gm[1] += c.w;
    gm[2] += d.x; gm[3] += d.y; gop += d.z;
    const float grgb[3] = {e.z, e.w, f.x};
    float Y[16];
    sh_basis(d.w, e.x, e.y, Y);
#pragma unroll
    for (int el = 0; el < 48; ++el) gsh[el] += Y[el / 3] * grgb[el % 3];
    if constexpr (kStats) {
      vs_grad += f.y;
      vs_count += f.z;
      max_radius = fmaxf(max_radius, f.w);
    }
  }
  {  // d c_k += sum over the views, 16-byte vectors over the row's first nb bands
    float4* gsh4 = reinterpret_cast<float4*>(out.sh + static_cast<size_t>(i) * 48);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      if (4 * q < nb * 3) {
        float4 w = gsh4[q];
        float* wp = reinterpret_cast<float*>(&w);
#pragma unroll
        for (int h = 0; h < 4; ++h)
          if (4 * q + h < nb * 3) wp[h] += gsh[4 * q + h];
        gsh4[q] = w;
      }
    }
  }
  Geo<float> G;
  gauss_setup<float, kScaleBF16>(g, i, G);
  float G4[4][4];
  G4[0][0] = G4s[0]; G4[0][1] = G4[1][0] = G4s[1]; G4[0][2] = G4[2][0] = G4s[2];
  G4[0][3] = G4[3][0] = G4s[3]; G4[1][1] = G4s[4]; G4[1][2] = G4[2][1] = G4s[5];
  G4[1][3] = G4[3][1] = G4s[6]; G4[2][2] = G4s[7]; G4[2][3] = G4[3][2] = G4s[8];
  G4[3][3] = G4s[9];
  float grot[8], gls[4];
  sigma4_backward<float>(G, G4, grot, gls);
  float4* gmo = reinterpret_cast<float4*>(out.mean) + i;
  float4 vm = *gmo;
  vm.x += gm[0]; vm.y += gm[1]; vm.z += gm[2]; vm.w += gm[3];
  *gmo = vm;
  float4* gr = reinterpret_cast<float4*>(out.rotor) + 2 * static_cast<size_t>(i);
  float4 r0 = gr[0], r1 = gr[1];
  r0.x += grot[0]; r0.y += grot[1]; r0.z += grot[2]; r0.w += grot[3];
  r1.x += grot[4]; r1.y += grot[5]; r1.z += grot[6]; r1.w += grot[7];
  gr[0] = r0;
  gr[1] = r1;
  float4* gl = reinterpret_cast<float4*>(out.logscale) + i;
  float4 vl = *gl;
  vl.x += gls[0]; vl.y += gls[1]; vl.z += gls[2]; vl.w += gls[3];
  *gl = vl;
  out.logit[i] += gop * G.opacity * (1.0f - G.opacity);
  if (kStats && vs_count > 0.0f) {
    if (out.vs_grad) out.vs_grad[i] += vs_grad;
    if (out.vs_count) out.vs_count[i] += vs_count;
    if (out.max_radius) out.max_radius[i] = fmaxf(out.max_radius[i], max_radius);
  }
}

template <typename S, bool A, bool B>
static void launch_pre_bwd_t(const r4g_gaussians& g, const FrameLayout& L, void* frame, int sh_degree, bool tc,
                             const r4g_grads& out, cudaStream_t s) {
  const int nb = static_cast<int>((L.n + kBwdBlock - 1) / kBwdBlock);
  if constexpr (sizeof(S) == sizeof(float)) {
    if (L.nviews > 1) {  // the two-pass multi-view backward (FP32 slice)
      const bool stats = out.vs_grad || out.vs_count || out.max_radius;
      FrameHeader* hdr = at<FrameHeader>(frame, L.header);
      const uint32_t* touched = at<uint32_t>(frame, L.touched);
      uint32_t* ilist = at<uint32_t>(frame, L.ilist);
      float4* ipart = at<float4>(frame, L.ipart);
      // (the blend backward zeroed the item counter)
      const int nbm = static_cast<int>((L.m + 1023) / 1024);
      launch_pdl(list_items_kernel, nbm, 1024, 0, s, touched, static_cast<uint32_t>(L.m), ilist, hdr);
      const int nbg = static_cast<int>((L.m + kGatherBlock - 1) / kGatherBlock);
      auto kgt = stats ? preprocess_bwd_gather_kernel<true> : preprocess_bwd_gather_kernel<false>;
      launch_pdl(kgt, nbg, kGatherBlock, 0, s, static_cast<const uint32_t*>(ilist),
                 static_cast<const uint32_t*>(at<uint32_t>(frame, L.ioffs)), touched,
                 static_cast<const float4*>(at<float4>(frame, L.gbuf)),
                 static_cast<const uint8_t*>(at<uint8_t>(frame, L.reach)), static_cast<const FrameHeader*>(hdr),
                 ipart);
      const int nbi = static_cast<int>((L.m + kBwdBlock - 1) / kBwdBlock);
      auto ki = stats ? preprocess_bwd_items_kernel<A, B, true> : preprocess_bwd_items_kernel<A, B, false>;
      launch_pdl(ki, nbi, kBwdBlock, 0, s, g, static_cast<const ViewDev*>(at<ViewDev>(frame, L.views)),
                 static_cast<const uint32_t*>(ilist), static_cast<const FrameHeader*>(hdr), sh_degree, tc, ipart);
      auto kg = stats ? preprocess_bwd_gauss_kernel<A, true> : preprocess_bwd_gauss_kernel<A, false>;
      launch_pdl(kg, nb, kBwdBlock, 0, s, g, L.nviews, static_cast<const uint32_t*>(at<uint32_t>(frame, L.glist)),
                 touched, static_cast<const float4*>(ipart), static_cast<const FrameHeader*>(hdr), sh_degree, out);
      return;
    }
  }
  const bool stats = out.vs_grad || out.vs_count || out.max_radius;
  // one thread per Gaussian over the views: every one-view call, and
  // multi-view calls of the FP64 debug slice
  auto k = stats ? preprocess_bwd_kernel<S, A, B, false, true> : preprocess_bwd_kernel<S, A, B, false, false>;
  if constexpr (sizeof(S) != sizeof(float)) {
    if (L.nviews > 1) k = stats ? preprocess_bwd_kernel<S, A, B, true, true> : preprocess_bwd_kernel<S, A, B, true, false>;
  }
  launch_pdl(k, nb, kBwdBlock, 0, s, g, static_cast<const ViewDev*>(at<ViewDev>(frame, L.views)), L.nviews,
             static_cast<const uint32_t*>(at<uint32_t>(frame, L.glist)),
             static_cast<const uint32_t*>(at<uint32_t>(frame, L.ioffs)),
             static_cast<const uint32_t*>(at<uint32_t>(frame, L.touched)),
             static_cast<const float4*>(at<float4>(frame, L.gbuf)),
             static_cast<const uint8_t*>(at<uint8_t>(frame, L.reach)),
             static_cast<const FrameHeader*>(at<FrameHeader>(frame, L.header)), sh_degree, tc, out);
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
