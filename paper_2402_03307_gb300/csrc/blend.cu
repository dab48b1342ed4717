// Tiled front-to-back alpha compositing (Sec. 3.1, Eq. 3) over the sorted
// per-tile Gaussian lists. One CTA per tile, one thread per pixel. Batches
// of CTA-size screen records are staged in shared memory; every pixel walks
// the batch applying the per-pixel rules
//   power = -1/2 d^T conic d, skip if power > 0 or power < -4.5,
//   alpha = min(0.99, opacity_t exp(power)), skip if alpha < 1/255,
//   stop before a Gaussian that would take T below 1e-4,
// and the CTA leaves as soon as every pixel has stopped (block-wide vote).
#include <cuda_runtime.h>

#include "r4g_internal.cuh"

namespace r4g {

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH)
    blend_fwd_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                     const float4* __restrict__ recA, const float4* __restrict__ recB,
                     const float4* __restrict__ recC, int width, int height, int tiles_x,
                     float bg0, float bg1, float bg2, float* __restrict__ out_rgb,
                     float* __restrict__ out_T, uint32_t* __restrict__ out_last) {
  constexpr int BS = TW * TH;
  __shared__ float4 sA[BS];
  __shared__ float4 sB[BS];
  __shared__ float4 sC[BS];
  const int tile = blockIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int px = tx * TW + static_cast<int>(threadIdx.x) % TW;
  const int py = ty * TH + static_cast<int>(threadIdx.x) / TW;
  const bool inside = px < width && py < height;
  const float fx = px + 0.5f, fy = py + 0.5f;
  const uint2 rg = ranges[tile];
  const int n = static_cast<int>(rg.y - rg.x);
  float T = 1.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
  uint32_t last = 0;
  bool done = !inside;
  for (int b = 0; b < n; b += BS) {
    if (__syncthreads_count(done) == BS) break;
    const int idx = b + static_cast<int>(threadIdx.x);
    if (idx < n) {
      const uint32_t gid = vals[rg.x + idx];
      sA[threadIdx.x] = recA[gid];
      sB[threadIdx.x] = recB[gid];
      sC[threadIdx.x] = recC[gid];
    }
    __syncthreads();
    const int cnt = min(BS, n - b);
    if (!done) {
      for (int j = 0; j < cnt; ++j) {
        const float4 A = sA[j];
        const float4 B = sB[j];
        float dx, dy;
        const float power = gauss_power(A, B.x, fx, fy, dx, dy);
        if (power > 0.0f || power < kPowerCut) continue;
        const float alpha = fminf(kAlphaMax, __fmul_rn(B.y, __expf(power)));
        if (alpha < kAlphaMin) continue;
        const float Tn = T * (1.0f - alpha);
        if (Tn < kTMin) {
          done = true;
          break;
        }
        const float4 Cc = sC[j];
        const float w = alpha * T;
        c0 += Cc.x * w;
        c1 += Cc.y * w;
        c2 += Cc.z * w;
        T = Tn;
        last = static_cast<uint32_t>(b + j + 1);
      }
    }
  }
  if (inside) {
    const size_t pix = static_cast<size_t>(py) * width + px;
    const size_t plane = static_cast<size_t>(width) * height;
    out_rgb[pix] = c0 + T * bg0;
    out_rgb[plane + pix] = c1 + T * bg1;
    out_rgb[2 * plane + pix] = c2 + T * bg2;
    out_T[pix] = T;
    out_last[pix] = last;
  }
}

cudaError_t launch_blend_fwd(const FrameLayout& L, void* frame, const uint32_t* vals,
                             const float* bg, float* out_rgb, float* out_T, uint32_t* out_last,
                             cudaStream_t s) {
  const float4* recA = at<float4>(frame, L.rec);
  const float4* recB = recA + L.n;
  const float4* recC = recB + L.n;
  const uint2* ranges = at<uint2>(frame, L.ranges);
  // the frame always keeps T and the last position for the backward
  float* T = at<float>(frame, L.tfinal);
  uint32_t* last = at<uint32_t>(frame, L.last);
  const size_t npix = static_cast<size_t>(L.width) * L.height;
#define R4G_BLEND(TW_, TH_)                                                                   \
  blend_fwd_kernel<TW_, TH_><<<L.ntiles, TW_ * TH_, 0, s>>>(ranges, vals, recA, recB, recC,   \
                                                             L.width, L.height, L.tiles_x,    \
                                                             bg[0], bg[1], bg[2], out_rgb, T, \
                                                             last)
  if (L.tile_w == 16 && L.tile_h == 16) R4G_BLEND(16, 16);
  else if (L.tile_w == 8 && L.tile_h == 8) R4G_BLEND(8, 8);
  else if (L.tile_w == 16 && L.tile_h == 32) R4G_BLEND(16, 32);
  else return cudaErrorInvalidValue;
#undef R4G_BLEND
  if (out_T) cudaMemcpyAsync(out_T, T, npix * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (out_last)
    cudaMemcpyAsync(out_last, last, npix * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}


// Backward of the blend. Each pixel re-walks its list back to front from the
// stored final transmittance T_N and last position: T_i = T_{i+1} / (1 - a_i),
// the colour already accumulated behind i is carried along, and per-Gaussian
// gradients (d mean2d, d conic, d opacity_t, d rgb) are summed over the warp
// with a transpose reduction (14 shuffles for 9 values) before one atomic add
// per value and warp. Decisions (cutoff, 1/255) are recomputed with the same
// code as the forward so the composited set is identical.
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH)
    blend_bwd_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                     const float4* __restrict__ recA, const float4* __restrict__ recB,
                     const float4* __restrict__ recC, int width, int height, int tiles_x,
                     float bg0, float bg1, float bg2, const float* __restrict__ Tfinal,
                     const uint32_t* __restrict__ lastpos, const float* __restrict__ grad_rgb,
                     float* __restrict__ rgrad) {
  constexpr int BS = TW * TH;
  __shared__ float4 sA[BS];
  __shared__ float4 sB[BS];
  __shared__ float4 sC[BS];
  __shared__ uint32_t sG[BS];
  __shared__ uint32_t s_max;
  const int tile = blockIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int px = tx * TW + static_cast<int>(threadIdx.x) % TW;
  const int py = ty * TH + static_cast<int>(threadIdx.x) / TW;
  const bool inside = px < width && py < height;
  const float fx = px + 0.5f, fy = py + 0.5f;
  const int lane = threadIdx.x & 31;
  const uint2 rg = ranges[tile];
  const int n = static_cast<int>(rg.y - rg.x);
  float T = 1.0f, Tf = 1.0f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
  uint32_t L = 0;
  if (inside) {
    const size_t pix = static_cast<size_t>(py) * width + px;
    const size_t plane = static_cast<size_t>(width) * height;
    T = Tfinal[pix];
    Tf = T;
    L = lastpos[pix];
    g0 = grad_rgb[pix];
    g1 = grad_rgb[plane + pix];
    g2 = grad_rgb[2 * plane + pix];
  }
  const float bgg = Tf * (bg0 * g0 + bg1 * g1 + bg2 * g2);  // d out / d(T_final) . g
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, L);
  if (lane == 0 && wmax) atomicMax(&s_max, wmax);
  __syncthreads();
  const int maxL = static_cast<int>(s_max);
  float S = 0.0f;  // sum over Gaussians behind i of g . c_k a_k T_k
  for (int b0 = ((maxL - 1) / BS) * BS; maxL > 0 && b0 >= 0; b0 -= BS) {
    const int idx = b0 + static_cast<int>(threadIdx.x);
    __syncthreads();
    if (idx < n) {
      const uint32_t gid = vals[rg.x + idx];
      sG[threadIdx.x] = gid;
      sA[threadIdx.x] = recA[gid];
      sB[threadIdx.x] = recB[gid];
      sC[threadIdx.x] = recC[gid];
    }
    __syncthreads();
    const int cnt = min(BS, n - b0);
    for (int j = cnt - 1; j >= 0; --j) {
      const int p = b0 + j;
      float v[9];
      bool contrib = false;
      if (p < static_cast<int>(L)) {
        const float4 A = sA[j];
        const float4 B = sB[j];
        float dx, dy;
        const float power = gauss_power(A, B.x, fx, fy, dx, dy);
        if (!(power > 0.0f || power < kPowerCut)) {
          const float e = __expf(power);
          const float araw = __fmul_rn(B.y, e);
          const float alpha = fminf(kAlphaMax, araw);
          if (!(alpha < kAlphaMin)) {
            contrib = true;
            const float4 Cc = sC[j];
            const float om = 1.0f - alpha;
            const float Ti = T / om;
            const float w = alpha * Ti;
            v[6] = g0 * w;
            v[7] = g1 * w;
            v[8] = g2 * w;
            const float gc = g0 * Cc.x + g1 * Cc.y + g2 * Cc.z;
            const float dalpha = gc * Ti - (S + bgg) / om;
            S += gc * w;
            T = Ti;
            const float da = (araw > kAlphaMax) ? 0.0f : dalpha;
            const float dpow = da * araw;
            v[5] = da * e;  // d opacity_t
            v[2] = -0.5f * dpow * dx * dx;
            v[3] = -dpow * dx * dy;
            v[4] = -0.5f * dpow * dy * dy;
            v[0] = dpow * (A.z * dx + A.w * dy);
            v[1] = dpow * (A.w * dx + B.x * dy);
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
        if (!contrib) {
#pragma unroll
          for (int k = 0; k < 9; ++k) v[k] = 0.0f;
        }
        // transpose reduction: values 0..7 end one per group of 4 lanes
        {
          const bool up = lane & 16;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float send = up ? v[k] : v[k + 4];
            const float keep = up ? v[k + 4] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
          }
        }
        {
          const bool up = lane & 8;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const float send = up ? v[k] : v[k + 2];
            const float keep = up ? v[k + 2] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
          }
        }
        {
          const bool up = lane & 4;
          const float send = up ? v[0] : v[1];
          const float keep = up ? v[1] : v[0];
          v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[8] += __shfl_xor_sync(0xffffffffu, v[8], o);
        const uint32_t gid = sG[j];
        float* dst = rgrad + static_cast<size_t>(gid) * 12;
        if ((lane & 3) == 0) {
          const int id = lane >> 2;  // value index 0..7
          atomicAdd(dst + (id < 6 ? id : id + 2), v[0]);
        }
        if (lane == 1) atomicAdd(dst + 10, v[8]);
      }
    }
  }
}

cudaError_t launch_blend_bwd(const FrameLayout& L, void* frame, const uint32_t* vals,
                             const float* bg, const float* grad_rgb, cudaStream_t s) {
  const float4* recA = at<float4>(frame, L.rec);
  const float4* recB = recA + L.n;
  const float4* recC = recB + L.n;
  const uint2* ranges = at<uint2>(frame, L.ranges);
  const float* T = at<float>(frame, L.tfinal);
  const uint32_t* last = at<uint32_t>(frame, L.last);
  float* rgrad = at<float>(frame, L.recgrad);
#define R4G_BLEND_BWD(TW_, TH_)                                                               \
  blend_bwd_kernel<TW_, TH_><<<L.ntiles, TW_ * TH_, 0, s>>>(ranges, vals, recA, recB, recC,   \
                                                             L.width, L.height, L.tiles_x,    \
                                                             bg[0], bg[1], bg[2], T, last,    \
                                                             grad_rgb, rgrad)
  if (L.tile_w == 16 && L.tile_h == 16) R4G_BLEND_BWD(16, 16);
  else if (L.tile_w == 8 && L.tile_h == 8) R4G_BLEND_BWD(8, 8);
  else if (L.tile_w == 16 && L.tile_h == 32) R4G_BLEND_BWD(16, 32);
  else return cudaErrorInvalidValue;
#undef R4G_BLEND_BWD
  return cudaGetLastError();
}

}  // namespace r4g
