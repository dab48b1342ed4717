// Tile binning of the rasteriser (Sec. 3.1): the exclusive scan of the
// per-Gaussian tile counts, the emission of one 64-bit key per (tile,
// Gaussian) pair -- key = tile_id << 32 | float_bits(depth), value = Gaussian
// index, in Gaussian-index order and row-major tile order within a Gaussian --
// and the per-tile [begin, end) ranges of the sorted key list.
#include <cuda_runtime.h>

#include "r4g_internal.cuh"

namespace r4g {

constexpr int kScanThreads = 1024;

// Exclusive scan of the per-block tile totals in place (one CTA); writes the
// pair count and the overflow flag into the frame header.
__global__ void __launch_bounds__(kScanThreads)
    scan_blocksums_kernel(uint32_t* blocksum, int nblocks, FrameHeader* hdr, uint32_t cap) {
  __shared__ uint32_t s_warp[kScanThreads / 32];
  __shared__ uint32_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < nblocks; base += kScanThreads) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < nblocks ? blocksum[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      s_warp[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t carry = s_carry;
    const uint32_t excl = carry + (warp ? s_warp[warp - 1] : 0u) + x - v;
    if (i < nblocks) blocksum[i] = excl;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) s_carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const uint32_t total = s_carry;
    hdr->key_needed = total;
    hdr->key_count = total < cap ? total : cap;
    if (total > cap) hdr->status |= 1u;
  }
}

// One thread per Gaussian (same blocking as the preprocess); each warp emits
// the keys of its 32 Gaussians cooperatively, 32 consecutive keys per step,
// so the writes are coalesced and a Gaussian with many tiles does not stall
// one lane.
__global__ void __launch_bounds__(kPreBlock)
    keybuild_kernel(const uint32_t* __restrict__ touched, const uint32_t* __restrict__ blockoff,
                    const uint2* __restrict__ rect, const float4* __restrict__ recB, int n,
                    int tiles_x, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                    uint32_t cap) {
  __shared__ uint32_t s_warp[kPreBlock / 32];
  const int i = blockIdx.x * kPreBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t cnt = i < n ? touched[i] : 0u;
  uint32_t x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint32_t wbase = blockoff[blockIdx.x];
  for (int w = 0; w < warp; ++w) wbase += s_warp[w];
  const uint32_t excl = x - cnt;  // within the warp
  const uint32_t wtotal = __shfl_sync(0xffffffffu, x, 31);
  uint2 r = make_uint2(0u, 0u);
  uint32_t zb = 0;
  if (cnt) {
    r = rect[i];
    zb = __float_as_uint(recB[i].z);
  }
  for (uint32_t j0 = 0; j0 < wtotal; j0 += 32) {
    const uint32_t j = j0 + lane;
    // owner = the last lane whose exclusive offset is <= j
    int own = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const uint32_t e = __shfl_sync(0xffffffffu, excl, own + step);
      if (e <= j) own += step;
    }
    const uint32_t oex = __shfl_sync(0xffffffffu, excl, own);
    const uint32_t orx = __shfl_sync(0xffffffffu, r.x, own);
    const uint32_t ory = __shfl_sync(0xffffffffu, r.y, own);
    const uint32_t oz = __shfl_sync(0xffffffffu, zb, own);
    if (j < wtotal) {
      const uint32_t local = j - oex;
      const uint32_t x0 = orx & 0xffffu, y0 = orx >> 16, x1 = ory & 0xffffu;
      const uint32_t w = x1 - x0;
      const uint32_t ty = y0 + local / w, tx = x0 + local % w;
      const uint32_t pos = wbase + j;
      if (pos < cap) {
        keys[pos] = (static_cast<uint64_t>(ty * static_cast<uint32_t>(tiles_x) + tx) << 32) | oz;
        vals[pos] = static_cast<uint32_t>(blockIdx.x * kPreBlock + warp * 32 + own);
      }
    }
  }
}

// ranges[tile] = [first, last+1) of the tile's keys in the sorted list.
__global__ void ranges_kernel(const uint64_t* __restrict__ keys, const FrameHeader* hdr,
                              uint2* __restrict__ ranges) {
  const uint32_t n = hdr->key_count;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t tile = static_cast<uint32_t>(keys[i] >> 32);
    if (i == 0 || static_cast<uint32_t>(keys[i - 1] >> 32) != tile) ranges[tile].x = i;
    if (i == n - 1 || static_cast<uint32_t>(keys[i + 1] >> 32) != tile) ranges[tile].y = i + 1;
  }
}

cudaError_t launch_binning(const FrameLayout& L, void* frame, cudaStream_t s) {
  if (L.n == 0) return cudaSuccess;
  FrameHeader* hdr = at<FrameHeader>(frame, L.header);
  uint32_t* bs = at<uint32_t>(frame, L.blocksum);
  scan_blocksums_kernel<<<1, kScanThreads, 0, s>>>(bs, L.nblocks, hdr, static_cast<uint32_t>(L.cap));
  const float4* recB = at<float4>(frame, L.rec) + L.n;
  keybuild_kernel<<<L.nblocks, kPreBlock, 0, s>>>(
      at<uint32_t>(frame, L.touched), bs, at<uint2>(frame, L.rect), recB, static_cast<int>(L.n),
      L.tiles_x, at<uint64_t>(frame, L.keys0), at<uint32_t>(frame, L.vals0),
      static_cast<uint32_t>(L.cap));
  return cudaGetLastError();
}

cudaError_t launch_ranges(const FrameLayout& L, void* frame, const uint64_t* keys, cudaStream_t s) {
  uint2* ranges = at<uint2>(frame, L.ranges);
  cudaMemsetAsync(ranges, 0, sizeof(uint2) * L.ntiles, s);
  if (L.n == 0) return cudaGetLastError();
  ranges_kernel<<<4 * 152, 256, 0, s>>>(keys, at<FrameHeader>(frame, L.header), ranges);
  return cudaGetLastError();
}

}  // namespace r4g
