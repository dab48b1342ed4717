// Stable LSD radix sort of (key, uint32 value) pairs, keys of 64, 32 or 16
// bits, up to 8-bit digits, reduce-then-scan per pass (no inter-CTA waits):
//   upsweep   : each CTA counts the digits of its contiguous chunk
//   scan      : one CTA turns the [digit][cta] counts into global offsets
//   downsweep : each CTA ranks its chunk tile by tile (stable: warp match +
//               per-warp histograms), stages the tile in shared memory in
//               digit order and writes each digit's run contiguously.
// The pair count may live in device memory (a render's key count), so the
// grid is fixed and every CTA derives its chunk from the count at run time.
// A NULL value input stands for the values 0, 1, 2, ... (the first pass of
// an index sort generates them instead of reading them).
#include <cuda_runtime.h>

#include "r4g_internal.cuh"

namespace r4g {

__device__ __forceinline__ uint32_t load_count(const uint32_t* dev, uint32_t host) {
  return dev ? *dev : host;
}

__device__ __forceinline__ void chunk_of(uint32_t n, int ctas, uint32_t& begin, uint32_t& end) {
  const uint32_t per = (n + ctas - 1) / ctas;
  const uint32_t chunk = ((per + kSortTile - 1) / kSortTile) * kSortTile;
  const uint64_t b = static_cast<uint64_t>(blockIdx.x) * chunk;
  begin = b < n ? static_cast<uint32_t>(b) : n;
  const uint64_t e = b + chunk;
  end = e < n ? static_cast<uint32_t>(e) : n;
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift, uint32_t mask) {
  return static_cast<uint32_t>(k >> shift) & mask;
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
    radix_upsweep_kernel(const K* __restrict__ keys, const uint32_t* count_dev, uint32_t count_host,
                         int shift, uint32_t mask, uint32_t* __restrict__ counts, int ctas) {
  constexpr int NW = kSortThreads / 32;
  constexpr int ILP = 8;
  __shared__ uint32_t s_hist[NW][kSortRadix];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < NW * kSortRadix; k += kSortThreads) (&s_hist[0][0])[k] = 0;
  __syncthreads();
  const uint32_t n = load_count(count_dev, count_host);
  uint32_t begin, end;
  chunk_of(n, ctas, begin, end);
  // the loop bounds are uniform over the CTA, so every warp takes part in
  // every ballot; ILP independent loads are issued before any is used
  for (uint32_t base = begin; base < end; base += kSortThreads * ILP) {
    uint32_t d[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint32_t i = base + u * kSortThreads + threadIdx.x;
      d[u] = i < end ? digit_of<K>(keys[i], shift, mask) : 0xffffffffu;
    }
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const bool ok = d[u] != 0xffffffffu;
      const uint32_t act = __ballot_sync(0xffffffffu, ok);
      if (ok) {
        const uint32_t peers = __match_any_sync(act, d[u]);
        if (lane == __ffs(peers) - 1) atomicAdd(&s_hist[warp][d[u]], __popc(peers));
      }
    }
  }
  __syncthreads();
  for (int dd = threadIdx.x; dd < kSortRadix; dd += kSortThreads) {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) c += s_hist[w][dd];
    counts[dd * ctas + blockIdx.x] = c;
  }
}

// Exclusive scan of counts[0 .. total) in place (digit-major), one CTA.
// Each thread owns a contiguous segment of total / kScanT entries (a
// multiple of 4, see sort_ctas_for) read as 16-byte vectors, eight loads in
// flight at a time; the segment is read again (from L2) for the write-back.
constexpr int kScanT = 1024;
__global__ void __launch_bounds__(kScanT) radix_scan_kernel(uint32_t* counts, int total) {
  __shared__ uint32_t s_warp[kScanT / 32];
  const int per = total / kScanT;  // entries per thread, multiple of 4
  const int nvec = per / 4;
  uint4* seg = reinterpret_cast<uint4*>(counts + static_cast<size_t>(threadIdx.x) * per);
  uint32_t sum = 0;
#pragma unroll 8
  for (int k = 0; k < nvec; ++k) {
    const uint4 v = seg[k];
    sum += v.x + v.y + v.z + v.w;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = sum;
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
    s_warp[lane] = w;
  }
  __syncthreads();
  uint32_t run = (warp ? s_warp[warp - 1] : 0u) + x - sum;
#pragma unroll 8
  for (int k = 0; k < nvec; ++k) {
    const uint4 v = seg[k];
    uint4 o;
    o.x = run; run += v.x;
    o.y = run; run += v.y;
    o.z = run; run += v.z;
    o.w = run; run += v.w;
    seg[k] = o;
  }
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
    radix_downsweep_kernel(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                           K* __restrict__ kout, uint32_t* __restrict__ vout,
                           const uint32_t* count_dev, uint32_t count_host, int shift,
                           uint32_t mask, const uint32_t* __restrict__ offsets, int ctas) {
  constexpr int NW = kSortThreads / 32;
  __shared__ uint32_t s_goff[kSortRadix];
  __shared__ uint32_t s_tstart[kSortRadix];
  __shared__ uint32_t s_tcount[kSortRadix];
  __shared__ uint32_t s_whist[NW][kSortRadix];
  __shared__ uint32_t s_scan[NW];
  __shared__ K s_k[kSortTile];
  __shared__ uint32_t s_v[kSortTile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t n = load_count(count_dev, count_host);
  uint32_t begin, end;
  chunk_of(n, ctas, begin, end);
  for (int d = threadIdx.x; d < kSortRadix; d += kSortThreads) s_goff[d] = offsets[d * ctas + blockIdx.x];

  for (uint32_t tb = begin; tb < end; tb += kSortTile) {
    const uint32_t tn = min(static_cast<uint32_t>(kSortTile), end - tb);
    for (int k = threadIdx.x; k < NW * kSortRadix; k += kSortThreads) (&s_whist[0][0])[k] = 0;
    __syncthreads();
    K k[kSortIPT];
    uint32_t v[kSortIPT], d[kSortIPT], rk[kSortIPT];
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
      const uint32_t li = warp * (32 * kSortIPT) + j * 32 + lane;
      const bool ok = li < tn;
      if (ok) {
        k[j] = kin[tb + li];
        v[j] = vin ? vin[tb + li] : tb + li;
        d[j] = digit_of<K>(k[j], shift, mask);
      } else {
        k[j] = 0;
        v[j] = 0;
        d[j] = 0xffffffffu;
      }
    }
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
      const bool ok = d[j] != 0xffffffffu;
      const uint32_t act = __ballot_sync(0xffffffffu, ok);
      rk[j] = 0;
      if (ok) {
        const uint32_t peers = __match_any_sync(act, d[j]);
        const uint32_t base = s_whist[warp][d[j]];
        __syncwarp(act);
        if (lane == __ffs(peers) - 1) s_whist[warp][d[j]] = base + __popc(peers);
        rk[j] = base + __popc(peers & lt_mask);
      }
      __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive over warps, and the tile's count
    for (int dd = threadIdx.x; dd < kSortRadix; dd += kSortThreads) {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t c = s_whist[w][dd];
        s_whist[w][dd] = run;
        run += c;
      }
      s_tcount[dd] = run;
    }
    __syncthreads();
    // exclusive scan of the 256 tile counts (kSortThreads == kSortRadix)
    {
      const uint32_t c = s_tcount[threadIdx.x];
      uint32_t x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_scan[warp] = x;
      __syncthreads();
      uint32_t pre = 0;
      for (int w = 0; w < warp; ++w) pre += s_scan[w];
      s_tstart[threadIdx.x] = pre + x - c;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
      if (d[j] != 0xffffffffu) {
        const uint32_t pos = s_tstart[d[j]] + s_whist[warp][d[j]] + rk[j];
        s_k[pos] = k[j];
        s_v[pos] = v[j];
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tn; i += kSortThreads) {
      const K key = s_k[i];
      const uint32_t dg = digit_of<K>(key, shift, mask);
      const uint32_t o = s_goff[dg] + i - s_tstart[dg];
      kout[o] = key;
      vout[o] = s_v[i];
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < kSortRadix; dd += kSortThreads) s_goff[dd] += s_tcount[dd];
    __syncthreads();
  }
}

// CTAs per pass: enough for the capacity, at most two per SM, and a multiple
// of 16 so that the scan's per-thread segment (256 * ctas / 1024 entries) is
// a whole number of 16-byte vectors.
int sort_ctas_for(int64_t cap) {
  const int64_t tiles = (cap + kSortTile - 1) / kSortTile;
  int64_t c = tiles < kSortMaxCtas ? tiles : kSortMaxCtas;
  c = (c + 15) / 16 * 16;
  return static_cast<int>(c < 16 ? 16 : c);
}

template <typename K>
static cudaError_t sort_passes(const K* kin, const uint32_t* vin, K* kbuf1, uint32_t* vbuf1, K* kbuf2,
                               uint32_t* vbuf2, const uint32_t* count_dev, uint32_t count_host,
                               int begin_bit, int end_bit, uint32_t* counts, int ctas,
                               cudaStream_t s, int* result_in_buf) {
  const K* ki = kin;
  const uint32_t* vi = vin;
  int which = 0;
  for (int shift = begin_bit; shift < end_bit; shift += kSortRadixBits) {
    const int bits = min(kSortRadixBits, end_bit - shift);
    const uint32_t mask = (1u << bits) - 1u;
    K* ko = (which == 1) ? kbuf2 : kbuf1;
    uint32_t* vo = (which == 1) ? vbuf2 : vbuf1;
    radix_upsweep_kernel<K><<<ctas, kSortThreads, 0, s>>>(ki, count_dev, count_host, shift, mask, counts, ctas);
    radix_scan_kernel<<<1, kScanT, 0, s>>>(counts, kSortRadix * ctas);
    radix_downsweep_kernel<K><<<ctas, kSortThreads, 0, s>>>(ki, vi, ko, vo, count_dev, count_host, shift, mask,
                                                             counts, ctas);
    ki = ko;
    vi = vo;
    which = (which == 1) ? 2 : 1;
  }
  *result_in_buf = which;
  return cudaGetLastError();
}

// Sorts bits [begin_bit, end_bit). Pass p reads the previous pass's output
// (p == 0: kin/vin) and writes buffer 1 when p is even, buffer 2 when odd;
// *result_in_buf receives 1 or 2 (or 0 when no pass ran).
cudaError_t launch_sort(const uint64_t* kin, const uint32_t* vin, uint64_t* kbuf1, uint32_t* vbuf1,
                        uint64_t* kbuf2, uint32_t* vbuf2, const uint32_t* count_dev, uint32_t count_host,
                        int64_t cap, int begin_bit, int end_bit, uint32_t* counts, int ctas,
                        cudaStream_t s, int* result_in_buf) {
  (void)cap;
  return sort_passes<uint64_t>(kin, vin, kbuf1, vbuf1, kbuf2, vbuf2, count_dev, count_host, begin_bit, end_bit,
                               counts, ctas, s, result_in_buf);
}

}  // namespace r4g
