// Single-kernel-per-pass stable LSD radix sort of (uint32 key, uint32 value)
// pairs for the render's two sorts (Gaussian depth keys, tile ids), after the
// "Onesweep" scheme: one histogram kernel counts the digits of every pass at
// once; each pass is then a single kernel in which a CTA
//   1. takes the next tile of 2048 items from an atomic ticket (so every tile
//      before it belongs to a CTA that is already running),
//   2. ranks its items stably by the pass's digit (the lanes holding the
//      same digit found by one warp ballot per digit bit, per-warp
//      histograms), publishes its per-digit counts,
//   3. looks back over the tiles before it, summing their published counts
//      until it meets a tile that has published its inclusive prefix, and
//      publishes its own prefix,
//   4. scatters its items, staged in shared memory in digit order, to
//      digit start + prefix + local rank.
// The look-back reads a window of 4 predecessors per round and backs off
// (32 ns doubling to 256 ns) after a round without progress: wider windows
// and tight polling measured slower, the statuses' cache lines being shared
// by every waiting CTA. It only waits on tiles that publish their counts
// before they wait themselves; each wait is bounded by an iteration limit
// after which the CTA sets an error bit in the frame header, treats the tile
// as empty and carries on (the image is then wrong and the status reports it,
// but nothing hangs). Counts and values are limited to 2^30. A launch sized
// for the key capacity has more CTAs than tiles; the surplus leaves at once.
#include <cuda_runtime.h>

#include "r4g.h"
#include "r4g_internal.cuh"
#include "onesweep.cuh"

namespace r4g {

constexpr int kOsHistCtas = 2 * 152;

// Digit histograms of every pass: hist[p * 256 + d] for digits of bits
// [8 p, 8 p + 8) of the keys, limited to `bits` bits in total (at most four
// passes). Shared-memory atomics into one sub-histogram per pair of warps,
// eight loads in flight per thread.
// kRel (the depth sort): digits of key - kmin, keys 0xffffffff not counted.
template <bool kRel>
__global__ void __launch_bounds__(kSortThreads)
    onesweep_hist_kernel(const uint32_t* __restrict__ keys, const uint32_t* count_dev, uint32_t count_host,
                         int passes, int bits, uint32_t* __restrict__ hist, const FrameHeader* hdr) {
  griddep_wait();
  griddep_launch_dependents();
  constexpr int NS = kSortThreads / 64;  // sub-histograms
  __shared__ uint32_t s_h[NS][4][kSortRadix];
  for (int k = threadIdx.x; k < NS * 4 * kSortRadix; k += kSortThreads) (&s_h[0][0][0])[k] = 0;
  __syncthreads();
  const uint32_t n = count_dev ? *count_dev : count_host;
  const uint32_t kmin = kRel ? ~hdr->dkey_minc : 0u;
  const int sub = threadIdx.x / 64;
  constexpr int ILP = 8;
  for (uint32_t base = blockIdx.x * kSortThreads * ILP; base < n; base += gridDim.x * kSortThreads * ILP) {
    uint32_t key[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint32_t i = base + u * kSortThreads + threadIdx.x;
      key[u] = i < n ? keys[i] : 0u;
    }
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      if (base + u * kSortThreads + threadIdx.x < n && (!kRel || key[u] != 0xffffffffu)) {
        const uint32_t r = key[u] - kmin;
        for (int p = 0; p < passes; ++p) {
          const int sh = p * kSortRadixBits;
          const int nb = min(kSortRadixBits, bits - sh);
          atomicAdd(&s_h[sub][p][(r >> sh) & ((1u << nb) - 1u)], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int p = 0; p < passes; ++p)
    for (int d = threadIdx.x; d < kSortRadix; d += kSortThreads) {
      uint32_t c = 0;
#pragma unroll
      for (int q = 0; q < NS; ++q) c += s_h[q][p][d];
      if (c) atomicAdd(&hist[p * kSortRadix + d], c);
    }
}

// kRel (the depth sort, pass `pass`): digits of key - kmin; the first pass
// drops keys 0xffffffff (its output holds the n_visible others, which the
// later passes sort); a pass beyond depth_passes(hdr) exits at once.
template <bool kRel>
__global__ void __launch_bounds__(kSortThreads, 5)
    onesweep_pass_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                         uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const uint32_t* count_dev,
                         uint32_t count_host, int shift, uint32_t mask, const uint32_t* __restrict__ hist,
                         uint32_t* status, uint32_t* ticket, uint32_t* err, uint32_t withheld_tile,
                         uint32_t spin_limit, const FrameHeader* hdr, int pass) {
  __shared__ uint32_t s_tile;
  __shared__ OsShared S;
  __shared__ uint32_t s_k[kOsTile];
  __shared__ uint32_t s_v[kOsTile];
  griddep_wait();
  griddep_launch_dependents();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t kmin = 0u;
  if constexpr (kRel) {
    if (pass >= depth_passes(hdr)) return;  // the key range is narrower: nothing left to sort
    kmin = ~hdr->dkey_minc;
  }
  const uint32_t n = kRel ? (pass == 0 ? count_host : hdr->n_visible) : (count_dev ? *count_dev : count_host);
  if (static_cast<uint64_t>(blockIdx.x) * kOsTile >= n) return;  // more CTAs than tiles: leave at once
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  os_clear(S);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t tb64 = static_cast<uint64_t>(t) * kOsTile;
  if (tb64 >= n) return;  // grid sized for the capacity; CTA-uniform exit
  const uint32_t tb = static_cast<uint32_t>(tb64);
  const uint32_t tn = min(static_cast<uint32_t>(kOsTile), n - tb);

  // ---- load and rank the tile (stable: warp w holds items [w*256, w*256+256))
  uint32_t k[kOsIPT], v[kOsIPT], d[kOsIPT];
#pragma unroll
  for (int j = 0; j < kOsIPT; ++j) {
    const uint32_t li = warp * (32 * kOsIPT) + j * 32 + lane;
    if (li < tn) {
      k[j] = kin[tb + li];
      v[j] = vin ? vin[tb + li] : tb + li;
      d[j] = (kRel && k[j] == 0xffffffffu) ? 0xffffffffu : ((k[j] - kmin) >> shift) & mask;
    } else {
      k[j] = 0;
      v[j] = 0;
      d[j] = 0xffffffffu;
    }
  }
  os_rank_scatter(k, v, d, t, n, kmin, shift, mask, hist, status, err, withheld_tile, spin_limit, S, s_k, s_v,
                  kout, vout);
}

// Clears what the passes expect at zero (instead of a memset, so that the
// sort's kernels follow one another with programmatic launches): the
// histograms unless the caller filled them, the tickets, and each pass's
// look-back statuses for the tiles the item count needs.
__global__ void onesweep_zero_kernel(uint32_t* __restrict__ hist, int hist_words, uint32_t* __restrict__ tickets,
                                     uint32_t* __restrict__ status, size_t pass_words, int passes,
                                     const uint32_t* count_dev, uint32_t count_host) {
  griddep_wait();
  griddep_launch_dependents();
  const uint32_t n = count_dev ? *count_dev : count_host;
  const size_t words = static_cast<size_t>((n + kOsTile - 1) / kOsTile) * kSortRadix;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  const size_t i0 = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (int p = 0; p < passes; ++p)
    for (size_t i = i0; i < words; i += stride) status[p * pass_words + i] = 0u;
  if (i0 < 32) tickets[i0] = 0u;
  for (size_t i = i0; i < static_cast<size_t>(hist_words); i += stride) hist[i] = 0u;
}

cudaError_t launch_depth_sort(const uint32_t* kin, uint32_t* kbuf1, uint32_t* vbuf1, uint32_t* kbuf2, uint32_t* vbuf2,
                              int64_t m, const FrameHeader* hdr, void* scratch, uint32_t* err, cudaStream_t s) {
  constexpr int passes = 32 / kSortRadixBits;
  if (m == 0) return cudaSuccess;
  const int64_t tiles = (m + kOsTile - 1) / kOsTile;
  uint32_t* hist = static_cast<uint32_t*>(scratch);
  uint32_t* tickets = hist + passes * kSortRadix;
  uint32_t* status = tickets + 32;
  const size_t pass_words = static_cast<size_t>(tiles) * kSortRadix;
  const int hist_ctas = static_cast<int>(tiles < kOsHistCtas ? tiles : kOsHistCtas);
  cudaError_t e = launch_pdl(onesweep_hist_kernel<true>, hist_ctas, kSortThreads, 0, s, kin,
                             static_cast<const uint32_t*>(nullptr), static_cast<uint32_t>(m), passes, 32, hist, hdr);
  const uint32_t* ki = kin;
  const uint32_t* vi = nullptr;
  for (int p = 0; p < passes && e == cudaSuccess; ++p) {
    uint32_t* ko = (p % 2 == 0) ? kbuf1 : kbuf2;
    uint32_t* vo = (p % 2 == 0) ? vbuf1 : vbuf2;
    e = launch_pdl(onesweep_pass_kernel<true>, static_cast<unsigned>(tiles), kSortThreads, 0, s, ki, vi, ko, vo,
                   static_cast<const uint32_t*>(nullptr), static_cast<uint32_t>(m), p * kSortRadixBits,
                   (1u << kSortRadixBits) - 1u, static_cast<const uint32_t*>(hist + p * kSortRadix),
                   status + static_cast<size_t>(p) * pass_words, tickets + p, err, 0xffffffffu, kSpinLimit, hdr, p);
    ki = ko;
    vi = vo;
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

uint32_t* onesweep_tickets(void* scratch, int bits) {
  const int passes = (bits + kSortRadixBits - 1) / kSortRadixBits;
  return static_cast<uint32_t*>(scratch) + passes * kSortRadix;
}

uint32_t* onesweep_status(void* scratch, int bits) { return onesweep_tickets(scratch, bits) + 32; }

size_t onesweep_scratch_bytes(int64_t cap, int bits) {
  const int passes = (bits + kSortRadixBits - 1) / kSortRadixBits;
  const int64_t tiles = (cap + kOsTile - 1) / kOsTile;
  return sizeof(uint32_t) * (static_cast<size_t>(passes) * kSortRadix       // histograms
                             + 32                                           // tickets
                             + static_cast<size_t>(passes) * tiles * kSortRadix);  // status
}

cudaError_t prepare_onesweep(void* scratch, int64_t cap, int bits, bool hist_ready, cudaStream_t s) {
  const int passes = (bits + kSortRadixBits - 1) / kSortRadixBits;
  if (passes == 0 || cap == 0) return cudaSuccess;
  const size_t hbytes = sizeof(uint32_t) * passes * kSortRadix;
  uint32_t* tickets = static_cast<uint32_t*>(scratch) + passes * kSortRadix;
  return hist_ready ? cudaMemsetAsync(tickets, 0, onesweep_scratch_bytes(cap, bits) - hbytes, s)
                    : cudaMemsetAsync(scratch, 0, onesweep_scratch_bytes(cap, bits), s);
}

cudaError_t launch_onesweep(const uint32_t* kin, const uint32_t* vin, uint32_t* kbuf1, uint32_t* vbuf1,
                            uint32_t* kbuf2, uint32_t* vbuf2, const uint32_t* count_dev, uint32_t count_host,
                            int64_t cap, int bits, void* scratch, uint32_t* err, cudaStream_t s,
                            int* result_in_buf, bool hist_ready, bool prepared, uint32_t withheld_tile,
                            uint32_t spin_limit, int first_pass) {
  const int passes = (bits + kSortRadixBits - 1) / kSortRadixBits;
  *result_in_buf = 0;
  if (passes == 0 || cap == 0) return cudaSuccess;
  const int64_t tiles = (cap + kOsTile - 1) / kOsTile;
  uint32_t* hist = static_cast<uint32_t*>(scratch);
  uint32_t* tickets = hist + passes * kSortRadix;
  uint32_t* status = tickets + 32;
  // the histograms either come ready (filled by the caller's kernels) or are
  // counted here; tickets and statuses always start at zero (cleared here
  // unless the caller did it with prepare_onesweep)
  const size_t pass_words = static_cast<size_t>(tiles) * kSortRadix;
  if (!prepared) {
    const cudaError_t e =
        launch_pdl(onesweep_zero_kernel, kOsHistCtas, kSortThreads, 0, s, hist, hist_ready ? 0 : passes * kSortRadix,
                   tickets, status, pass_words, passes, count_dev, count_host);
    if (e != cudaSuccess) return e;
  }
  if (!hist_ready) {
    const int hist_ctas = static_cast<int>(tiles < kOsHistCtas ? tiles : kOsHistCtas);
    const cudaError_t e = launch_pdl(onesweep_hist_kernel<false>, hist_ctas, kSortThreads, 0, s, kin, count_dev,
                                     count_host, passes, bits, hist, static_cast<const FrameHeader*>(nullptr));
    if (e != cudaSuccess) return e;
  }
  // passes before first_pass ran elsewhere (the emission runs the tile sort's
  // first): pass p writes buffer 1 when p is even, buffer 2 when odd
  int which = first_pass == 0 ? 0 : ((first_pass - 1) % 2 == 0 ? 1 : 2);
  const uint32_t* ki = which == 1 ? kbuf1 : which == 2 ? kbuf2 : kin;
  const uint32_t* vi = which == 1 ? vbuf1 : which == 2 ? vbuf2 : vin;
  for (int p = first_pass; p < passes; ++p) {
    const int shift = p * kSortRadixBits;
    const int nb = min(kSortRadixBits, bits - shift);
    uint32_t* ko = (which == 1) ? kbuf2 : kbuf1;
    uint32_t* vo = (which == 1) ? vbuf2 : vbuf1;
    const cudaError_t e =
        launch_pdl(onesweep_pass_kernel<false>, static_cast<unsigned>(tiles), kSortThreads, 0, s, ki, vi, ko, vo,
                   count_dev, count_host, shift, (1u << nb) - 1u, static_cast<const uint32_t*>(hist + p * kSortRadix),
                   status + static_cast<size_t>(p) * pass_words, tickets + p, err, withheld_tile,
                   spin_limit ? spin_limit : kSpinLimit, static_cast<const FrameHeader*>(nullptr), p);
    if (e != cudaSuccess) return e;
    ki = ko;
    vi = vo;
    which = (which == 1) ? 2 : 1;
  }
  *result_in_buf = which;
  return cudaGetLastError();
}

}  // namespace r4g

// ---- r4g_sort32: the render's sort as an entry point of its own ----------------
// scratch: [error word | pad to 256 B][keys n][values n][onesweep scratch]
namespace {
constexpr size_t kS32Align = 256;
size_t s32_al(size_t x) { return (x + kS32Align - 1) / kS32Align * kS32Align; }
size_t s32_bytes(int64_t n, int bits) {
  return kS32Align + 2 * s32_al(sizeof(uint32_t) * static_cast<size_t>(n)) + r4g::onesweep_scratch_bytes(n, bits);
}
r4g_status s32_fail(r4g_status st, const char* msg) {
  r4g::set_last_error(msg);
  return st;
}
r4g_status s32_run(const uint32_t* keys_in, const uint32_t* values_in, uint32_t* keys_out, uint32_t* values_out,
                   int64_t n, int32_t bits, void* scratch, size_t scratch_bytes, void* stream,
                   uint32_t withheld_tile, uint32_t spin_limit) {
  if (n < 0 || n >= (int64_t(1) << 30)) return s32_fail(R4G_EINVAL, "r4g_sort32: n out of range (< 2^30)");
  if (bits < 1 || bits > 32) return s32_fail(R4G_EINVAL, "r4g_sort32: bits must be in [1, 32]");
  if (!scratch || scratch_bytes < s32_bytes(n, bits)) return s32_fail(R4G_EWORKSPACE, "r4g_sort32: scratch too small");
  if (reinterpret_cast<uintptr_t>(scratch) % kS32Align) return s32_fail(R4G_EINVAL, "r4g_sort32: scratch not 256-byte aligned");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* err = static_cast<uint32_t*>(scratch);
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return s32_fail(R4G_ECUDA, cudaGetErrorString(e));
  if (n == 0) return R4G_OK;
  if (!keys_in || !keys_out || !values_out) return s32_fail(R4G_EINVAL, "r4g_sort32: NULL buffer");
  if (keys_in == keys_out || (values_in && values_in == values_out))
    return s32_fail(R4G_EINVAL, "r4g_sort32: outputs alias inputs");
  char* base = static_cast<char*>(scratch) + kS32Align;
  uint32_t* tk = reinterpret_cast<uint32_t*>(base);
  uint32_t* tv = reinterpret_cast<uint32_t*>(base + s32_al(sizeof(uint32_t) * n));
  void* os = base + 2 * s32_al(sizeof(uint32_t) * n);
  // pass p writes buffer 1 when p is even: an odd pass count ends in buffer 1
  const int passes = (bits + r4g::kSortRadixBits - 1) / r4g::kSortRadixBits;
  const bool odd = passes % 2 == 1;
  int which = 0;
  e = r4g::launch_onesweep(keys_in, values_in, odd ? keys_out : tk, odd ? values_out : tv, odd ? tk : keys_out,
                           odd ? tv : values_out, nullptr, static_cast<uint32_t>(n), n, bits, os, err, s, &which,
                           false, false, withheld_tile, spin_limit);
  if (e != cudaSuccess) return s32_fail(R4G_ECUDA, cudaGetErrorString(e));
  return R4G_OK;
}
}  // namespace

extern "C" r4g_status r4g_sort32_scratch_bytes(int64_t n, int32_t bits, size_t* bytes) {
  if (!bytes) return s32_fail(R4G_EINVAL, "r4g_sort32_scratch_bytes: NULL output");
  if (n < 0 || n >= (int64_t(1) << 30) || bits < 1 || bits > 32)
    return s32_fail(R4G_EINVAL, "r4g_sort32_scratch_bytes: n or bits out of range");
  *bytes = s32_bytes(n, bits);
  return R4G_OK;
}

extern "C" r4g_status r4g_sort32(const uint32_t* keys_in, const uint32_t* values_in, uint32_t* keys_out,
                                 uint32_t* values_out, int64_t n, int32_t bits, void* scratch, size_t scratch_bytes,
                                 void* stream) {
  return s32_run(keys_in, values_in, keys_out, values_out, n, bits, scratch, scratch_bytes, stream, 0xffffffffu, 0u);
}

extern "C" r4g_status r4g_sort32_wait_test(const uint32_t* keys_in, const uint32_t* values_in, uint32_t* keys_out,
                                           uint32_t* values_out, int64_t n, int32_t bits, void* scratch,
                                           size_t scratch_bytes, void* stream, uint32_t withheld_tile,
                                           uint32_t spin_limit) {
  if (spin_limit == 0 || spin_limit > (1u << 16))
    return s32_fail(R4G_EINVAL, "r4g_sort32_wait_test: spin_limit must be in [1, 65536]");
  return s32_run(keys_in, values_in, keys_out, values_out, n, bits, scratch, scratch_bytes, stream, withheld_tile,
                 spin_limit);
}

extern "C" r4g_status r4g_sort32_status(const void* scratch, void* stream) {
  if (!scratch) return s32_fail(R4G_EINVAL, "r4g_sort32_status: NULL scratch");
  uint32_t w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, scratch, sizeof(w), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return s32_fail(R4G_ECUDA, cudaGetErrorString(e));
  if (w & 2u) return s32_fail(R4G_ETIMEOUT, "r4g_sort32: a look-back wait ran out (the result is invalid)");
  return R4G_OK;
}
