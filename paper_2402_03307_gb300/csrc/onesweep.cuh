// Device side of the one-kernel-per-pass radix sort (see onesweep.cu): the
// look-back status flags, and the part of a pass that follows the loading of
// a tile -- stable ranking by the pass's digit, publication of the tile's
// digit counts, the bounded decoupled look-back for its exclusive prefix, and
// the scatter -- shared by the pass kernel and by the pair emission that runs
// the tile sort's first pass on the pairs it has just built.
#pragma once
#include <cstdint>

#include "r4g_internal.cuh"

namespace r4g {

constexpr uint32_t kFlagAgg = 1u << 30;     // tile count published
constexpr uint32_t kFlagPrefix = 2u << 30;  // inclusive prefix published
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr int kOsIPT = 8;                           // items per thread
constexpr int kOsTile = kSortThreads * kOsIPT;      // 2048 items per tile
constexpr int kOsWin = 4;                           // predecessors read per look-back round
constexpr int kOsWarps = kSortThreads / 32;

__device__ __forceinline__ uint32_t load_volatile(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void store_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Shared memory of a pass (besides the staging of keys and values).
struct OsShared {
  uint32_t dstart[kSortRadix];  // global start of each digit + tile prefix
  uint32_t tstart[kSortRadix];  // tile-local start of each digit
  uint32_t whist[kOsWarps][kSortRadix];
  uint32_t scan[kOsWarps];
  uint32_t tot;                 // items of the tile the pass keeps
};

// Zero the per-warp digit histograms (before the tile's ranking; the caller
// synchronises the CTA after it).
__device__ __forceinline__ void os_clear(OsShared& S) {
  for (int k = threadIdx.x; k < kOsWarps * kSortRadix; k += kSortThreads) (&S.whist[0][0])[k] = 0;
}

// The tile `t` of a pass, its items loaded: warp w holds items
// [w*256, w*256 + 256), item j*32 + lane of the warp in k[j], v[j] with
// digit d[j] (0xffffffff: no item, or an item the pass drops). Digits are
// (key - kmin) >> shift & mask. hist: the pass's digit totals over the
// kept items; n: items of the pass (positions are checked against it). Each
// wait of the look-back is bounded by spin_limit rounds without progress,
// after which err gets bit 2 (withheld_tile: a tile that never publishes, a
// test of that bound). s_k, s_v: 2048-entry staging arrays.
// kChain (the tile sort's second pass taken group by group): the look-back
// stops at tile chain0, the first tile of its chain, which publishes its
// count as its prefix; digit dd starts at dbase (thread dd's argument)
// instead of the histogram's exclusive scan, and dlive says whether any tile
// of the chain can hold it (hist is not read).
template <bool kChain = false>
__device__ __forceinline__ void os_rank_scatter(const uint32_t (&k)[kOsIPT], const uint32_t (&v)[kOsIPT],
                                                const uint32_t (&d)[kOsIPT], uint32_t t, uint32_t n, uint32_t kmin,
                                                int shift, uint32_t mask, const uint32_t* __restrict__ hist,
                                                uint32_t* status, uint32_t* err, uint32_t withheld_tile,
                                                uint32_t spin_limit, OsShared& S, uint32_t* s_k, uint32_t* s_v,
                                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                uint32_t chain0 = 0u, uint32_t dbase = 0u, bool dlive = false) {
  constexpr int NW = kOsWarps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t rk[kOsIPT];
#pragma unroll
  for (int j = 0; j < kOsIPT; ++j) {
    const bool ok = d[j] != 0xffffffffu;
    const uint32_t act = __ballot_sync(0xffffffffu, ok);
    rk[j] = 0;
    uint32_t peers = act;
#pragma unroll
    for (int b = 0; b < kSortRadixBits; ++b) {
      const uint32_t bit = (d[j] >> b) & 1u;
      const uint32_t bal = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bal : ~bal;
    }
    if (ok) {
      const uint32_t base = S.whist[warp][d[j]];
      __syncwarp(act);
      if (lane == __ffs(peers) - 1) S.whist[warp][d[j]] = base + __popc(peers);
      rk[j] = base + __popc(peers & lt_mask);
    }
    __syncwarp();
  }
  __syncthreads();
  // per digit (thread = digit): exclusive over warps, tile count
  const int dd = threadIdx.x;
  uint32_t cnt = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint32_t c = S.whist[w][dd];
    S.whist[w][dd] = cnt;
    cnt += c;
  }
  // ---- publish the tile's count, then look back for its exclusive prefix
  // (a digit no item of the pass has -- the histogram says so -- needs no
  // status and no look-back: its count is zero in every tile)
  const uint32_t h = kChain ? 0u : hist[dd];
  const bool live = kChain ? dlive : h != 0u;
  // withheld_tile (a test of the bounded wait only; otherwise no tile): that
  // tile never publishes, so its successors' waits run out
  const bool publish = t != withheld_tile;
  uint32_t* st = status + static_cast<size_t>(t) * kSortRadix;
  if (live && publish) store_relaxed(st + dd, (t == chain0 ? kFlagPrefix : kFlagAgg) | cnt);
  // Look-back, kOsWin predecessors per round (their statuses are read in
  // parallel): add published counts newest first until a published prefix;
  // a round that makes no progress counts against the spin limit.
  uint32_t excl = 0;
  if (t > chain0 && live) {
    constexpr int WIN = kOsWin;
    const int64_t k0 = static_cast<int64_t>(chain0);
    int64_t kt = static_cast<int64_t>(t) - 1;
    uint32_t idle = 0, nap = 32u;
    bool found = false;
    while (!found && kt >= k0) {
      uint32_t sv[WIN];
#pragma unroll
      for (int w = 0; w < WIN; ++w)
        sv[w] = (kt - w >= k0) ? load_volatile(status + static_cast<size_t>(kt - w) * kSortRadix + dd) : kFlagPrefix;
      int used = 0;
#pragma unroll
      for (int w = 0; w < WIN; ++w) {
        if (found || used < w) continue;           // stopped earlier in this window
        if ((sv[w] & ~kValMask) == 0u) continue;   // not ready: retry from here
        if (kt - w >= k0) excl += sv[w] & kValMask;
        ++used;
        if (sv[w] & kFlagPrefix) found = true;
      }
      kt -= used;
      if (used == 0) {
        if (++idle >= spin_limit) {  // gave up: record it and go on
          atomicOr(err, 2u);
          break;
        }
        __nanosleep(nap);
        nap = nap < 256u ? 2u * nap : 256u;
      }
    }
    if (publish) store_relaxed(st + dd, kFlagPrefix | (excl + cnt));
  }
  // global digit start: exclusive scan of this pass's histogram (+ tile prefix)
  {
    uint32_t x = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) S.scan[warp] = x;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < warp; ++w) pre += S.scan[w];
    S.dstart[dd] = (kChain ? dbase : pre + x - h) + excl;
    __syncthreads();
    // tile-local digit starts: exclusive scan of the tile counts
    x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) S.scan[warp] = x;
    __syncthreads();
    pre = 0;
    for (int w = 0; w < warp; ++w) pre += S.scan[w];
    S.tstart[dd] = pre + x - cnt;
    if (dd == kSortRadix - 1) S.tot = pre + x;  // items of the tile this pass keeps
  }
  __syncthreads();
  // ---- stage in digit order, then write each digit's run contiguously
#pragma unroll
  for (int j = 0; j < kOsIPT; ++j) {
    if (d[j] != 0xffffffffu) {
      const uint32_t pos = S.tstart[d[j]] + S.whist[warp][d[j]] + rk[j];
      s_k[pos] = k[j];
      s_v[pos] = v[j];
    }
  }
  __syncthreads();
  const uint32_t tk = S.tot;
  for (uint32_t i = threadIdx.x; i < tk; i += kSortThreads) {
    const uint32_t key = s_k[i];
    const uint32_t dg = ((key - kmin) >> shift) & mask;
    const uint32_t o = S.dstart[dg] + i - S.tstart[dg];
    if (o < n) {  // only false after a key-capacity overflow, whose result is discarded
      kout[o] = key;
      vout[o] = s_v[i];
    }
  }
}

}  // namespace r4g
