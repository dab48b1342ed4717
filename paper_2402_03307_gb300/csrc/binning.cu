// Tile binning of the rasteriser (Sec. 3.1). The (view, Gaussian) items of
// all the views of a call are first put in depth order (a stable radix sort
// of their depth bits, ties by item index), then one (tile, item) pair is
// emitted per tile an item's box covers, in that order and row-major within
// an item. Tile ids are global over the views, so a tile's pairs all come
// from one view, and a stable sort of the pairs by tile id gives, bit for
// bit, the order of a stable sort of 64-bit keys tile_id << 32 |
// float_bits(depth) emitted in Gaussian-index order, view by view.
// This file holds: the per-block totals of tile counts in depth order, their
// exclusive scan, per-item offsets (in depth order and by item), the
// emission balanced over the output pairs, the per-view tile counts -> the
// [begin, end) ranges of the sorted list, and the export of the equivalent
// 64-bit keys.
#include <cuda_runtime.h>

#include "r4g_internal.cuh"
#include "onesweep.cuh"
#include "tile_rows.cuh"

namespace r4g {

constexpr int kScanThreads = 1024;
constexpr int kTileCountsMaxSmem = kMaxTiles * 4;
constexpr int kTileClasses = 64;  // list-length classes of the blend's tile order

// blocksum[b] = sum of touched[order[j]] over the block's depth positions.
// The depth order holds the hdr->n_visible items with tiles; it ends in
// ord_odd when the depth sort ran an odd number of passes, else in ord_even.
__device__ __forceinline__ const uint32_t* depth_order(const uint32_t* ord_odd, const uint32_t* ord_even,
                                                       const FrameHeader* hdr) {
  return (depth_passes(hdr) & 1) ? ord_odd : ord_even;
}

__global__ void __launch_bounds__(kPreBlock)
    depth_blocksum_kernel(const uint32_t* __restrict__ touched, const uint32_t* ord_odd, const uint32_t* ord_even,
                          const FrameHeader* hdr, uint32_t* __restrict__ blocksum) {
  griddep_wait();
  griddep_launch_dependents();
  __shared__ uint32_t s_sum[kPreBlock / 32];
  const uint32_t* __restrict__ order = depth_order(ord_odd, ord_even, hdr);
  const int nk = static_cast<int>(hdr->n_visible);
  const int j = blockIdx.x * kPreBlock + threadIdx.x;
  const uint32_t c = j < nk ? touched[order[j]] : 0u;
  const uint32_t ws = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0;
#pragma unroll
    for (int w = 0; w < kPreBlock / 32; ++w) a += s_sum[w];
    blocksum[blockIdx.x] = a;
  }
}

// Exclusive scan of the per-block totals in place (one CTA); writes the pair
// count and the overflow flag into the frame header.
__global__ void __launch_bounds__(kScanThreads)
    scan_blocksums_kernel(uint32_t* blocksum, int nblocks, FrameHeader* hdr, uint32_t cap) {
  griddep_wait();
  griddep_launch_dependents();
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

// Exclusive offset of every Gaussian's first pair, in depth order, and its
// tile rectangle gathered into depth order (same blocking as
// depth_blocksum_kernel; blockoff holds the scanned block totals).
constexpr int kEmitChunk = 2048;

// kSelfScan (a call with at most kSelfScanBlocks blocks): blockoff holds the
// unscanned block totals, and each block sums those before it itself (the
// one-CTA scan launch is skipped); the last block writes the pair count and
// the overflow flag into the frame header, as scan_blocksums_kernel does.

template <bool kSelfScan>
__global__ void __launch_bounds__(kPreBlock)
    depth_offsets_kernel(const uint32_t* __restrict__ touched, const uint32_t* ord_odd, const uint32_t* ord_even,
                         const uint32_t* __restrict__ blockoff, const uint2* __restrict__ rect,
                         const ViewDev* __restrict__ views, uint32_t ng, int m, uint32_t* __restrict__ offs,
                         uint32_t* __restrict__ ioffs, uint4* __restrict__ srect, uint32_t* __restrict__ chunk_start,
                         uint32_t nchunks, FrameHeader* hdr, uint32_t cap) {
  griddep_wait();
  griddep_launch_dependents();
  __shared__ uint32_t s_warp[kPreBlock / 32];
  __shared__ uint32_t s_pre[kPreBlock / 32];
  const int j = blockIdx.x * kPreBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t pre = 0;  // kSelfScan: this thread's share of the blocks before this one
  if constexpr (kSelfScan)
    for (int b = threadIdx.x; b < static_cast<int>(blockIdx.x); b += kPreBlock) pre += blockoff[b];
  const uint32_t* __restrict__ order = depth_order(ord_odd, ord_even, hdr);
  const int nk = static_cast<int>(hdr->n_visible);  // the depth order's length (<= m)
  const uint32_t item = j < nk ? order[j] : 0u;
  const uint32_t cnt = j < nk ? touched[item] : 0u;
  uint32_t x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  if constexpr (kSelfScan) {
    pre = __reduce_add_sync(0xffffffffu, pre);
    if (lane == 0) s_pre[warp] = pre;
  }
  __syncthreads();
  uint32_t base;
  if constexpr (kSelfScan) {
    base = 0;
#pragma unroll
    for (int w = 0; w < kPreBlock / 32; ++w) base += s_pre[w];
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {  // the pair count of the call
      uint32_t total = base;
#pragma unroll
      for (int w = 0; w < kPreBlock / 32; ++w) total += s_warp[w];
      hdr->key_needed = total;
      hdr->key_count = total < cap ? total : cap;
      if (total > cap) atomicOr(&hdr->status, 1u);
    }
  } else {
    base = blockoff[blockIdx.x];
  }
  for (int w = 0; w < warp; ++w) base += s_warp[w];
  if (j < m) {
    const uint32_t o = base + x - cnt;
    offs[j] = o;
    if (cnt) {
      ioffs[item] = o;
      const ViewDev& V = views[item / ng];
      const uint2 r = rect[item];
      srect[j] = make_uint4(r.x, r.y, V.tile_off, static_cast<uint32_t>(V.tiles_x));
    } else {
      srect[j] = make_uint4(0u, 0u, 0u, 1u);
    }
    // this item owns the first pair of every emission chunk starting in [o, o + cnt)
    for (uint32_t c = (o + kEmitChunk - 1) / kEmitChunk; cnt && c * kEmitChunk < o + cnt && c < nchunks; ++c)
      chunk_start[c] = static_cast<uint32_t>(j);
  }
}

// Pair emission balanced over the output: chunk c holds pairs
// [c E, (c + 1) E) of the depth-ordered list (CTAs stride over the chunks). Gaussians with pairs are at the
// front of the depth order (a Gaussian without tiles has the largest key), so
// their offsets increase strictly and a chunk of E pairs involves at most
// E + 1 of them: their offsets are loaded into shared memory. Each thread
// emits a run of E / 256 consecutive pairs: one binary search finds the
// Gaussian of the run's first pair, later pairs step through its tiles and on
// into the next Gaussian. Pair q of Gaussian j is its l-th tile, l = q -
// offs[j], counting the intervals of its tile rows top to bottom (emit_run).
// The runs are
// staged in shared memory (slots swizzled so that neither the run-wise writes
// nor the pair-wise reads meet bank conflicts) and written out coalesced. The
// Gaussian holding the chunk's first pair comes from depth_offsets_kernel.
constexpr int kEmitRun = kEmitChunk / kPreBlock;  // consecutive pairs per thread
static_assert(kEmitChunk % kPreBlock == 0 && kEmitRun == 8, "the slot swizzle assumes runs of 8");

__device__ __forceinline__ uint32_t emit_slot(uint32_t i) { return i ^ ((i >> 5) & 7u); }

// A Gaussian's pairs in emission order: tile rows top to bottom, in each the
// interval of columns its contributing ellipse meets, as the preprocess
// stored them (tile_rows.cuh; every column of the row for a rectangle too
// large to store spans for).
struct EmitG {
  uint32_t tile_off, tiles_x, gid;
  int x0, x1, y0, y1;
  bool span;
  uint4 s0, s1;  // 16 rows x (first column - x0, width) bytes
  int k, c1, col;  // current row (relative to y0), its last column, the current column
};

__device__ __forceinline__ uint32_t span_word(const EmitG& G, int w) {
  switch (w) {
    case 0: return G.s0.x;
    case 1: return G.s0.y;
    case 2: return G.s0.z;
    case 3: return G.s0.w;
    case 4: return G.s1.x;
    case 5: return G.s1.y;
    case 6: return G.s1.z;
    default: return G.s1.w;
  }
}

// First column and width of row k.
__device__ __forceinline__ void span_row(const EmitG& G, int k, int& c0, int& w) {
  if (!G.span) {
    c0 = G.x0;
    w = G.x1 - G.x0;
    return;
  }
  const uint32_t h = span_word(G, k >> 1) >> (16 * (k & 1));
  c0 = G.x0 + static_cast<int>(h & 0xffu);
  w = static_cast<int>((h >> 8) & 0xffu);
}

__device__ __forceinline__ void emit_load(EmitG& G, uint4 r, uint32_t gid, const uint4* __restrict__ spans) {
  G.tile_off = r.z;
  G.tiles_x = r.w;
  G.gid = gid;
  G.x0 = static_cast<int>(r.x & 0xffffu);
  G.x1 = static_cast<int>(r.y & 0xffffu);
  G.y0 = static_cast<int>(r.x >> 16);
  G.y1 = static_cast<int>(r.y >> 16);
  G.span = span_mode(G.x0, G.x1, G.y0, G.y1);
  if (G.span) {
    G.s0 = spans[2 * static_cast<size_t>(gid)];
    G.s1 = spans[2 * static_cast<size_t>(gid) + 1];
  }
}

// Place G on its pair l.
__device__ __forceinline__ void emit_locate(EmitG& G, uint32_t l) {
  const int rows = G.y1 - G.y0;
  if (!G.span) {
    const uint32_t w = static_cast<uint32_t>(G.x1 - G.x0);
    G.k = static_cast<int>(l / w);
    G.col = G.x0 + static_cast<int>(l - static_cast<uint32_t>(G.k) * w);
    G.c1 = G.x1 - 1;
    return;
  }
  for (G.k = 0; G.k < rows; ++G.k) {
    int c0, w;
    span_row(G, G.k, c0, w);
    if (l < static_cast<uint32_t>(w)) {
      G.col = c0 + static_cast<int>(l);
      G.c1 = c0 + w - 1;
      return;
    }
    l -= static_cast<uint32_t>(w);
  }
  G.k = rows - 1;  // unreachable when the counts agree; stays inside the rectangle
  G.col = G.c1 = G.x0;
}

// The next pair of G (rows with tiles are consecutive).
__device__ __forceinline__ void emit_step(EmitG& G) {
  if (++G.col <= G.c1) return;
  const int rows = G.y1 - G.y0;
  while (++G.k < rows) {
    int c0, w;
    span_row(G, G.k, c0, w);
    if (w > 0) {
      G.col = c0;
      G.c1 = c0 + w - 1;
      return;
    }
  }
  G.k = rows - 1;  // past the Gaussian's last pair: the caller moves to the next one
  G.col = G.c1;
}

// The thread's run of kEmitRun pairs qa, qa + 1, ... (< qend) of an
// emission chunk starting at q0: one binary search for the run's first
// Gaussian among the chunk's window of items (offsets s_off, m of them),
// then a step through its row intervals and on into the next Gaussian;
// tile ids and items staged in swizzled slots.
__device__ __forceinline__ void emit_run(uint32_t qa, uint32_t qend, uint32_t q0, int jlo, int m,
                                         const uint32_t* s_off, const uint4* __restrict__ srect,
                                         const uint32_t* __restrict__ order, const uint4* __restrict__ spans,
                                         uint32_t* s_key, uint32_t* s_gid) {
  if (qa >= qend) return;
  int lo = 0, hi = m - 1;  // last i with s_off[i] <= qa
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_off[mid] <= qa) lo = mid;
    else hi = mid - 1;
  }
  EmitG G;
  emit_load(G, srect[jlo + lo], order[jlo + lo], spans);
  emit_locate(G, qa - s_off[lo]);
  uint32_t next = lo + 1 < m ? s_off[lo + 1] : 0xffffffffu;
#pragma unroll 1
  for (int u = 0; u < kEmitRun; ++u) {
    const uint32_t q = qa + u;
    if (q >= qend) break;
    if (q >= next) {  // the run enters the next Gaussian (past any without pairs)
      do {
        ++lo;
        next = lo + 1 < m ? s_off[lo + 1] : 0xffffffffu;
      } while (q >= next);
      emit_load(G, srect[jlo + lo], order[jlo + lo], spans);
      emit_locate(G, q - s_off[lo]);
    }
    const uint32_t slot = emit_slot(q - q0);
    s_key[slot] = G.tile_off + static_cast<uint32_t>(G.y0 + G.k) * G.tiles_x + static_cast<uint32_t>(G.col);
    s_gid[slot] = G.gid;
    emit_step(G);
  }
}

__global__ void __launch_bounds__(kPreBlock)
    emit_kernel(const uint32_t* __restrict__ offs, const uint4* __restrict__ srect,
                const uint32_t* ord_odd, const uint32_t* ord_even, const uint32_t* __restrict__ chunk_start, int n,
                const FrameHeader* hdr, const uint4* __restrict__ spans, uint32_t* __restrict__ tkeys,
                uint32_t* __restrict__ egid, uint32_t* __restrict__ ident) {
  griddep_wait();
  griddep_launch_dependents();
  const uint32_t* __restrict__ order = depth_order(ord_odd, ord_even, hdr);
  __shared__ uint32_t s_off[kEmitChunk + 1];
  __shared__ uint32_t s_key[kEmitChunk];
  __shared__ uint32_t s_gid[kEmitChunk];
  const uint32_t K = hdr->key_count;
  // grid-stride over the output chunks: the grid is sized for the device,
  // the chunk count is only known here
  for (uint32_t c = blockIdx.x; static_cast<uint64_t>(c) * kEmitChunk < K; c += gridDim.x) {
    const uint32_t q0 = c * kEmitChunk;
    const int jlo = static_cast<int>(chunk_start[c]);
    // window of items: up to the item holding the next chunk's first pair
    const int jhi = (q0 + kEmitChunk < K) ? static_cast<int>(chunk_start[c + 1]) : n - 1;
    const int m = min(kEmitChunk + 1, min(jhi, n - 1) - jlo + 1);
    __syncthreads();  // the previous chunk is done with the shared arrays
    for (int i = threadIdx.x; i < m; i += kPreBlock) s_off[i] = offs[jlo + i];
    __syncthreads();
    const uint32_t qend = min(K, q0 + kEmitChunk);
    emit_run(q0 + threadIdx.x * kEmitRun, qend, q0, jlo, m, s_off, srect, order, spans, s_key, s_gid);
    __syncthreads();
    for (uint32_t i = threadIdx.x; q0 + i < qend; i += kPreBlock) {
      const uint32_t slot = emit_slot(i);
      tkeys[q0 + i] = s_key[slot];
      egid[q0 + i] = s_gid[slot];
      if (ident) ident[q0 + i] = q0 + i;  // a single-tile image has no tile sort to generate the values
    }
  }
}

// The emission fused with the tile sort's first radix pass: CTAs take the
// emission chunks by ticket (chunk c, pairs [c E, (c + 1) E) of the
// depth-ordered list, is tile c of the pass), build the chunk's (tile id,
// item) pairs in shared memory exactly as emit_kernel does, write each pair's
// item, and rank and scatter the tile ids by their low digit with the
// emission indices as values (the pass of onesweep.cu, on keys that never go
// through global memory; the digit histogram comes ready from the tile
// counts). A CTA takes its next chunk only after publishing the previous
// one's prefix, so every chunk it waits on belongs to a running CTA.
static_assert(kEmitChunk == kOsTile && kPreBlock == kSortThreads, "an emission chunk is one sort tile");

__global__ void __launch_bounds__(kPreBlock, 5)
    emit_sort_kernel(const uint32_t* __restrict__ offs, const uint4* __restrict__ srect, const uint32_t* ord_odd,
                     const uint32_t* ord_even, const uint32_t* __restrict__ chunk_start, int n, FrameHeader* hdr,
                     const uint4* __restrict__ spans, uint32_t* __restrict__ egid, uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                     const uint32_t* __restrict__ hist, uint32_t* status, uint32_t* ticket, uint32_t mask) {
  griddep_wait();
  griddep_launch_dependents();
  __shared__ uint32_t s_off[kEmitChunk + 1];
  __shared__ uint32_t s_key[kEmitChunk];  // the chunk's tile ids, then the pass's staging of keys
  __shared__ uint32_t s_gid[kEmitChunk];  // the chunk's items, then the pass's staging of values
  __shared__ OsShared S;
  __shared__ uint32_t s_c;
  const uint32_t* __restrict__ order = depth_order(ord_odd, ord_even, hdr);
  const uint32_t K = hdr->key_count;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    __syncthreads();  // the previous chunk is done with the shared arrays
    if (threadIdx.x == 0) s_c = atomicAdd(ticket, 1u);
    os_clear(S);
    __syncthreads();
    const uint32_t c = s_c;
    if (static_cast<uint64_t>(c) * kEmitChunk >= K) break;
    const uint32_t q0 = c * kEmitChunk;
    const int jlo = static_cast<int>(chunk_start[c]);
    const int jhi = (q0 + kEmitChunk < K) ? static_cast<int>(chunk_start[c + 1]) : n - 1;
    const int m = min(kEmitChunk + 1, min(jhi, n - 1) - jlo + 1);
    for (int i = threadIdx.x; i < m; i += kPreBlock) s_off[i] = offs[jlo + i];
    __syncthreads();
    const uint32_t qend = min(K, q0 + kEmitChunk);
    emit_run(q0 + threadIdx.x * kEmitRun, qend, q0, jlo, m, s_off, srect, order, spans, s_key, s_gid);
    __syncthreads();
    const uint32_t tn = qend - q0;
    for (uint32_t i = threadIdx.x; i < tn; i += kPreBlock) egid[q0 + i] = s_gid[emit_slot(i)];
    uint32_t k[kOsIPT], v[kOsIPT], d[kOsIPT];
#pragma unroll
    for (int j = 0; j < kOsIPT; ++j) {
      const uint32_t li = warp * (32 * kOsIPT) + j * 32 + lane;
      k[j] = li < tn ? s_key[emit_slot(li)] : 0u;
      v[j] = q0 + li;
      d[j] = li < tn ? (k[j] & mask) : 0xffffffffu;
    }
    // (os_rank_scatter synchronises the CTA before it stages into s_key / s_gid)
    os_rank_scatter(k, v, d, c, K, 0u, 0, mask, hist, status, &hdr->status, 0xffffffffu, kSpinLimit, S, s_key,
                    s_gid, kout, vout);
  }
}

cudaError_t launch_emit_sort(const FrameLayout& L, void* frame, uint32_t* kout, uint32_t* vout, const uint32_t* hist,
                             uint32_t* status, uint32_t* ticket, cudaStream_t s) {
  if (L.n == 0) return cudaSuccess;
  const int64_t chunks = (L.cap + kEmitChunk - 1) / kEmitChunk;
  if (chunks == 0) return cudaSuccess;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, emit_sort_kernel, kPreBlock, 0);
  const int64_t resident = static_cast<int64_t>(per > 0 ? per : 1) * (sms > 0 ? sms : 1);
  const int64_t grid = chunks < resident ? chunks : resident;
  const int nb = L.tile_bits < kSortRadixBits ? L.tile_bits : kSortRadixBits;
  cudaError_t e = launch_pdl(emit_sort_kernel, static_cast<unsigned>(grid), kPreBlock, 0, s,
                             static_cast<const uint32_t*>(at<uint32_t>(frame, L.offs)),
                             static_cast<const uint4*>(at<uint4>(frame, L.srect)),
                             static_cast<const uint32_t*>(at<uint32_t>(frame, L.ord1)),
                             static_cast<const uint32_t*>(at<uint32_t>(frame, L.ord0)),
                             static_cast<const uint32_t*>(at<uint32_t>(frame, L.chunks)), static_cast<int>(L.m),
                             at<FrameHeader>(frame, L.header), static_cast<const uint4*>(at<uint4>(frame, L.spans)),
                             at<uint32_t>(frame, L.egid), kout, vout, hist, status, ticket, (1u << nb) - 1u);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Inclusive scan over the lanes of a warp.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// The tile sort's second pass (tile ids of 9 to 16 bits), chunk by chunk in
// group order. The first pass (run by the emission) leaves the list grouped
// by the low 8 bits g of the tile id, each group in emission (depth) order;
// group g holds the pairs of the tiles g + 256 h. The chunks of 2048 pairs
// are numbered group after group and each is ranked and scattered by h as in a
// onesweep pass, but its look-back stops at the first chunk of its group, and
// digit h of group g starts at the range of tile g + 256 h, which the tile
// counts already hold: a chunk waits on the chunks of its own group only (a
// few) instead of on every chunk before it. The result is the onesweep pass's
// bit for bit. The group order has at most one partial chunk per group more
// than the list has chunks (kChainSlack pairs of status room).
__global__ void __launch_bounds__(kSortThreads, 5)
    tile_chain_pass_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                           uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const uint32_t* __restrict__ hist0,
                           const uint2* __restrict__ ranges, FrameHeader* hdr, uint32_t* status, uint32_t* ticket,
                           int hbits, int ntiles) {
  __shared__ uint32_t s_tile;
  __shared__ OsShared S;
  __shared__ uint32_t s_k[kOsTile];
  __shared__ uint32_t s_v[kOsTile];
  __shared__ uint32_t s_cpre[kSortRadix + 1];  // first chunk of each group in group order; [256]: all chunks
  __shared__ uint32_t s_gpre[kSortRadix];      // first pair of each group
  __shared__ uint32_t s_sc[kOsWarps][2];
  griddep_wait();
  griddep_launch_dependents();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h = threadIdx.x;  // thread h: group h in the scans, digit h in the pass
  const uint32_t K = hdr->key_count;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  os_clear(S);
  {  // exclusive scans of the groups' sizes and chunk counts
    const uint32_t gn = hist0[h];
    const uint32_t gc = (gn + kOsTile - 1) / kOsTile;
    const uint32_t xn = warp_incl_scan(gn, lane), xc = warp_incl_scan(gc, lane);
    if (lane == 31) {
      s_sc[warp][0] = xn;
      s_sc[warp][1] = xc;
    }
    __syncthreads();
    uint32_t pn = 0, pc = 0;
    for (int w = 0; w < warp; ++w) {
      pn += s_sc[w][0];
      pc += s_sc[w][1];
    }
    s_gpre[h] = pn + xn - gn;
    s_cpre[h] = pc + xc - gc;
    if (h == kSortRadix - 1) s_cpre[kSortRadix] = pc + xc;
  }
  __syncthreads();
  const uint32_t t = s_tile;
  if (t >= s_cpre[kSortRadix]) return;  // grid sized for the capacity; CTA-uniform exit
  int g = 0;  // the chunk's group: the last g whose first chunk is at or before t
#pragma unroll
  for (int step = kSortRadix / 2; step >= 1; step >>= 1)
    if (g + step < kSortRadix && s_cpre[g + step] <= t) g += step;
  const uint32_t chain0 = s_cpre[g];
  const uint32_t gb = s_gpre[g] + (t - chain0) * kOsTile;  // the chunk's first pair
  const uint32_t ge = min(s_gpre[g] + hist0[g], K);       // after an overflow the group may run past the list
  const uint32_t tn = gb < ge ? min(static_cast<uint32_t>(kOsTile), ge - gb) : 0u;
  const uint32_t mask = (1u << hbits) - 1u;
  uint32_t k[kOsIPT], v[kOsIPT], d[kOsIPT];
#pragma unroll
  for (int j = 0; j < kOsIPT; ++j) {
    const uint32_t li = warp * (32 * kOsIPT) + j * 32 + lane;
    if (li < tn) {
      k[j] = kin[gb + li];
      v[j] = vin[gb + li];
      d[j] = (k[j] >> kSortRadixBits) & mask;
    } else {
      k[j] = 0;
      v[j] = 0;
      d[j] = 0xffffffffu;
    }
  }
  // digit h of this group: tile g + 256 h, its range's begin; a tile without pairs needs no status
  const int tile = g + (h << kSortRadixBits);
  const bool exists = static_cast<uint32_t>(h) <= mask && tile < ntiles;
  const uint2 rg = exists ? ranges[tile] : make_uint2(0u, 0u);
  os_rank_scatter<true>(k, v, d, t, K, 0u, kSortRadixBits, mask, nullptr, status, &hdr->status, 0xffffffffu,
                        kSpinLimit, S, s_k, s_v, kout, vout, chain0, rg.x, rg.y > rg.x);
}

cudaError_t launch_tile_chain_pass(const FrameLayout& L, void* frame, const uint32_t* kin, const uint32_t* vin,
                                   uint32_t* kout, uint32_t* vout, void* tsort, cudaStream_t s) {
  if (L.n == 0 || L.cap == 0) return cudaSuccess;
  const int64_t tiles = (L.cap + kOsTile - 1) / kOsTile;
  const int64_t grid = tiles + kSortRadix;  // at most one partial chunk per group more
  uint32_t* status = onesweep_status(tsort, L.tile_bits) + static_cast<size_t>(tiles) * kSortRadix;  // pass 1's
  const cudaError_t e = launch_pdl(tile_chain_pass_kernel, static_cast<unsigned>(grid), kSortThreads, 0, s, kin, vin,
                                   kout, vout, static_cast<const uint32_t*>(tsort),
                                   static_cast<const uint2*>(at<uint2>(frame, L.ranges)),
                                   at<FrameHeader>(frame, L.header), status, onesweep_tickets(tsort, L.tile_bits) + 1,
                                   L.tile_bits - kSortRadixBits, L.ntiles);
  return e != cudaSuccess ? e : cudaGetLastError();
}


// Per-tile pair counts from the per-row difference arrays the preprocess
// filled (+1 at the first tile of a Gaussian's interval in a tile row, -1
// after its last: prefix sums along x, in shared memory with warp scans), their
// exclusive scan in tile order as the [begin, end) ranges of the tile-sorted
// list, and the digit histograms of the tile sort's radix passes. One CTA per
// view; the difference array is copied into dynamic shared memory. Needs only
// what the preprocess wrote.
__global__ void __launch_bounds__(1024)
    tile_counts_kernel(const uint32_t* __restrict__ tdiff, const ViewDev* __restrict__ views, uint32_t cap,
                       const FrameHeader* hdr, uint2* __restrict__ ranges, uint32_t* __restrict__ hist,
                       int passes, uint32_t* __restrict__ torder) {
  extern __shared__ uint32_t s_c[];  // tiles_y x tiles_x counts of this CTA's view
  __shared__ uint32_t s_h[4][kSortRadix];
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const int v = blockIdx.x;
  const ViewDev& V = views[v];
  const int tiles_x = V.tiles_x, tiles_y = V.tiles_y;
  const uint32_t toff = V.tile_off;
  const uint32_t* td = tdiff + V.tdiff_off;
  const int st = tiles_x + 1;
  const int ntiles = tiles_x * tiles_y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int k = threadIdx.x; k < 4 * kSortRadix; k += blockDim.x) (&s_h[0][0])[k] = 0;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) s_c[t] = td[(t / tiles_x) * st + (t % tiles_x)];
  __shared__ bool s_overflow;
  if (threadIdx.x == 0) {  // the view's first pair: pairs of the views before it
    uint32_t base = 0, total = 0;
    for (int u = 0; u < kMaxViews; ++u) {
      if (u < v) base += hdr->view_pairs[u];
      total += hdr->view_pairs[u];
    }
    s_carry = base;
    s_overflow = total > cap;
  }
  __syncthreads();
  for (int y = warp; y < tiles_y; y += nwarp) {  // each warp: running sums along its rows
    uint32_t carry = 0;
    for (int x0 = 0; x0 < tiles_x; x0 += 32) {
      const int x = x0 + lane;
      const uint32_t val = x < tiles_x ? s_c[y * tiles_x + x] : 0u;
      const uint32_t inc = warp_incl_scan(val, lane) + carry;
      if (x < tiles_x) s_c[y * tiles_x + x] = inc;
      carry = __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  __syncthreads();
  // after a key-capacity overflow the list is incomplete: every tile gets an
  // empty range so nothing downstream reads it (the frame reports the
  // overflow). The pair count is the sum of the views' counts the preprocess
  // kept, so this kernel can run before the binning.
  const bool overflow = s_overflow;
  for (int base = 0; base < ntiles; base += blockDim.x) {
    const int t = base + threadIdx.x;
    const uint32_t c = t < ntiles ? s_c[t] : 0u;
    const uint32_t x = warp_incl_scan(c, lane);
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = warp_incl_scan(lane < nwarp ? s_warp[lane] : 0u, lane);
      s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t start = s_carry + (warp ? s_warp[warp - 1] : 0u) + x - c;
    if (t < ntiles) {
      ranges[toff + t] = overflow ? make_uint2(0u, 0u) : make_uint2(start, start + c);
      if (c) {
        const uint32_t gt = toff + static_cast<uint32_t>(t);
        for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(gt >> (8 * p)) & 0xff], c);
      }
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = start + c;
    __syncthreads();
  }
  for (int p = 0; p < passes; ++p)
    for (int d = threadIdx.x; d < kSortRadix; d += blockDim.x)
      if (s_h[p][d]) atomicAdd(&hist[p * kSortRadix + d], s_h[p][d]);
  // The order in which the persistent blends take this view's tiles: longest
  // list first (64 classes of the list length, a counting sort), so that the
  // last tiles handed out are short and the SMs finish together. Any order
  // gives the same images: tiles are independent. (torder null: index order.)
  if (!torder) return;
  __shared__ uint32_t s_cls[kTileClasses];
  __shared__ uint32_t s_max;
  if (threadIdx.x == 0) s_max = 0;
  for (int k = threadIdx.x; k < kTileClasses; k += blockDim.x) s_cls[k] = 0;
  __syncthreads();
  uint32_t mx = 0;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) mx = max(mx, s_c[t]);
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0) atomicMax(&s_max, mx);
  __syncthreads();
  const uint64_t top = static_cast<uint64_t>(s_max) + 1;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x)  // class 0: the longest lists
    atomicAdd(&s_cls[kTileClasses - 1 - static_cast<int>(s_c[t] * static_cast<uint64_t>(kTileClasses) / top)], 1u);
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the class sizes (kTileClasses = 64: two per lane)
    const uint32_t a = s_cls[2 * lane], b = s_cls[2 * lane + 1];
    const uint32_t x = warp_incl_scan(a + b, lane);
    s_cls[2 * lane] = x - a - b;
    s_cls[2 * lane + 1] = x - b;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    const int c = kTileClasses - 1 - static_cast<int>(s_c[t] * static_cast<uint64_t>(kTileClasses) / top);
    torder[toff + atomicAdd(&s_cls[c], 1u)] = toff + static_cast<uint32_t>(t);
  }
}

// The sort carries each pair's emission index e; egid[e] is its Gaussian.
__global__ void export_keys_kernel(const uint32_t* __restrict__ tkeys, const uint32_t* __restrict__ vals,
                                   const uint32_t* __restrict__ egid, const float4* __restrict__ recB,
                                   const FrameHeader* hdr, uint32_t ng, uint32_t cap, uint64_t* __restrict__ out) {
  const uint32_t n = hdr->key_count;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t e = vals[i];  // out of range only in an overflowed (invalid) frame
    const uint32_t g = e < cap ? egid[e] : ng;
    out[i] = (static_cast<uint64_t>(tkeys[i]) << 32) | (g < ng ? __float_as_uint(recB[g].z) : 0u);
  }
}

__global__ void export_values_kernel(const uint32_t* __restrict__ vals, const uint32_t* __restrict__ egid,
                                     const FrameHeader* hdr, uint32_t cap, uint32_t* __restrict__ out) {
  const uint32_t n = hdr->key_count;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t e = vals[i];
    out[i] = e < cap ? egid[e] : 0xffffffffu;
  }
}


cudaError_t launch_binning(const FrameLayout& L, void* frame, cudaStream_t s) {
  if (L.n == 0) return cudaSuccess;
  FrameHeader* hdr = at<FrameHeader>(frame, L.header);
  const uint32_t* ord_odd = at<uint32_t>(frame, L.ord1);   // where the depth sort's odd pass counts end
  const uint32_t* ord_even = at<uint32_t>(frame, L.ord0);
  uint32_t* bs = at<uint32_t>(frame, L.blocksum);
  const uint32_t* touched = at<uint32_t>(frame, L.touched);
  const int m = static_cast<int>(L.m);
  uint32_t* offs = at<uint32_t>(frame, L.offs);
  uint4* srect = at<uint4>(frame, L.srect);
  uint32_t* cstart = at<uint32_t>(frame, L.chunks);
  const int64_t chunks = (L.cap + kEmitChunk - 1) / kEmitChunk;
  cudaError_t e = launch_pdl(depth_blocksum_kernel, L.nblocks, kPreBlock, 0, s, touched, ord_odd, ord_even,
                             static_cast<const FrameHeader*>(hdr), bs);
  const bool self_scan = L.nblocks <= kSelfScanBlocks;
  if (e == cudaSuccess && !self_scan)
    e = launch_pdl(scan_blocksums_kernel, 1, kScanThreads, 0, s, bs, L.nblocks, hdr, static_cast<uint32_t>(L.cap));
  if (e == cudaSuccess)
    e = launch_pdl(self_scan ? depth_offsets_kernel<true> : depth_offsets_kernel<false>, L.nblocks, kPreBlock, 0, s,
                   touched, ord_odd, ord_even, static_cast<const uint32_t*>(bs),
                   static_cast<const uint2*>(at<uint2>(frame, L.rect)),
                   static_cast<const ViewDev*>(at<ViewDev>(frame, L.views)), static_cast<uint32_t>(L.n), m, offs,
                   at<uint32_t>(frame, L.ioffs), srect, cstart, static_cast<uint32_t>(chunks), hdr,
                   static_cast<uint32_t>(L.cap));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t egrid = chunks < 8LL * sms ? chunks : 8LL * sms;  // eight 256-thread CTAs per SM
  // with a tile sort, the emission runs with its first pass (launch_emit_sort)
  if (chunks > 0 && L.tile_bits == 0)
    e = launch_pdl(emit_kernel, static_cast<unsigned>(egrid), kPreBlock, 0, s, static_cast<const uint32_t*>(offs),
                   static_cast<const uint4*>(srect), ord_odd, ord_even, static_cast<const uint32_t*>(cstart), m,
                   static_cast<const FrameHeader*>(hdr), static_cast<const uint4*>(at<uint4>(frame, L.spans)),
                   at<uint32_t>(frame, L.keys0), at<uint32_t>(frame, L.egid),
                   L.tile_bits == 0 ? at<uint32_t>(frame, L.vals0) : nullptr);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_tile_counts(const FrameLayout& L, void* frame, uint32_t* hist, int passes, cudaStream_t s) {
  const size_t smem = sizeof(uint32_t) * static_cast<size_t>(L.max_view_tiles);
  if (smem > kTileCountsMaxSmem) return cudaErrorInvalidValue;
  // opt in to large dynamic shared memory (a per-device function attribute)
  cudaFuncSetAttribute(tile_counts_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileCountsMaxSmem);
  tile_counts_kernel<<<L.nviews, 1024, smem, s>>>(at<uint32_t>(frame, L.tdiff), at<ViewDev>(frame, L.views),
                                                  static_cast<uint32_t>(L.cap), at<FrameHeader>(frame, L.header),
                                                  at<uint2>(frame, L.ranges), hist, passes,
                                                  const_cast<uint32_t*>(tile_order(L, frame)));
  return cudaGetLastError();
}

cudaError_t launch_export_keys(const FrameLayout& L, void* frame, const uint32_t* tile_keys,
                               const uint32_t* vals, uint64_t* out, cudaStream_t s) {
  if (L.n == 0) return cudaSuccess;
  const float4* recB = at<float4>(frame, L.rec) + L.m;
  export_keys_kernel<<<4 * 152, 256, 0, s>>>(tile_keys, vals, at<uint32_t>(frame, L.egid), recB,
                                             at<FrameHeader>(frame, L.header), static_cast<uint32_t>(L.m),
                                             static_cast<uint32_t>(L.cap), out);
  return cudaGetLastError();
}

cudaError_t launch_export_values(const FrameLayout& L, void* frame, const uint32_t* vals, uint32_t* out,
                                 cudaStream_t s) {
  if (L.n == 0) return cudaSuccess;
  export_values_kernel<<<4 * 152, 256, 0, s>>>(vals, at<uint32_t>(frame, L.egid), at<FrameHeader>(frame, L.header),
                                               static_cast<uint32_t>(L.cap), out);
  return cudaGetLastError();
}


}  // namespace r4g
