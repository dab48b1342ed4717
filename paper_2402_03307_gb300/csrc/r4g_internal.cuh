// Internal declarations shared by the CUDA translation units of libr4g.
#pragma once
#include <cstddef>
#include <cstdint>
#include <utility>

#include <cuda_runtime.h>

#include "r4g.h"

namespace r4g {

// Per-pixel and per-Gaussian thresholds of the compositing rules (Sec. 3.1
// rasteriser, Sec. 3.2.2 visibility threshold).
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kPowerCut = -4.5f;     // 3-sigma ellipse: d^T conic d <= 9
constexpr float kTemporalCut = 16.0f;  // lambda (t - mu_t)^2 > 16 culls
constexpr float kNear = 0.2f;
constexpr float kDilation = 0.3f;      // low-pass term added to the 2D covariance
constexpr float kClampFov = 1.3f;      // J is taken with x/z, y/z within 1.3 tan(fov/2)

// Camera as the kernels see it.
struct CamDev {
  float R[9];
  float t[3];
  float pos[3];  // camera centre in world space, -R^T t
  float fx, fy, cx, cy;
  float limx, limy;  // 1.3 tan(fov/2) per axis
  int width, height;
};

// Views of one call. A call renders V (camera, t) views of the same
// Gaussians; every per-Gaussian array of the frame holds V * N items, item
// v * N + i being Gaussian i seen by view v. Tile ids are global: view v owns
// [tile_off, tile_off + tiles_x * tiles_y). Images, T and stop positions are
// packed view after view (view v's pixels start at pix_off).
constexpr int kMaxViews = 64;

struct __align__(16) ViewDev {  // kernel-side view table entry (in the frame), 128 bytes
  CamDev cam;
  float t;
  int tiles_x, tiles_y;
  uint32_t tile_off, pix_off, tdiff_off;
  uint32_t pad[3];
};
static_assert(sizeof(ViewDev) == 128 && alignof(ViewDev) == 16, "view table entry size and alignment");

struct ViewGeom {  // host-side view geometry (what the launch sizes depend on)
  int width, height, tiles_x, tiles_y;
  uint32_t tile_off, pix_off, tdiff_off;
};

// Frame header at the start of every frame buffer (device memory).
struct FrameHeader {
  uint32_t status;        // bit 0: key overflow, bit 1: a sort look-back gave up waiting
  uint32_t key_count;     // pairs actually written (min(needed, capacity))
  uint32_t key_needed;    // pairs the render needed
  uint32_t n_visible;     // visible (view, Gaussian) items
  unsigned long long composited;  // composited (pixel, Gaussian) pairs, counted on request
  uint32_t n_glist;       // Gaussians visible in at least one view (the backward's work list)
  uint32_t next_tile;     // work counter of the persistent blend
  uint32_t next_tile_bwd; // work counter of the persistent blend backward
  uint32_t n_reached;     // pairs whose gradient slot the last backward wrote (cleared with next_tile_bwd)
  uint32_t n_ilist;       // visible (view, Gaussian) items listed for a multi-view backward
  uint32_t dkey_minc;     // ~(smallest depth key of the items with tiles), by atomicMax from 0
  uint32_t dkey_max;      // largest depth key of the items with tiles
  uint32_t pad[51];
  uint32_t view_pairs[kMaxViews];  // (tile, Gaussian) pairs per view
};
static_assert(sizeof(FrameHeader) == 512, "frame header size");

// Byte offsets of the regions of a frame; computed on the host.
struct FrameLayout {
  size_t header, views, rec, rect, spans, touched, tdiff, dkey0, dkey1, ord0, ord1, offs, ioffs, srect, chunks,
      blocksum, glist, keys0, vals0, keys1, vals1, egid, gbuf, reach, ranges, torder, tfinal, last, sortcnt,
      onesweep, tsort, ilist, ipart, total;
  int64_t n, cap;
  int64_t m;         // items: n * nviews
  int nviews;
  ViewGeom geom[kMaxViews];
  int tile_w, tile_h;
  int ntiles;        // tiles of all views
  int64_t npix;      // pixels of all views
  int tdiff_words;   // difference-array entries of all views
  int max_view_tiles;
  int width, height, tiles_x, tiles_y;  // of view 0
  int nblocks;       // preprocess-order blocks over the items (kPreBlock each)
  int sort_ctas;     // CTAs of each radix pass over the keys
  int depth_ctas;    // CTAs of each radix pass over the depth keys of the items
  int tile_bits;     // ceil(log2(ntiles)): bits of the tile sort
  bool keys_in_1;    // the tile-sorted values end in vals1 (else vals0)
};

constexpr int kPreBlock = 256;     // items per preprocess-order / key-build block
constexpr int kPreFwdBlock = 128;  // Gaussians per preprocess (forward) block
constexpr int kSelfScanBlocks = 2048;  // up to this many blocks, the depth-order offsets scan themselves
// The blends take tiles longest list first when the call's screen records fit
// well within L2 (the tiles then share them wherever they lie); beyond that,
// in index order, where neighbouring tiles in flight together reuse records.
constexpr int64_t kTileOrderMaxRecordBytes = int64_t(64) << 20;
constexpr int kMaxTiles = 51200;   // tiles per view (the tile-count kernel keeps them in shared memory)
constexpr int kSortThreads = 256;
constexpr int kSortIPT = 8;        // items per thread per tile
constexpr int kSortTile = kSortThreads * kSortIPT;
constexpr int kSortRadixBits = 8;
constexpr int kSortRadix = 1 << kSortRadixBits;
constexpr int kSortMaxCtas = 2 * 152;  // two CTAs per SM of a GB300; a multiple of 16

int sort_ctas_for(int64_t cap);
// Sets the message r4g_last_error(NULL) returns on this host thread.
void set_last_error(const char* msg);
// Layout of a frame for n Gaussians and nviews views of the given sizes.
FrameLayout make_layout(int64_t n, const int* widths, const int* heights, int nviews, int64_t cap, int tile_w,
                        int tile_h);

// Exponent of a Gaussian at a pixel, power = -1/2 (a dx^2 + 2 b dx dy + c dy^2),
// with A = (mean2d.x, mean2d.y, a, b). Every rounding step is explicit so the
// forward and backward blends take bit-identical per-pixel decisions.
__device__ __forceinline__ float gauss_power(const float4& A, float c, float fx, float fy,
                                             float& dx, float& dy) {
  dx = __fsub_rn(fx, A.x);
  dy = __fsub_rn(fy, A.y);
  float q = __fmul_rn(__fmul_rn(A.z, dx), dx);
  q = __fmaf_rn(__fmul_rn(c, dy), dy, q);
  const float cross = __fmul_rn(__fmul_rn(A.w, dx), dy);
  return __fmaf_rn(-0.5f, q, -cross);
}

// ---- programmatic dependent launch ---------------------------------------------
// The render's kernels follow one another on one stream. Launched with
// launch_pdl, a kernel is scheduled while its predecessor finishes (the
// predecessor lets its dependents launch as soon as all its CTAs have
// started: griddep_launch_dependents); it then waits in griddep_wait, before
// touching any memory, until the predecessor has completed and its writes
// are visible. Both are no-ops for a kernel launched the ordinary way.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename T>
inline T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

// The blends' tile order for the frame (written by the tile counts kernel), or
// nullptr for index order.
inline const uint32_t* tile_order(const FrameLayout& L, void* frame) {
  return 48 * L.m <= kTileOrderMaxRecordBytes ? at<uint32_t>(frame, L.torder) : nullptr;
}

// ---- launchers (return cudaGetLastError() after enqueueing) -----------------
// View table of the frame from host views (views_dev NULL) or device views,
// then the per-item preprocess (a one-view call builds the table inside the
// preprocess kernel).
cudaError_t launch_setup_views(const FrameLayout& L, void* frame, const r4g_view* views_host,
                               const r4g_view* views_dev, cudaStream_t s);
cudaError_t launch_preprocess_fwd(const r4g_gaussians& g, const FrameLayout& L, void* frame, int sh_degree,
                                  uint32_t flags, const r4g_view* views_host, const r4g_view* views_dev,
                                  cudaStream_t s);
// scan of the tile counts in depth order and key emission (tile key, index)
cudaError_t launch_binning(const FrameLayout& L, void* frame, cudaStream_t s);
// the pair emission fused with the tile sort's first radix pass (tile_bits > 0;
// hist: the tile sort's histograms, status / ticket: its first pass's)
cudaError_t launch_emit_sort(const FrameLayout& L, void* frame, uint32_t* kout, uint32_t* vout, const uint32_t* hist,
                             uint32_t* status, uint32_t* ticket, cudaStream_t s);
cudaError_t launch_sort(const uint64_t* kin, const uint32_t* vin, uint64_t* kbuf1,
                        uint32_t* vbuf1, uint64_t* kbuf2, uint32_t* vbuf2,
                        const uint32_t* count_dev, uint32_t count_host, int64_t cap,
                        int begin_bit, int end_bit, uint32_t* counts, int ctas,
                        cudaStream_t s, int* result_in_buf);
// One-kernel-per-pass radix sort of (uint32 key, uint32 value) on key bits
// [0, bits) (see onesweep.cu); scratch holds onesweep_scratch_bytes(cap, bits).
size_t onesweep_scratch_bytes(int64_t cap, int bits);
cudaError_t launch_onesweep(const uint32_t* kin, const uint32_t* vin, uint32_t* kbuf1, uint32_t* vbuf1,
                            uint32_t* kbuf2, uint32_t* vbuf2, const uint32_t* count_dev, uint32_t count_host,
                            int64_t cap, int bits, void* scratch, uint32_t* err, cudaStream_t s,
                            int* result_in_buf, bool hist_ready = false, bool prepared = false,
                            uint32_t withheld_tile = 0xffffffffu, uint32_t spin_limit = 0u, int first_pass = 0);
// The scratch of launch_onesweep: histograms [passes][256], tickets [32], then
// each pass's look-back statuses ([tiles][256] words per pass).
uint32_t* onesweep_tickets(void* scratch, int bits);
uint32_t* onesweep_status(void* scratch, int bits);
// The render's depth sort: a stable sort of the items' depth keys (float bits,
// 0xffffffff for an item without tiles, which the first pass drops), the
// values being the item indices. Digits are taken from key - kmin (kmin the
// smallest key of the items with tiles, from the frame header), so the passes
// beyond the width of the frame's key range exit at once; the order ends in
// buffer 1 when the pass count depth_passes(hdr) is odd, else in buffer 2.
// The scratch must be zero (the render's first memset clears it).
cudaError_t launch_depth_sort(const uint32_t* kin, uint32_t* kbuf1, uint32_t* vbuf1, uint32_t* kbuf2, uint32_t* vbuf2,
                              int64_t m, const FrameHeader* hdr, void* scratch, uint32_t* err, cudaStream_t s);
__device__ __forceinline__ int depth_passes(const FrameHeader* hdr) {
  const uint32_t n = hdr->n_visible;
  const uint32_t range = hdr->dkey_max - ~hdr->dkey_minc;
  return n == 0 ? 1 : range < (1u << 8) ? 1 : range < (1u << 16) ? 2 : range < (1u << 24) ? 3 : 4;
}
// What launch_onesweep clears before its passes (tickets, statuses and, unless
// hist_ready, the histograms), enqueued separately so it can run early on
// another stream; then call launch_onesweep with prepared = true.
cudaError_t prepare_onesweep(void* scratch, int64_t cap, int bits, bool hist_ready, cudaStream_t s);
// per-tile counts -> ranges and the tile sort's digit histograms (hist[p][256],
// zeroed by the caller)
cudaError_t launch_tile_counts(const FrameLayout& L, void* frame, uint32_t* hist, int passes, cudaStream_t s);
// The tile sort's second pass taken group by group (tile ids of 9 to 16
// bits): look-back chains one low-digit group long. Its statuses need
// kChainSlack pairs' worth of room beyond the key capacity's.
constexpr int64_t kChainSlack = int64_t(256) * 2048;
cudaError_t launch_tile_chain_pass(const FrameLayout& L, void* frame, const uint32_t* kin, const uint32_t* vin,
                                   uint32_t* kout, uint32_t* vout, void* tsort, cudaStream_t s);
// 64-bit (tile << 32 | depth bits) keys of the sorted list, for export
cudaError_t launch_export_keys(const FrameLayout& L, void* frame, const uint32_t* tile_keys,
                               const uint32_t* vals, uint64_t* out, cudaStream_t s);
// item index of each sorted pair (the sort carries emission indices)
cudaError_t launch_export_values(const FrameLayout& L, void* frame, const uint32_t* vals, uint32_t* out,
                                 cudaStream_t s);
cudaError_t launch_blend_fwd(const FrameLayout& L, void* frame, const uint32_t* vals,
                             const float* bg, float* out_rgb, float* out_T,
                             uint32_t* out_last, bool count, cudaStream_t s);
cudaError_t launch_blend_bwd(const FrameLayout& L, void* frame, const uint32_t* vals,
                             const float* bg, const float* grad_rgb, cudaStream_t s);
cudaError_t launch_preprocess_bwd(const r4g_gaussians& g, const FrameLayout& L, void* frame, int sh_degree,
                                  uint32_t flags, r4g_grads grads, cudaStream_t s);

}  // namespace r4g
