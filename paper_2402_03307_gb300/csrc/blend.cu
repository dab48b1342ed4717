// Tiled front-to-back alpha compositing (Sec. 3.1, Eq. 3) and its backward.
//
// Persistent CTAs take tiles; each thread owns Q packed pairs of
// horizontally adjacent pixels (Q = 2 for tiles 16 wide, 1 for 8x8 tiles)
// and evaluates them with Blackwell's packed FP32x2 instructions; a
// Gaussian's per-row terms are computed once for all of the thread's pixels.
// Each warp owns a (8 Q) x 8 block of the tile. Batches of screen
// records are staged in shared memory with every operand already duplicated
// into the (x, x) pairs the packed instructions take. While staging, each Gaussian gets one bit per warp
// telling whether its contributing ellipse can reach a pixel centre of that
// warp's block; a warp then walks only the set bits of a 32-entry ballot, so
// Gaussians that cannot touch it cost nothing. Every pixel applies the exact
// rules of the rasteriser:
//   power = -1/2 d^T conic d, skip if power > 0 or power < -4.5,
//   alpha = min(0.99, opacity_t exp(power)), skip if alpha < 1/255,
//   stop before a Gaussian that would take T below 1e-4.
// The exponent is evaluated in base 2 with the opacity folded in
// (power' = log2(e) power, alpha = 2^(power' + log2 opacity_t)). The cutoff
// and the 1/255 rule form one window pmin <= power' <= 0,
// pmin = max(-4.5 log2 e, -log2(255 opacity_t)), tested on the shifted
// exponent as |(power' + log2 opacity_t - mid - log2 opacity_t) / half| <= 1. A pixel that stops moves to
// infinity, so no later Gaussian reaches it; a warp whose pixels have all
// stopped leaves the batch, a CTA whose pixels have all stopped leaves the
// tile. The forward and the backward call the same evaluator, so they take
// bit-identical decisions. The frame keeps, per pixel, the number of list
// entries it considered (the stop position); the backward walks back from it.
#include <cuda_runtime.h>

#include "r4g_internal.cuh"

namespace r4g {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.69314718055994531f;
constexpr float kCut2 = kPowerCut * kLog2e;  // cutoff on power'
constexpr uint32_t kClampBit = 1u << 31;     // opacity_t > 0.99: alpha may need the clamp
constexpr float kFar = 3.0e38f;              // where a stopped pixel moves

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Each warp owns a block of 8 rows, 4 threads across, each thread Q packed
// pairs: 8x8 pixels with Q = 1, 16x8 with Q = 2. Two pairs per thread share
// the Gaussian's per-row terms and its staged operands and halve the warp
// reductions of the backward per pixel; the wider block costs a few more
// Gaussians that only graze it.
template <int TW, int TH>
struct Blend {
  static constexpr int Q = TW % 16 == 0 ? 2 : 1;  // packed pixel pairs per thread
  static constexpr int BW = 8 * Q;                // warp block width
  static constexpr int NT = TW * TH / (2 * Q);    // threads per CTA
  static constexpr int NW = NT / 32;              // warps per CTA
  static constexpr int WX = TW / BW;              // warp blocks across the tile
  static constexpr int PCOLS = 4;                 // thread columns of a warp block
  static constexpr int WROWS = 8;                 // pixel rows of a warp block
  static_assert(TW % BW == 0 && TH % 8 == 0 && NW >= 1 && NW <= 16, "tile shape");
  __device__ static int px0(int tx, int warp) { return tx * TW + (warp % WX) * BW; }
  __device__ static int py0(int ty, int warp) { return ty * TH + (warp / WX) * 8; }
};

// A staged Gaussian, operands duplicated for the packed pairs:
//   p0 = (-mx, -mx, -my, -my)     p1 = (A', A', B', B')
//   p2 = (C', C', lo, lo)         p3 = (r, r, g, g)
//   p4 = (b, b, ih, ih)           p5 = (nm, nm)
// with power' = A' dx^2 + B' dx dy + C' dy^2, lo = log2 o (the opacity enters
// the exponent: alpha = 2^(power' + lo)), ih = 1 / half, nm = -(mid + lo) / half
// (the window on power' shifted by lo); m: the warp-block bits and the clamp
// bit; o: opacity_t. StagedG is an entry in registers; a batch is staged as
// a StageSet, one array per operand group: the lanes of a warp write
// consecutive entries of each array and read the lanes' consecutive mask
// words without bank conflicts, and a warp that evaluates an entry reads it
// as a broadcast.
struct StagedG {
  float4 p0, p1, p2, p3, p4;
  float2 p5;
  uint32_t m;
  float o;
};

template <int N>
struct StageSet {
  float4 p0[N], p1[N], p2[N], p3[N], p4[N];
  float2 p5[N];
  uint32_t mask[N];
  float o[N];
  __device__ __forceinline__ StagedG get(int j) const {
    StagedG g;
    g.p0 = p0[j];
    g.p1 = p1[j];
    g.p2 = p2[j];
    g.p3 = p3[j];
    g.p4 = p4[j];
    g.p5 = p5[j];
    g.m = mask[j];
    g.o = o[j];
    return g;
  }
};

// Can the Gaussian's contributing region {q <= min(9, 2 ln(255 o))}, q = d^T conic d,
// contain a pixel centre of the rectangle [x0, x1] x [y0, y1]? Exact minimum of
// q over the rectangle (inside, or on one of the four edges), compared with a
// threshold thr that carries a relative and an absolute slack so the answer is
// conservative under FP32; boc = b / c and boa = b / a.
__device__ __forceinline__ bool ellipse_meets_rect(const float4 A, float c, float thr, float boc, float boa,
                                                   float x0, float x1, float y0, float y1) {
  const float mx = A.x, my = A.y, a = A.z, b = A.w;
  if (mx >= x0 && mx <= x1 && my >= y0 && my <= y1) return true;
  float qmin = 3.4e38f;
#pragma unroll
  for (int e = 0; e < 2; ++e) {  // vertical edges: minimise over dy
    const float dx = (e ? x1 : x0) - mx;
    float dy = -boc * dx;
    dy = fminf(fmaxf(dy, y0 - my), y1 - my);
    qmin = fminf(qmin, a * dx * dx + 2.0f * b * dx * dy + c * dy * dy);
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {  // horizontal edges: minimise over dx
    const float dy = (e ? y1 : y0) - my;
    float dx = -boa * dy;
    dx = fminf(fmaxf(dx, x0 - mx), x1 - mx);
    qmin = fminf(qmin, a * dx * dx + 2.0f * b * dx * dy + c * dy * dy);
  }
  return qmin <= thr;
}

// Stage one batch entry: record -> shared memory, plus the warp-block bits.
template <int TW, int TH>
__device__ __forceinline__ void stage_entry(const float4* __restrict__ recA, const float4* __restrict__ recB,
                                            const float4* __restrict__ recC, uint32_t gid, uint32_t ng, int tx,
                                            int ty, StageSet<Blend<TW, TH>::NT>& sg, int i) {
  using B = Blend<TW, TH>;
  if (gid >= ng) {  // defensive: an entry that reaches no pixel
    sg.mask[i] = 0u;
    sg.o[i] = 0.0f;
    return;
  }
  const float4 A = recA[gid], Bv = recB[gid], C = recC[gid];
  const float Ap = -0.5f * kLog2e * A.z, Bp = -kLog2e * A.w, Cp = -0.5f * kLog2e * Bv.x, o = Bv.y;
  // the record carries log2(255 o) and max(log2 o, -126) (the preprocess's)
  const float l255 = Bv.w, lo = C.w;
  const float pmin = fmaxf(kCut2, -l255);
  const float mid = 0.5f * pmin, half = fmaxf(-0.5f * pmin, 1e-6f);
  const float ih = 1.0f / half, nm = -(mid + lo) * ih;
  uint32_t m = o > kAlphaMax ? kClampBit : 0u;
  // the contributing ellipse q <= min(9, 2 ln(255 o)), with slack
  const float thr = fminf(9.0f, 2.0f * kLn2 * l255) * 1.001f + 1e-3f;
  const float boc = A.w / Bv.x, boa = A.w / A.z;
#pragma unroll
  for (int w = 0; w < B::NW; ++w) {  // pixel centres of warp w's block
    const float x0 = B::px0(tx, w) + 0.5f, x1 = x0 + static_cast<float>(B::BW - 1);
    const float y0 = B::py0(ty, w) + 0.5f, y1 = y0 + 7.0f;
    if (ellipse_meets_rect(A, Bv.x, thr, boc, boa, x0, x1, y0, y1)) m |= 1u << w;
  }
  sg.p0[i] = make_float4(-A.x, -A.x, -A.y, -A.y);
  sg.p1[i] = make_float4(Ap, Ap, Bp, Bp);
  sg.p2[i] = make_float4(Cp, Cp, lo, lo);
  sg.p3[i] = make_float4(C.x, C.x, C.y, C.y);
  sg.p4[i] = make_float4(C.z, C.z, ih, ih);
  sg.p5[i] = make_float2(nm, nm);
  sg.mask[i] = m;
  sg.o[i] = o;
}

// Evaluation of one staged Gaussian at the thread's Q pixel pairs (PX[q],
// py): power' + log2 opacity_t, alpha = 2^(power' + log2 opacity_t) before the
// clamp, and whether the window takes it, every rounding explicit. dy and the
// row terms B' dy and C' dy^2 + log2 opacity_t are shared by the pairs (they
// are the same numbers a pair alone would compute).
template <int Q>
struct PairEval {
  float2 araw[Q], dx[Q];
  float dy;
  bool v[2 * Q];
};

template <int Q>
__device__ __forceinline__ void eval_pairs(const StagedG& g, const float2 (&PX)[Q], float2 PY, PairEval<Q>& r) {
  const float4 p0 = g.p0, p1 = g.p1, p2 = g.p2, p4 = g.p4;
  const float2 p5 = g.p5;
  const float2 dy = __fadd2_rn(PY, make_float2(p0.z, p0.w));
  const float2 bdy = __fmul2_rn(make_float2(p1.z, p1.w), dy);
  const float2 u = __ffma2_rn(__fmul2_rn(make_float2(p2.x, p2.y), dy), dy, make_float2(p2.z, p2.w));
  r.dy = dy.x;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    r.dx[q] = __fadd2_rn(PX[q], make_float2(p0.x, p0.y));
    const float2 t = __ffma2_rn(make_float2(p1.x, p1.y), r.dx[q], bdy);
    const float2 p = __ffma2_rn(r.dx[q], t, u);
    r.araw[q] = make_float2(ex2_approx(p.x), ex2_approx(p.y));
    const float2 w = __ffma2_rn(p, make_float2(p4.z, p4.w), make_float2(p5.x, p5.y));
    r.v[2 * q] = fabsf(w.x) <= 1.0f;
    r.v[2 * q + 1] = fabsf(w.y) <= 1.0f;
  }
}

// Per-thread state of the forward walk over a tile list (pixel j = 2 q + h
// is lane h of pair q).
template <int Q>
struct FwdState {
  float2 PX[Q], T[Q], cr[Q], cg[Q], cb[Q];
  uint32_t stop[2 * Q], last[2 * Q], pairs;
  bool done[2 * Q];
};

__device__ __forceinline__ float& lane_of(float2& v, int h) { return h ? v.y : v.x; }

// Composite one evaluated Gaussian into the thread's pixels. kClamp: the
// Gaussian's opacity_t exceeds 0.99 so alpha is clamped; kLast: track the
// last composited position. Returns true when every pixel of the warp has
// stopped.
// Returns kApplyDone when every pixel of the warp has stopped, and
// kApplyStopped when some pixel of the warp stopped at this Gaussian.
constexpr int kApplyDone = 1, kApplyStopped = 2;

template <bool kClamp, bool kLast, int Q>
__device__ __forceinline__ int fwd_apply(FwdState<Q>& S, PairEval<Q>& ev, const StagedG& g, uint32_t pos) {
  float2 a[Q], Tn[Q];
  float tmin = 3.0e38f;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    a[q] = make_float2(ev.v[2 * q] ? ev.araw[q].x : 0.0f, ev.v[2 * q + 1] ? ev.araw[q].y : 0.0f);
    if constexpr (kClamp) a[q] = make_float2(fminf(a[q].x, kAlphaMax), fminf(a[q].y, kAlphaMax));
    Tn[q] = __ffma2_rn(make_float2(-S.T[q].x, -S.T[q].y), a[q], S.T[q]);  // T (1 - alpha)
    tmin = fminf(tmin, fminf(Tn[q].x, Tn[q].y));  // only a taken Gaussian can take T below 1e-4
  }
  int ret = 0;
  if (__any_sync(0xffffffffu, tmin < kTMin)) {
    // stop before this Gaussian: it is not composited; the pixel is done
    bool all = true;
#pragma unroll
    for (int j = 0; j < 2 * Q; ++j) {
      const int q = j >> 1, h = j & 1;
      if (lane_of(Tn[q], h) < kTMin) {
        lane_of(a[q], h) = 0.0f;
        lane_of(Tn[q], h) = lane_of(S.T[q], h);
        lane_of(S.PX[q], h) = kFar;
        ev.v[j] = false;
        S.done[j] = true;
        S.stop[j] = pos;
      }
      all = all && S.done[j];
    }
    ret = kApplyStopped | (__all_sync(0xffffffffu, all) ? kApplyDone : 0);
  }
  const float4 p3 = g.p3, p4 = g.p4;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float2 w = __fmul2_rn(a[q], S.T[q]);
    S.cr[q] = __ffma2_rn(make_float2(p3.x, p3.y), w, S.cr[q]);
    S.cg[q] = __ffma2_rn(make_float2(p3.z, p3.w), w, S.cg[q]);
    S.cb[q] = __ffma2_rn(make_float2(p4.x, p4.y), w, S.cb[q]);
    S.T[q] = Tn[q];
  }
  if constexpr (kLast) {  // instrumented variant: last composited position and a pair count
#pragma unroll
    for (int j = 0; j < 2 * Q; ++j) {
      S.last[j] = ev.v[j] ? pos + 1 : S.last[j];
      S.pairs += ev.v[j] ? 1u : 0u;
    }
  }
  return ret;
}

// Walk the set bits of one 32-entry group, two Gaussians per iteration: the
// two evaluations are independent and overlap; the composites stay in order.
// A pixel that stops inside an iteration has moved to infinity before the
// second composite only through its done flag: the second evaluation saw the
// old position, so its result is discarded for that pixel. (The backward
// walks one entry at a time: two would cost it more in occupancy than they
// gain in overlap.)
template <bool kClamp, bool kLast, int Q, int N>
__device__ __forceinline__ bool fwd_group(FwdState<Q>& S, const StageSet<N>& sg, int base, uint32_t bits,
                                          uint32_t cbits, float2 PY, uint32_t pos0) {
  while (bits) {
    const int j0 = __ffs(bits) - 1;
    bits &= bits - 1;
    if (bits) {
      const int j1 = __ffs(bits) - 1;
      bits &= bits - 1;
      PairEval<Q> e0, e1;
      const StagedG g0 = sg.get(base + j0), g1 = sg.get(base + j1);
      eval_pairs<Q>(g0, S.PX, PY, e0);
      eval_pairs<Q>(g1, S.PX, PY, e1);
      const bool c0 = kClamp && ((cbits >> j0) & 1u), c1 = kClamp && ((cbits >> j1) & 1u);
      const int r0 = c0 ? fwd_apply<true, kLast, Q>(S, e0, g0, pos0 + j0)
                        : fwd_apply<false, kLast, Q>(S, e0, g0, pos0 + j0);
      if (r0 & kApplyDone) return true;
      if (r0 & kApplyStopped) {  // (warp-uniform) a pixel stopped: the second result is void there
#pragma unroll
        for (int j = 0; j < 2 * Q; ++j) e1.v[j] = e1.v[j] && !S.done[j];
      }
      if ((c1 ? fwd_apply<true, kLast, Q>(S, e1, g1, pos0 + j1)
              : fwd_apply<false, kLast, Q>(S, e1, g1, pos0 + j1)) & kApplyDone)
        return true;
    } else {
      PairEval<Q> e0;
      const StagedG g0 = sg.get(base + j0);
      eval_pairs<Q>(g0, S.PX, PY, e0);
      const bool c0 = kClamp && ((cbits >> j0) & 1u);
      if ((c0 ? fwd_apply<true, kLast, Q>(S, e0, g0, pos0 + j0)
              : fwd_apply<false, kLast, Q>(S, e0, g0, pos0 + j0)) & kApplyDone)
        return true;
    }
  }
  return false;
}

template <int TW, int TH>
constexpr int fwd_min_blocks() {
  return Blend<TW, TH>::NT <= 32 ? 16 : Blend<TW, TH>::NT <= 64 ? 14 : Blend<TW, TH>::NT <= 128 ? 7 : 3;
}

// Where a global tile id lies: its view (binary search over the views'
// first tile ids), the tile's position in the view and the view's image.
struct TileLoc {
  int tx, ty, width, height;
  uint32_t pix_off;
};

__device__ __forceinline__ TileLoc locate_tile(const ViewDev* __restrict__ views, int nviews, int tile) {
  int lo = 0, hi = nviews - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (static_cast<int>(views[mid].tile_off) <= tile) lo = mid;
    else hi = mid - 1;
  }
  const ViewDev& V = views[lo];
  const int local = tile - static_cast<int>(V.tile_off);
  TileLoc t;
  t.tx = local % V.tiles_x;
  t.ty = local / V.tiles_x;
  t.width = V.cam.width;
  t.height = V.cam.height;
  t.pix_off = V.pix_off;
  return t;
}

// The tile's pixels, front to back over its list.
template <int TW, int TH, bool kLast>
__device__ __forceinline__ void blend_fwd_tile(int tile, StageSet<Blend<TW, TH>::NT>& sg,
                                               const uint2* __restrict__ ranges,
                                               const uint32_t* __restrict__ vals, const float4* __restrict__ recA,
                                               const float4* __restrict__ recB, const float4* __restrict__ recC,
                                               const uint32_t* __restrict__ egid, uint32_t ng, uint32_t cap,
                                               const ViewDev* __restrict__ views, int nviews, float bg0, float bg1,
                                               float bg2, float* __restrict__ out_rgb, float* __restrict__ out_T,
                                               uint32_t* __restrict__ out_stop, uint32_t* __restrict__ out_last,
                                               unsigned long long* __restrict__ pair_count) {
  using B = Blend<TW, TH>;
  constexpr int BS = B::NT, Q = B::Q;
  const TileLoc loc = locate_tile(views, nviews, tile);
  const int tx = loc.tx, ty = loc.ty, width = loc.width, height = loc.height;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int px = B::px0(tx, warp) + 2 * Q * (lane % B::PCOLS);  // the thread's pixels: px .. px + 2Q - 1
  const int py = B::py0(ty, warp) + lane / B::PCOLS;
  bool in[2 * Q];
#pragma unroll
  for (int j = 0; j < 2 * Q; ++j) in[j] = px + j < width && py < height;
  const float2 PY = make_float2(py + 0.5f, py + 0.5f);
  const uint2 rg = ranges[tile];
  const int n = static_cast<int>(rg.y - rg.x);
  FwdState<Q> S;
  bool all_done = true;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    S.PX[q] = make_float2(in[2 * q] ? px + 2 * q + 0.5f : kFar, in[2 * q + 1] ? px + 2 * q + 1.5f : kFar);
    S.T[q] = make_float2(1.0f, 1.0f);
    S.cr[q] = S.cg[q] = S.cb[q] = make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int j = 0; j < 2 * Q; ++j) {
    S.stop[j] = static_cast<uint32_t>(n);
    S.last[j] = 0;
    S.done[j] = !in[j];
    all_done = all_done && S.done[j];
  }
  S.pairs = 0;
  const uint32_t wbit = 1u << warp;
  for (int b = 0; b < n; b += BS) {
    all_done = true;
#pragma unroll
    for (int j = 0; j < 2 * Q; ++j) all_done = all_done && S.done[j];
    if (__syncthreads_count(all_done) == BS) break;
    const int idx = b + static_cast<int>(threadIdx.x);
    if (idx < n) {
      const uint32_t e = vals[rg.x + idx];  // emission index of the pair
      stage_entry<TW, TH>(recA, recB, recC, e < cap ? egid[e] : ng, ng, tx, ty, sg, threadIdx.x);
    }
    __syncthreads();
    const int cnt = min(BS, n - b);
    bool wdone = __all_sync(0xffffffffu, all_done);
    for (int j0 = 0; j0 < cnt && !wdone; j0 += 32) {
      const uint32_t m = (j0 + lane < cnt) ? sg.mask[j0 + lane] : 0u;
      uint32_t bits = __ballot_sync(0xffffffffu, m & wbit);
      const uint32_t cbits = __ballot_sync(0xffffffffu, m & kClampBit);
      const uint32_t pos0 = static_cast<uint32_t>(b + j0);
      // no Gaussian of this group needs the alpha clamp: the common path
      wdone = cbits == 0u ? fwd_group<false, kLast, Q>(S, sg, j0, bits, cbits, PY, pos0)
                          : fwd_group<true, kLast, Q>(S, sg, j0, bits, cbits, PY, pos0);
    }
  }
  const size_t plane = static_cast<size_t>(width) * height;
  float* img = out_rgb + 3 * static_cast<size_t>(loc.pix_off);
#pragma unroll
  for (int j = 0; j < 2 * Q; ++j) {
    if (!in[j]) continue;
    const int q = j >> 1, h = j & 1;
    const float T = lane_of(S.T[q], h);
    const size_t pix = static_cast<size_t>(py) * width + px + j;
    img[pix] = lane_of(S.cr[q], h) + T * bg0;
    img[plane + pix] = lane_of(S.cg[q], h) + T * bg1;
    img[2 * plane + pix] = lane_of(S.cb[q], h) + T * bg2;
    out_T[loc.pix_off + pix] = T;
    out_stop[loc.pix_off + pix] = S.stop[j];
    if constexpr (kLast) {
      if (out_last) out_last[loc.pix_off + pix] = S.last[j];
    }
  }
  if constexpr (kLast) {
    const uint32_t wsum = __reduce_add_sync(0xffffffffu, S.pairs);
    if (lane == 0 && wsum) atomicAdd(pair_count, static_cast<unsigned long long>(wsum));
  }
}

// Persistent blend: each CTA takes tiles (of every view of the call) from a
// work counter in the frame header until none is left.
template <int TW, int TH, bool kLast>
__global__ void __launch_bounds__(Blend<TW, TH>::NT, (fwd_min_blocks<TW, TH>()))
    blend_fwd_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                     const float4* __restrict__ recA, const float4* __restrict__ recB,
                     const float4* __restrict__ recC, const uint32_t* __restrict__ egid, uint32_t ng,
                     uint32_t cap, const ViewDev* __restrict__ views, int nviews, int ntiles, FrameHeader* hdr,
                     float bg0, float bg1, float bg2, float* __restrict__ out_rgb, float* __restrict__ out_T,
                     uint32_t* __restrict__ out_stop, uint32_t* __restrict__ out_last,
                     unsigned long long* __restrict__ pair_count, const uint32_t* __restrict__ torder) {
  griddep_wait();
  griddep_launch_dependents();
  __shared__ StageSet<Blend<TW, TH>::NT> sg;
  __shared__ int s_tile;
  for (;;) {
    __syncthreads();  // the previous tile is done with s_tile and sg
    if (threadIdx.x == 0) {  // the next tile: in the frame's tile order when there is one
      const uint32_t k = atomicAdd(&hdr->next_tile, 1u);
      s_tile = k < static_cast<uint32_t>(ntiles) ? static_cast<int>(torder ? torder[k] : k) : ntiles;
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= ntiles) break;
    blend_fwd_tile<TW, TH, kLast>(tile, sg, ranges, vals, recA, recB, recC, egid, ng, cap, views, nviews, bg0, bg1,
                                  bg2, out_rgb, out_T, out_stop, out_last, pair_count);
  }
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Per-thread state of the backward walk (Q packed pixel pairs).
template <int Q>
struct BwdState {
  float2 PX[Q], T[Q], U[Q], gr[Q], gg[Q], gb[Q];  // T_{i+1}; U = colour-gradient behind i + T_N (g . bg); dL/d out
  uint32_t L[2 * Q];                              // stop positions
};

// Backward of one list entry at position p for the thread's pixels.
// With alpha_i = opacity_t 2^power' and the per-pixel upstream gradient g:
//   T_i = T_{i+1} / (1 - alpha_i),
//   dL/dalpha_i = (g . c_i) T_i - U_{i+1} / (1 - alpha_i),
//   U_i = U_{i+1} + (g . c_i) alpha_i T_i,
//   dL/dc_i = g alpha_i T_i.
// The entry's geometric gradients are all linear in dq = dL/dalpha_i alpha_i
// (dalpha/dpower = alpha), so the thread accumulates the raw moments
//   D = sum dq, M0 = sum dq dx, M1 = sum dq dy, Qxx = sum dq dx^2,
//   Qxy = sum dq dx dy, Qyy = sum dq dy^2
// (the thread's pixels share dy) and the conversion to d mean2d, d conic and
// d opacity_t happens once per (tile, entry). Out: v[9] = D, M0, M1, Qxx,
// Qxy, Qyy, dr, dg, db. Returns false when no pixel of the warp takes it.
template <bool kClamp, int Q>
__device__ __forceinline__ bool bwd_entry(BwdState<Q>& S, const StagedG& gs, uint32_t p, float2 PY, float v[9]) {
  PairEval<Q> ev;
  eval_pairs<Q>(gs, S.PX, PY, ev);
  bool a[2 * Q], any = false;
#pragma unroll
  for (int j = 0; j < 2 * Q; ++j) {
    a[j] = p < S.L[j] && ev.v[j];
    any = any || a[j];
  }
  if (!__any_sync(0xffffffffu, any)) return false;
  const float4 p3 = gs.p3, p4 = gs.p4;
  float2 sdq, st, sqq, scr, scg, scb;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const bool a0 = a[2 * q], a1 = a[2 * q + 1];
    const float2 ar = make_float2(a0 ? ev.araw[q].x : 0.0f, a1 ? ev.araw[q].y : 0.0f);
    float2 al = ar;
    if constexpr (kClamp) al = make_float2(fminf(ar.x, kAlphaMax), fminf(ar.y, kAlphaMax));
    const float2 om = __ffma2_rn(al, make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));  // 1 - alpha >= 0.01
    // a pixel that does not take the entry has alpha = 0, 1 - alpha = 1 and a reciprocal of exactly 1
    const float2 iom = make_float2(rcp_approx(om.x), rcp_approx(om.y));
    const float2 Ti = __fmul2_rn(S.T[q], iom);
    const float2 w = __fmul2_rn(al, Ti);
    const float2 gc = __ffma2_rn(S.gb[q], make_float2(p4.x, p4.y),
                                 __ffma2_rn(S.gg[q], make_float2(p3.z, p3.w),
                                            __fmul2_rn(S.gr[q], make_float2(p3.x, p3.y))));
    float2 da = __fmul2_rn(iom, __ffma2_rn(gc, S.T[q], make_float2(-S.U[q].x, -S.U[q].y)));
    S.U[q] = __ffma2_rn(gc, w, S.U[q]);
    S.T[q] = Ti;
    if constexpr (kClamp) {  // a clamped alpha does not depend on power' or opacity_t
      if (ar.x > kAlphaMax) da.x = 0.0f;
      if (ar.y > kAlphaMax) da.y = 0.0f;
    }
    const float2 dq = __fmul2_rn(da, ar);  // zero for pixels that do not take the entry
    const float2 t = __fmul2_rn(dq, ev.dx[q]);
    const float2 qq = __fmul2_rn(t, ev.dx[q]);
    const float2 cr = __fmul2_rn(S.gr[q], w), cg = __fmul2_rn(S.gg[q], w), cb = __fmul2_rn(S.gb[q], w);
    if (q == 0) {  // packed sums over the thread's pairs, halves added at the end
      sdq = dq; st = t; sqq = qq; scr = cr; scg = cg; scb = cb;
    } else {
      sdq = __fadd2_rn(sdq, dq);
      st = __fadd2_rn(st, t);
      sqq = __fadd2_rn(sqq, qq);
      scr = __fadd2_rn(scr, cr);
      scg = __fadd2_rn(scg, cg);
      scb = __fadd2_rn(scb, cb);
    }
  }
  v[0] = sdq.x + sdq.y;
  v[1] = st.x + st.y;
  v[3] = sqq.x + sqq.y;
  v[6] = scr.x + scr.y;
  v[7] = scg.x + scg.y;
  v[8] = scb.x + scb.y;
  v[2] = ev.dy * v[0];
  v[4] = ev.dy * v[1];
  v[5] = ev.dy * v[2];
  return true;
}

// Sum v[0..8] over the warp: values 0..7 by a transpose reduction (they end
// one per group of 4 lanes: value k in lane 4k), value 8 by a butterfly.
__device__ __forceinline__ void warp_reduce9(float v[9], int lane) {
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
}

// Backward of the blend. Each pixel re-walks its list back to front from its
// stop position and the stored final transmittance T_N (bwd_entry). Per
// (warp, entry) the raw moments are summed over the warp (warp_reduce9) into
// the warp's shared-memory slab; at the end of each batch every entry sums
// the warps' slabs in a fixed order, converts the moments to d mean2d,
// d conic, d opacity_t and d rgb, and writes them once into the per-pair
// buffer (indexed by the pair's emission index), which the preprocess
// backward sums per Gaussian. No float atomics: the gradient is
// deterministic.
template <int TW, int TH>
__device__ __forceinline__ void blend_bwd_tile(int tile, StageSet<Blend<TW, TH>::NT>& sg, uint32_t* sE,
                                               uint32_t* sTook, uint32_t& s_max,
                                               float* s_slab,
                                               const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                                               const float4* __restrict__ recA, const float4* __restrict__ recB,
                                               const float4* __restrict__ recC, const uint32_t* __restrict__ egid,
                                               uint32_t ng, uint32_t cap, const ViewDev* __restrict__ views,
                                               int nviews, float bg0, float bg1, float bg2,
                                               const float* __restrict__ Tfinal, const uint32_t* __restrict__ stoppos,
                                               const float* __restrict__ grad_rgb, float4* __restrict__ gbuf,
                                               uint8_t* __restrict__ reach, uint32_t* n_reached) {
  using B = Blend<TW, TH>;
  constexpr int BS = B::NT, Q = B::Q;
  const TileLoc loc = locate_tile(views, nviews, tile);
  const int tx = loc.tx, ty = loc.ty, width = loc.width, height = loc.height;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int px = B::px0(tx, warp) + 2 * Q * (lane % B::PCOLS);  // the thread's pixels: px .. px + 2Q - 1
  const int py = B::py0(ty, warp) + lane / B::PCOLS;
  const float2 PY = make_float2(py + 0.5f, py + 0.5f);
  const uint2 rg = ranges[tile];
  const int n = static_cast<int>(rg.y - rg.x);
  const size_t plane = static_cast<size_t>(width) * height;
  const float* gimg = grad_rgb + 3 * static_cast<size_t>(loc.pix_off);
  BwdState<Q> S;
  uint32_t lmax = 0;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float T[2] = {1.f, 1.f}, U[2] = {0.f, 0.f}, g[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    uint32_t L[2] = {0u, 0u};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int x = px + 2 * q + h;
      if (x < width && py < height) {
        const size_t pix = static_cast<size_t>(py) * width + x;
        T[h] = Tfinal[loc.pix_off + pix];
        L[h] = stoppos[loc.pix_off + pix];
        g[h][0] = gimg[pix];
        g[h][1] = gimg[plane + pix];
        g[h][2] = gimg[2 * plane + pix];
        U[h] = T[h] * (bg0 * g[h][0] + bg1 * g[h][1] + bg2 * g[h][2]);  // T_N (g . bg)
      }
    }
    S.PX[q] = make_float2(px + 2 * q + 0.5f, px + 2 * q + 1.5f);
    S.T[q] = make_float2(T[0], T[1]);
    S.U[q] = make_float2(U[0], U[1]);
    S.gr[q] = make_float2(g[0][0], g[1][0]);
    S.gg[q] = make_float2(g[0][1], g[1][1]);
    S.gb[q] = make_float2(g[0][2], g[1][2]);
    S.L[2 * q] = L[0];
    S.L[2 * q + 1] = L[1];
    lmax = max(lmax, max(L[0], L[1]));
  }
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, lmax);  // this warp's walk ends here
  if (lane == 0 && wmax) atomicMax(&s_max, wmax);
  __syncthreads();
  const int maxL = static_cast<int>(s_max);
  const uint32_t wbit = 1u << warp;
  for (int b0 = ((maxL - 1) / BS) * BS; maxL > 0 && b0 >= 0; b0 -= BS) {
    const int idx = b0 + static_cast<int>(threadIdx.x);
    __syncthreads();
    for (int k = threadIdx.x; k < B::NW * BS * 9 / 4; k += BS)
      reinterpret_cast<float4*>(s_slab)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    sTook[threadIdx.x] = 0u;
    if (idx < n) {
      const uint32_t e = vals[rg.x + idx];
      sE[threadIdx.x] = e;
      stage_entry<TW, TH>(recA, recB, recC, e < cap ? egid[e] : ng, ng, tx, ty, sg, threadIdx.x);
    }
    __syncthreads();
    const int cnt = min(BS, n - b0);
    for (int j0 = ((cnt - 1) / 32) * 32; j0 >= 0; j0 -= 32) {
      const uint32_t m = (j0 + lane < cnt && static_cast<uint32_t>(b0 + j0 + lane) < wmax)
                             ? sg.mask[j0 + lane] : 0u;
      uint32_t bits = __ballot_sync(0xffffffffu, m & wbit);
      const uint32_t cbits = __ballot_sync(0xffffffffu, m & kClampBit);
      while (bits) {
        const int jj = 31 - __clz(bits);
        bits &= ~(1u << jj);
        const uint32_t p = static_cast<uint32_t>(b0 + j0 + jj);
        float v[9];
        const StagedG gj = sg.get(j0 + jj);
        const bool took = ((cbits >> jj) & 1u) ? bwd_entry<true, Q>(S, gj, p, PY, v)
                                               : bwd_entry<false, Q>(S, gj, p, PY, v);
        if (took) {
          if (lane == 0) atomicOr(&sTook[j0 + jj], wbit);
          warp_reduce9(v, lane);
          float* dst = s_slab + (warp * BS + j0 + jj) * 9;
          if ((lane & 3) == 0) dst[lane >> 2] = v[0];
          if (lane == 1) dst[8] = v[8];
        }
      }
    }
    __syncthreads();
    {  // pairs of the batch that get a gradient slot (a statistic of the frame)
      const uint32_t tk = __ballot_sync(0xffffffffu, idx < n && sE[threadIdx.x] < cap && sTook[threadIdx.x] != 0u);
      if (lane == 0 && tk) atomicAdd(n_reached, static_cast<uint32_t>(__popc(tk)));
    }
    // each entry of the batch: sum over the warps (fixed order), convert, one write
    if (idx < n) {
      float acc[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
#pragma unroll
      for (int w = 0; w < B::NW; ++w) {
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] += s_slab[(w * BS + threadIdx.x) * 9 + k];
      }
      const uint32_t e = sE[threadIdx.x];
      if (e < cap) {
        // only entries a pixel of the tile composited have a gradient; the
        // others are flagged, not written (in a scene whose pixels saturate
        // early most of a tile's list is never reached)
        const bool took = sTook[threadIdx.x] != 0u;
        reach[e] = took ? 1u : 0u;
        if (took) {
          // power' = A' dx^2 + B' dx dy + C' dy^2 with A' = -a/(2 ln 2), B' = -b/ln 2,
          // C' = -c/(2 ln 2) for the conic (a, b, c); d power/d mean = (a dx + b dy, b dx + c dy)
          const float4 p1 = sg.p1[threadIdx.x];
          const float Ap = p1.x, Bp = p1.z, Cp = sg.p2[threadIdx.x].x, o = sg.o[threadIdx.x];
          float4 r0, r1, r2;
          r0.x = -(2.0f * Ap * acc[1] + Bp * acc[2]) * kLn2;  // d mean2d.x
          r0.y = -(Bp * acc[1] + 2.0f * Cp * acc[2]) * kLn2;  // d mean2d.y
          r0.z = -0.5f * acc[3];                             // d conic a
          r0.w = -acc[4];                                    // d conic b
          r1.x = -0.5f * acc[5];                             // d conic c
          r1.y = o > 0.0f ? acc[0] / o : 0.0f;               // d opacity_t (alpha = opacity_t 2^power')
          r1.z = r1.w = 0.0f;
          r2 = make_float4(acc[6], acc[7], acc[8], 1.0f);    // d rgb; w = 1: a pixel of the tile composited it
          float4* d = gbuf + 3 * static_cast<size_t>(e);
          d[0] = r0;
          d[1] = r1;
          d[2] = r2;
        }
      }
    }
  }
  // list entries no pixel of the tile reached: no gradient
  const int start = maxL > 0 ? ((maxL - 1) / BS) * BS + BS : 0;
  for (int i = start + static_cast<int>(threadIdx.x); i < n; i += BS) {
    const uint32_t e = vals[rg.x + i];
    if (e < cap) reach[e] = 0u;
  }
}

template <int TW, int TH>
constexpr int bwd_min_blocks() {
  return Blend<TW, TH>::NT <= 32 ? 16 : Blend<TW, TH>::NT <= 64 ? 11 : Blend<TW, TH>::NT <= 128 ? 5 : 2;
}

// Persistent blend backward over the tiles of every view of the call.
template <int TW, int TH>
__global__ void __launch_bounds__(Blend<TW, TH>::NT, (bwd_min_blocks<TW, TH>()))
    blend_bwd_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                     const float4* __restrict__ recA, const float4* __restrict__ recB,
                     const float4* __restrict__ recC, const uint32_t* __restrict__ egid, uint32_t ng,
                     uint32_t cap, const ViewDev* __restrict__ views, int nviews, int ntiles, FrameHeader* hdr,
                     float bg0, float bg1, float bg2, const float* __restrict__ Tfinal,
                     const uint32_t* __restrict__ stoppos, const float* __restrict__ grad_rgb,
                     float4* __restrict__ gbuf, uint8_t* __restrict__ reach, const uint32_t* __restrict__ torder) {
  griddep_wait();
  griddep_launch_dependents();
  // the multi-view preprocess backward that follows lists its items anew;
  // the count of pairs with a gradient starts again
  if (blockIdx.x == 0 && threadIdx.x == 0) hdr->n_ilist = 0u;
  __shared__ StageSet<Blend<TW, TH>::NT> sg;
  __shared__ uint32_t sE[Blend<TW, TH>::NT];
  __shared__ uint32_t sTook[Blend<TW, TH>::NT];  // per batch entry: warps that composited it
  __shared__ uint32_t s_max;
  __shared__ int s_tile;
  extern __shared__ __align__(16) float s_slab[];  // [NW][BS][9] per-warp sums of the batch's entries
  for (;;) {
    __syncthreads();  // the previous tile is done with the shared buffers
    if (threadIdx.x == 0) {  // the next tile: in the frame's tile order when there is one
      const uint32_t k = atomicAdd(&hdr->next_tile_bwd, 1u);
      s_tile = k < static_cast<uint32_t>(ntiles) ? static_cast<int>(torder ? torder[k] : k) : ntiles;
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= ntiles) break;
    blend_bwd_tile<TW, TH>(tile, sg, sE, sTook, s_max, s_slab, ranges, vals, recA, recB, recC, egid, ng, cap, views,
                           nviews, bg0, bg1, bg2, Tfinal, stoppos, grad_rgb, gbuf, reach, &hdr->n_reached);
  }
}

// CTAs of a persistent launch: as many as fit on the device at once, at
// most one per tile.
template <typename K>
static int persistent_ctas(K kernel, int threads, size_t smem, int ntiles) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  const long long c = static_cast<long long>(per > 0 ? per : 1) * (sms > 0 ? sms : 1);
  return static_cast<int>(c < ntiles ? c : ntiles);
}

cudaError_t launch_blend_fwd(const FrameLayout& L, void* frame, const uint32_t* vals,
                             const float* bg, float* out_rgb, float* out_T, uint32_t* out_last, bool count,
                             cudaStream_t s) {
  const float4* recA = at<float4>(frame, L.rec);
  const float4* recB = recA + L.m;
  const float4* recC = recB + L.m;
  const uint2* ranges = at<uint2>(frame, L.ranges);
  // the frame always keeps T and the stop positions for the backward
  float* T = at<float>(frame, L.tfinal);
  uint32_t* stop = at<uint32_t>(frame, L.last);
  const ViewDev* views = at<ViewDev>(frame, L.views);
  FrameHeader* hdr = at<FrameHeader>(frame, L.header);
  const uint32_t* torder = tile_order(L, frame);
#define R4G_BLEND(TW_, TH_, LAST_)                                                                          \
  e = launch_pdl(blend_fwd_kernel<TW_, TH_, LAST_>,                                                         \
                 persistent_ctas(blend_fwd_kernel<TW_, TH_, LAST_>, Blend<TW_, TH_>::NT, 0, L.ntiles),        \
                 Blend<TW_, TH_>::NT, 0, s, ranges, vals, recA, recB, recC, egid, static_cast<uint32_t>(L.m),    \
                 static_cast<uint32_t>(L.cap), views, L.nviews, L.ntiles, hdr, bg[0], bg[1], bg[2], out_rgb, T,   \
                 stop, out_last, pairs, torder)
  const uint32_t* egid = at<uint32_t>(frame, L.egid);
  // the instrumented variant serves both the last-contributor output and the pair count
  const bool lst = out_last != nullptr || count;
  unsigned long long* pairs = &hdr->composited;
  cudaError_t e = cudaSuccess;
  if (L.tile_w == 16 && L.tile_h == 16) {
    if (lst) R4G_BLEND(16, 16, true); else R4G_BLEND(16, 16, false);
  } else if (L.tile_w == 8 && L.tile_h == 8) {
    if (lst) R4G_BLEND(8, 8, true); else R4G_BLEND(8, 8, false);
  } else if (L.tile_w == 16 && L.tile_h == 32) {
    if (lst) R4G_BLEND(16, 32, true); else R4G_BLEND(16, 32, false);
  } else {
    return cudaErrorInvalidValue;
  }
#undef R4G_BLEND
  if (e != cudaSuccess) return e;
  if (out_T) cudaMemcpyAsync(out_T, T, static_cast<size_t>(L.npix) * sizeof(float), cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

cudaError_t launch_blend_bwd(const FrameLayout& L, void* frame, const uint32_t* vals,
                             const float* bg, const float* grad_rgb, cudaStream_t s) {
  const float4* recA = at<float4>(frame, L.rec);
  const float4* recB = recA + L.m;
  const float4* recC = recB + L.m;
  const uint2* ranges = at<uint2>(frame, L.ranges);
  const float* T = at<float>(frame, L.tfinal);
  const uint32_t* stop = at<uint32_t>(frame, L.last);
  const uint32_t* egid = at<uint32_t>(frame, L.egid);
  const ViewDev* views = at<ViewDev>(frame, L.views);
  FrameHeader* hdr = at<FrameHeader>(frame, L.header);
  float4* gbuf = at<float4>(frame, L.gbuf);
  uint8_t* reach = at<uint8_t>(frame, L.reach);
  const uint32_t* torder = tile_order(L, frame);
  // the backward's work counter and its count of pairs with a gradient (the
  // render zeroed the forward's counter)
  static_assert(offsetof(FrameHeader, n_reached) == offsetof(FrameHeader, next_tile_bwd) + 4, "adjacent counters");
  cudaMemsetAsync(&hdr->next_tile_bwd, 0, 2 * sizeof(uint32_t), s);
#define R4G_BLEND_BWD(TW_, TH_)                                                                           \
  {                                                                                                       \
    const size_t slab = sizeof(float) * 9 * Blend<TW_, TH_>::NW * Blend<TW_, TH_>::NT;                   \
    cudaFuncSetAttribute(blend_bwd_kernel<TW_, TH_>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                         static_cast<int>(slab));                                                         \
    e = launch_pdl(blend_bwd_kernel<TW_, TH_>,                                                            \
                   persistent_ctas(blend_bwd_kernel<TW_, TH_>, Blend<TW_, TH_>::NT, slab, L.ntiles),      \
                   Blend<TW_, TH_>::NT, slab, s, ranges, vals, recA, recB, recC, egid,                    \
                   static_cast<uint32_t>(L.m), static_cast<uint32_t>(L.cap), views, L.nviews, L.ntiles, hdr, \
                   bg[0], bg[1], bg[2], T, stop, grad_rgb, gbuf, reach, torder);                          \
  }
  cudaError_t e = cudaSuccess;
  if (L.tile_w == 16 && L.tile_h == 16) R4G_BLEND_BWD(16, 16)
  else if (L.tile_w == 8 && L.tile_h == 8) R4G_BLEND_BWD(8, 8)
  else if (L.tile_w == 16 && L.tile_h == 32) R4G_BLEND_BWD(16, 32)
  else return cudaErrorInvalidValue;
#undef R4G_BLEND_BWD
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace r4g
