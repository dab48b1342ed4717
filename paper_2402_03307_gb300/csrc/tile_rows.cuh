// The tiles a Gaussian's contributing ellipse meets, row by row of tiles.
//
// A pixel takes a Gaussian only where q = d^T conic d <= min(9, 2 ln(255 o))
// (the 3-sigma cutoff and the alpha >= 1/255 rule of Sec. 3.1). Within the
// Gaussian's tile rectangle, tile row ty is a band of pixel-centre rows; the
// ellipse's slice through that band is convex, so the tiles of the row that
// it meets are the columns its x-extent covers: an interval. The x-extent of
// the slice is the ellipse's own extreme x where the extreme point's dy lies
// in the band, else the boundary's x at the band edge nearer to it (the left
// boundary x(dy) is convex, the right one concave).
//
// The preprocess counts these tiles (and marks them in the per-row
// difference array of tile counts) and the pair emission enumerates them
// again from the screen record; both call tile_row_span on the same record
// values with every operation spelled out (rounded multiplies and adds, the
// hardware's approximate reciprocal and square root, no contraction), so the
// two agree bit for bit in any translation unit. The threshold carries 1% and
// 0.01 of slack over the blends' own test (1.001 and 1e-3), far above those
// approximations' ~1e-6 relative error, so no pixel a blend composites falls
// outside the listed tiles; an ellipse too elongated for its FP32 determinant
// to be trusted keeps every tile of its rectangle. Columns are counted from
// the pixel centres the slice's x-extent covers.
#pragma once

#include "r4g_internal.cuh"

namespace r4g {

__device__ __forceinline__ float span_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float span_sqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct TileEllipse {
  float mx, my, a, b, c, thr, det, ia, rx, ry, dyl, dyr;
  bool exact;  // false: every tile of the rectangle
};

// From the screen record: centre, conic (a, b, c) and log2(255 o_t).
__device__ __forceinline__ TileEllipse tile_ellipse(float mx, float my, float a, float b, float c, float l255) {
  constexpr float kLn2x2 = 1.3862943611198906f;  // 2 ln 2
  TileEllipse E;
  E.mx = mx;
  E.my = my;
  E.a = a;
  E.b = b;
  E.c = c;
  E.thr = __fadd_rn(__fmul_rn(1.01f, fminf(9.0f, __fmul_rn(kLn2x2, l255))), 0.01f);
  const float ac = __fmul_rn(a, c);
  E.det = __fsub_rn(ac, __fmul_rn(b, b));
  E.exact = a > 0.0f && c > 0.0f && E.det > __fmul_rn(1e-3f, ac);
  if (E.exact) {
    const float idet = span_rcp(E.det);
    E.ia = span_rcp(a);
    E.rx = span_sqrt(__fmul_rn(__fmul_rn(E.thr, c), idet));  // |dx| over the ellipse
    E.ry = span_sqrt(__fmul_rn(__fmul_rn(E.thr, a), idet));  // |dy| over the ellipse
    E.dyl = __fmul_rn(__fmul_rn(b, E.rx), span_rcp(c));      // dy of the leftmost point
    E.dyr = -E.dyl;                                           // dy of the rightmost point
  } else {
    E.ia = E.rx = E.ry = E.dyl = E.dyr = 0.0f;
  }
  return E;
}

// Columns [c0, c1] of tile row ty (tiles 2^tws x 2^ths pixels) that the
// ellipse meets, within the rectangle columns [x0, x1); false if none.
__device__ __forceinline__ bool tile_row_span(const TileEllipse& E, int ty, int tws, int ths, int x0, int x1, int& c0,
                                              int& c1) {
  if (!E.exact) {
    c0 = x0;
    c1 = x1 - 1;
    return x0 < x1;
  }
  const float ya = __fsub_rn(__fadd_rn(static_cast<float>(ty << ths), 0.5f), E.my);
  const float yb = __fsub_rn(__fadd_rn(static_cast<float>((ty + 1) << ths), -0.5f), E.my);
  const float lo = fmaxf(ya, -E.ry), hi = fminf(yb, E.ry);
  if (lo > hi) return false;
  // the boundary at the band's edges: x = (-b dy -+ sqrt(thr a - det dy^2)) / a
  const float sl = span_sqrt(fmaxf(__fsub_rn(__fmul_rn(E.thr, E.a), __fmul_rn(E.det, __fmul_rn(lo, lo))), 0.0f));
  const float sh = span_sqrt(fmaxf(__fsub_rn(__fmul_rn(E.thr, E.a), __fmul_rn(E.det, __fmul_rn(hi, hi))), 0.0f));
  const float bl = -__fmul_rn(E.b, lo), bh = -__fmul_rn(E.b, hi);
  const float xl = (E.dyl >= lo && E.dyl <= hi)
                       ? -E.rx
                       : fminf(__fmul_rn(__fsub_rn(bl, sl), E.ia), __fmul_rn(__fsub_rn(bh, sh), E.ia));
  const float xr = (E.dyr >= lo && E.dyr <= hi)
                       ? E.rx
                       : fmaxf(__fmul_rn(__fadd_rn(bl, sl), E.ia), __fmul_rn(__fadd_rn(bh, sh), E.ia));
  // pixel columns whose centre x + 0.5 lies in [mx + xl, mx + xr], then their tiles
  const float pa = ceilf(__fsub_rn(__fadd_rn(E.mx, xl), 0.5f));
  const float pb = floorf(__fsub_rn(__fadd_rn(E.mx, xr), 0.5f));
  const float lim = static_cast<float>(x1 << tws);  // beyond the rectangle on either side
  const int ia = static_cast<int>(fminf(fmaxf(pa, -1.0f), lim));
  const int ib = static_cast<int>(fminf(fmaxf(pb, -1.0f), lim));
  if (ib < 0 || ia > ib) return false;
  c0 = max(ia < 0 ? 0 : ia >> tws, x0);
  c1 = min(ib >> tws, x1 - 1);
  return c0 <= c1;
}

// Row spans are stored per item for rectangles of at most kSpanRows tile rows
// and kSpanCols columns: byte 2k = first column - x0 of row y0 + k, byte
// 2k + 1 = its width (0: none). Larger rectangles keep every tile (both the
// preprocess and the emission take the whole row).
constexpr int kSpanRows = 16, kSpanCols = 255;

__device__ __forceinline__ bool span_mode(int x0, int x1, int y0, int y1) {
  return y1 - y0 <= kSpanRows && x1 - x0 <= kSpanCols;
}

__host__ __device__ constexpr int log2_pow2(int v) { return v <= 1 ? 0 : 1 + log2_pow2(v >> 1); }

}  // namespace r4g
