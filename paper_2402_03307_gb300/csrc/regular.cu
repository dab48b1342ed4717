// Regularisers of the optimisation (Sec. 3.3): the entropy loss on the
// opacities, L_entropy = 1/N sum_i -o_i log o_i, and the 4D consistency
// loss on the speeds s_i = V_i / W_i of the sliced Gaussians (Sec. 3.2.2),
// L_consistent4D = 1/N sum_i || s_i - 1/K sum_{j in Omega_i} s_j ||_1, with
// Omega_i the K nearest neighbours of Gaussian i in 4D (Euclidean, each axis
// divided by the spatial or temporal scene scale).
//
// The 4D K-nearest-neighbour search: the scaled means are binned into a
// uniform 4D grid (about four points per cell), sorted by cell with the
// render's radix sort, and each point searches rings of cells around its
// own until its K-th distance is no larger than the distance to any cell it
// has not searched, so the result is exact. Ties in distance go to the
// smaller index.
//
// The consistency gradient sends sign terms to the neighbours; they are
// summed as integers (one 64-bit atomic per neighbour), so the gradient is
// deterministic. Loss values are reduced in a fixed order.
#include <cuda_runtime.h>

#include <cmath>

#include "preprocess_common.cuh"

namespace r4g {

constexpr int kKnnBlock = 256;
constexpr float kKnnMargin = 1e-5f;  // relative slack of the exactness bound

struct KnnGrid {
  float lo[4];   // lower corner of the scaled bounding box
  float h, ih;   // cell size and its inverse
  int dims[4];   // cells per axis
  uint32_t ncells;
};

// Order-preserving map of a float to an unsigned integer (min/max atomics).
__device__ __forceinline__ uint32_t f2ord(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Scaled coordinates and their bounding box (bbox[0..3] minima, [4..7] maxima).
__global__ void __launch_bounds__(kKnnBlock)
    knn_scale_kernel(const float4* __restrict__ means, int n, float inv_xyz, float inv_t, float4* __restrict__ q,
                     uint32_t* __restrict__ bbox) {
  __shared__ uint32_t s_b[8];
  if (threadIdx.x < 8) s_b[threadIdx.x] = threadIdx.x < 4 ? 0xffffffffu : 0u;
  __syncthreads();
  const int i = blockIdx.x * kKnnBlock + threadIdx.x;
  if (i < n) {
    const float4 m = means[i];
    const float4 v = make_float4(__fmul_rn(m.x, inv_xyz), __fmul_rn(m.y, inv_xyz), __fmul_rn(m.z, inv_xyz),
                                 __fmul_rn(m.w, inv_t));
    q[i] = v;
    const float c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      atomicMin(&s_b[d], f2ord(c[d]));
      atomicMax(&s_b[4 + d], f2ord(c[d]));
    }
  }
  __syncthreads();
  if (threadIdx.x < 4) atomicMin(&bbox[threadIdx.x], s_b[threadIdx.x]);
  else if (threadIdx.x < 8) atomicMax(&bbox[threadIdx.x], s_b[threadIdx.x]);
}

// Grid parameters (one thread): the cell size gives about four points per
// cell over the axes with a non-zero extent; a degenerate axis gets one cell.
// The cell count is kept below maxcells.
__global__ void knn_grid_kernel(const uint32_t* __restrict__ bbox, int n, uint32_t maxcells, KnnGrid* g) {
  double lo[4], ext[4];
  int nd = 0;
  double vol = 1.0;
  for (int d = 0; d < 4; ++d) {
    lo[d] = ord2f(bbox[d]);
    ext[d] = static_cast<double>(ord2f(bbox[4 + d])) - lo[d];
    if (ext[d] > 1e-30) {
      ++nd;
      vol *= ext[d];
    }
  }
  double h = 1.0;
  if (nd > 0) h = pow(vol / fmax(1.0, n / 4.0), 1.0 / nd);
  int dims[4];
  bool fits = false;
  for (int it = 0; it < 200 && !fits; ++it) {
    double cells = 1.0;
    for (int d = 0; d < 4; ++d) {
      dims[d] = ext[d] > 1e-30 ? static_cast<int>(fmin(ceil(ext[d] / h), 65535.0)) : 1;
      if (dims[d] < 1) dims[d] = 1;
      cells *= dims[d];
    }
    fits = cells <= maxcells;
    if (!fits) h *= 1.25;
  }
  if (!fits) {  // never expected: one cell holds every point (still exact)
    for (int d = 0; d < 4; ++d) dims[d] = 1;
    h = 1e30;
  }
  KnnGrid r;
  uint32_t nc = 1;
  for (int d = 0; d < 4; ++d) {
    r.lo[d] = static_cast<float>(lo[d]);
    r.dims[d] = dims[d];
    nc *= static_cast<uint32_t>(dims[d]);
  }
  r.h = static_cast<float>(h);
  r.ih = static_cast<float>(1.0 / h);
  r.ncells = nc;
  *g = r;
}

__device__ __forceinline__ int cell_coord(float q, float lo, float ih, int dim) {
  const int c = static_cast<int>(floorf(__fmul_rn(__fsub_rn(q, lo), ih)));
  return min(max(c, 0), dim - 1);
}

__device__ __forceinline__ uint32_t cell_id(const int c[4], const KnnGrid& g) {
  return ((static_cast<uint32_t>(c[3]) * g.dims[2] + c[2]) * g.dims[1] + c[1]) * g.dims[0] + c[0];
}

__global__ void __launch_bounds__(kKnnBlock)
    knn_keys_kernel(const float4* __restrict__ q, int n, const KnnGrid* __restrict__ gp, uint32_t* __restrict__ keys) {
  const int i = blockIdx.x * kKnnBlock + threadIdx.x;
  if (i >= n) return;
  const KnnGrid g = *gp;
  const float4 v = q[i];
  const float c4[4] = {v.x, v.y, v.z, v.w};
  int c[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) c[d] = cell_coord(c4[d], g.lo[d], g.ih, g.dims[d]);
  keys[i] = cell_id(c, g);
}

// Cell ranges of the sorted points and the scaled coordinates in sorted order.
__global__ void __launch_bounds__(kKnnBlock)
    knn_cells_kernel(const uint32_t* __restrict__ skeys, const uint32_t* __restrict__ svals,
                     const float4* __restrict__ q, int n, uint2* __restrict__ cells, float4* __restrict__ qs) {
  const int p = blockIdx.x * kKnnBlock + threadIdx.x;
  if (p >= n) return;
  const uint32_t k = skeys[p];
  if (p == 0 || skeys[p - 1] != k) cells[k].x = static_cast<uint32_t>(p);
  if (p == n - 1 || skeys[p + 1] != k) cells[k].y = static_cast<uint32_t>(p + 1);
  qs[p] = q[svals[p]];
}

// Distance in the scaled space, summed in a fixed order.
__device__ __forceinline__ float dist2(const float4& a, const float4& b) {
  const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z), dw = __fsub_rn(a.w, b.w);
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)), __fmul_rn(dw, dw));
}

template <int K>
__device__ __forceinline__ void topk_insert(float (&bd)[K], int (&bi)[K], float d, int j) {
  if (!(d < bd[K - 1] || (d == bd[K - 1] && j < bi[K - 1]))) return;
  bd[K - 1] = d;
  bi[K - 1] = j;
#pragma unroll
  for (int k = K - 1; k > 0; --k) {  // bubble the new entry to its place
    const bool sw = bd[k] < bd[k - 1] || (bd[k] == bd[k - 1] && bi[k] < bi[k - 1]);
    if (sw) {
      const float td = bd[k];
      bd[k] = bd[k - 1];
      bd[k - 1] = td;
      const int ti = bi[k];
      bi[k] = bi[k - 1];
      bi[k - 1] = ti;
    }
  }
}

// One thread per point (in cell order, so neighbouring threads search
// neighbouring cells). Ring r visits the cells whose largest offset from the
// point's cell is r; the search stops once K neighbours are known and the
// K-th distance is at most the distance to the faces of the searched block.
template <int K>
__global__ void __launch_bounds__(kKnnBlock)
    knn_query_kernel(const uint32_t* __restrict__ skeys, const uint32_t* __restrict__ svals,
                     const float4* __restrict__ qs, const uint2* __restrict__ cells, int n,
                     const KnnGrid* __restrict__ gp, int32_t* __restrict__ out_idx, float* __restrict__ out_d2) {
  const int p = blockIdx.x * kKnnBlock + threadIdx.x;
  if (p >= n) return;
  const KnnGrid g = *gp;
  const float4 me = qs[p];
  const int self = static_cast<int>(svals[p]);
  const float mc[4] = {me.x, me.y, me.z, me.w};
  int c[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) c[d] = cell_coord(mc[d], g.lo[d], g.ih, g.dims[d]);
  float bd[K];
  int bi[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    bd[k] = INFINITY;
    bi[k] = 0x7fffffff;
  }
  int maxdim = max(max(g.dims[0], g.dims[1]), max(g.dims[2], g.dims[3]));
  for (int r = 0; r <= maxdim; ++r) {
    int lo[4], hi[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      lo[d] = max(c[d] - r, 0);
      hi[d] = min(c[d] + r, g.dims[d] - 1);
    }
    for (int c3 = lo[3]; c3 <= hi[3]; ++c3)
      for (int c2 = lo[2]; c2 <= hi[2]; ++c2)
        for (int c1 = lo[1]; c1 <= hi[1]; ++c1)
          for (int c0 = lo[0]; c0 <= hi[0]; ++c0) {
            const int off = max(max(abs(c0 - c[0]), abs(c1 - c[1])), max(abs(c2 - c[2]), abs(c3 - c[3])));
            if (off != r) continue;  // visited in an earlier ring
            const int cc[4] = {c0, c1, c2, c3};
            const uint2 rg = cells[cell_id(cc, g)];
            for (uint32_t s = rg.x; s < rg.y; ++s) {
              const int j = static_cast<int>(svals[s]);
              if (j == self) continue;
              topk_insert<K>(bd, bi, dist2(me, qs[s]), j);
            }
          }
    // distance to the nearest face of the searched block that is not a grid edge
    float b = INFINITY;
    bool whole = true;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      if (c[d] - r > 0) {
        b = fminf(b, mc[d] - (g.lo[d] + (c[d] - r) * g.h));
        whole = false;
      }
      if (c[d] + r < g.dims[d] - 1) {
        b = fminf(b, (g.lo[d] + (c[d] + r + 1) * g.h) - mc[d]);
        whole = false;
      }
    }
    if (whole) break;
    const float bb = fmaxf(b * (1.0f - kKnnMargin) - kKnnMargin * g.h, 0.0f);
    if (bi[K - 1] != 0x7fffffff && bd[K - 1] <= bb * bb) break;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    out_idx[static_cast<size_t>(self) * K + k] = bi[k] == 0x7fffffff ? -1 : bi[k];
    if (out_d2) out_d2[static_cast<size_t>(self) * K + k] = bd[k];
  }
}

// ---- regularisers -------------------------------------------------------------
// Per Gaussian: s = V / W (from Sigma4) and the entropy term and its gradient.
template <bool kScaleBF16>
__global__ void __launch_bounds__(kKnnBlock)
    reg_speed_kernel(r4g_gaussians g, float lam_e, float4* __restrict__ speed, float* __restrict__ part,
                     float* __restrict__ glogit) {
  __shared__ float s_w[kKnnBlock / 32];
  const int i = blockIdx.x * kKnnBlock + threadIdx.x;
  float e = 0.0f;
  if (i < g.n) {
    Geo<float> G;
    gauss_setup<float, kScaleBF16>(g, i, G);
    const float iw = 1.0f / G.C[9];
    speed[i] = make_float4(G.C[3] * iw, G.C[6] * iw, G.C[8] * iw, 0.0f);
    const float o = G.opacity;
    if (o > 0.0f) {
      const float lo = logf(o);
      e = -o * lo;
      // d(-o log o)/d logit = -(log o + 1) o (1 - o)
      if (glogit) glogit[i] += lam_e / static_cast<float>(g.n) * (-(lo + 1.0f) * o * (1.0f - o));
    }
  }
  float w = e;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < kKnnBlock / 32; ++k) t += s_w[k];
    part[blockIdx.x] = t;
  }
}

__device__ __forceinline__ int fsign(float x) { return x > 0.0f ? 1 : (x < 0.0f ? -1 : 0); }

// Per Gaussian i: r_i = s_i - mean of its neighbours' speeds, |r_i|_1 into
// the loss, sign(r_i) kept with i, and (sign(r_i) + 1) per axis plus an
// in-degree count of 1 sent to every neighbour in one 64-bit atomic (four
// 16-bit fields; a K-nearest-neighbour graph in 4D has bounded in-degree).
template <int K>
__global__ void __launch_bounds__(kKnnBlock)
    reg_consistency_kernel(const int32_t* __restrict__ knn, int n, const float4* __restrict__ speed,
                           uint32_t* __restrict__ sgn, unsigned long long* __restrict__ cnt,
                           float* __restrict__ part) {
  __shared__ float s_w[kKnnBlock / 32];
  const int i = blockIdx.x * kKnnBlock + threadIdx.x;
  float l = 0.0f;
  if (i < n) {
    const float4 si = speed[i];
    float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f;
    int nb[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      nb[k] = knn[static_cast<size_t>(i) * K + k];
      if (nb[k] < 0 || nb[k] >= n) nb[k] = i;  // an index outside [0, n) counts as the point itself
      const float4 sj = speed[nb[k]];
      m0 += sj.x;
      m1 += sj.y;
      m2 += sj.z;
    }
    const float r0 = si.x - m0 / K, r1 = si.y - m1 / K, r2 = si.z - m2 / K;
    l = fabsf(r0) + fabsf(r1) + fabsf(r2);
    const int g0 = fsign(r0), g1 = fsign(r1), g2 = fsign(r2);
    sgn[i] = static_cast<uint32_t>((g0 + 1) | ((g1 + 1) << 2) | ((g2 + 1) << 4));
    const unsigned long long inc = static_cast<unsigned long long>(g0 + 1) |
                                   (static_cast<unsigned long long>(g1 + 1) << 16) |
                                   (static_cast<unsigned long long>(g2 + 1) << 32) | (1ull << 48);
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (nb[k] != i) atomicAdd(&cnt[nb[k]], inc);
  }
  float w = l;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < kKnnBlock / 32; ++k) t += s_w[k];
    part[blockIdx.x] = t;
  }
}

// Per Gaussian j: dL/ds_j = lam / N (sign(r_j) - 1/K sum_{i: j in Omega_i} sign(r_i)),
// then s = V / W -> Sigma4 -> rotor and log-scales (added to the gradients).
template <int K, bool kScaleBF16>
__global__ void __launch_bounds__(kKnnBlock)
    reg_grad_kernel(r4g_gaussians g, float lam_c, const uint32_t* __restrict__ sgn,
                    const unsigned long long* __restrict__ cnt, r4g_grads out) {
  const int j = blockIdx.x * kKnnBlock + threadIdx.x;
  if (j >= g.n) return;
  const unsigned long long c = cnt[j];
  const int indeg = static_cast<int>((c >> 48) & 0xffffu);
  const int sum[3] = {static_cast<int>(c & 0xffffu) - indeg, static_cast<int>((c >> 16) & 0xffffu) - indeg,
                      static_cast<int>((c >> 32) & 0xffffu) - indeg};
  const int own = static_cast<int>(sgn[j]);
  const int sg[3] = {(own & 3) - 1, ((own >> 2) & 3) - 1, ((own >> 4) & 3) - 1};
  const float scale = lam_c / static_cast<float>(g.n);
  float ds[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) ds[d] = scale * (static_cast<float>(K * sg[d] - sum[d]) / K);
  if (ds[0] == 0.0f && ds[1] == 0.0f && ds[2] == 0.0f) return;
  Geo<float> G;
  gauss_setup<float, kScaleBF16>(g, j, G);
  const float W = G.C[9], iw = 1.0f / W;
  const float V[3] = {G.C[3], G.C[6], G.C[8]};
  // s = V / W: dV = ds / W, dW = -(ds . V) / W^2
  float G4[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) G4[a][b] = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) G4[d][3] = G4[3][d] = 0.5f * ds[d] * iw;  // symmetric: V appears twice
  G4[3][3] = -(ds[0] * V[0] + ds[1] * V[1] + ds[2] * V[2]) * iw * iw;
  float grot[8], gls[4];
  sigma4_backward<float>(G, G4, grot, gls);
  float4* gr = reinterpret_cast<float4*>(out.rotor) + 2 * static_cast<size_t>(j);
  float4 r0 = gr[0], r1 = gr[1];
  r0.x += grot[0]; r0.y += grot[1]; r0.z += grot[2]; r0.w += grot[3];
  r1.x += grot[4]; r1.y += grot[5]; r1.z += grot[6]; r1.w += grot[7];
  gr[0] = r0;
  gr[1] = r1;
  float4* gl = reinterpret_cast<float4*>(out.logscale) + j;
  float4 vl = *gl;
  vl.x += gls[0]; vl.y += gls[1]; vl.z += gls[2]; vl.w += gls[3];
  *gl = vl;
}

// Fixed-order sums of the per-block partials: out[0] = L_entropy,
// out[1] = L_consistent4D (both unweighted means).
__global__ void reg_final_kernel(const float* __restrict__ pe, const float* __restrict__ pc, int nb, int n,
                                 float* __restrict__ out) {
  __shared__ double s[2][256];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nb; k += 256) {
    a += pe[k];
    b += pc[k];
  }
  s[0][threadIdx.x] = a;
  s[1][threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int k = 0; k < 256; ++k) {
      ta += s[0][k];
      tb += s[1][k];
    }
    out[0] = static_cast<float>(ta / n);
    out[1] = static_cast<float>(tb / n);
  }
}

// ---- scratch layouts -----------------------------------------------------------
struct KnnScratch {
  size_t q, qs, keys0, vals0, keys1, vals1, sort, cells, bbox, grid, status, total;
  uint32_t maxcells;
  int bits;
};

static size_t al(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

static KnnScratch knn_layout(int64_t n) {
  KnnScratch L{};
  L.maxcells = static_cast<uint32_t>(4 * n + 16);
  int bits = 1;
  while ((uint64_t(1) << bits) < L.maxcells) ++bits;
  L.bits = bits;
  size_t o = 0;
  L.q = o;     o = al(o + 16 * n);
  L.qs = o;    o = al(o + 16 * n);
  L.keys0 = o; o = al(o + 4 * n);
  L.vals0 = o; o = al(o + 4 * n);
  L.keys1 = o; o = al(o + 4 * n);
  L.vals1 = o; o = al(o + 4 * n);
  L.sort = o;  o = al(o + onesweep_scratch_bytes(n, bits));
  L.cells = o; o = al(o + sizeof(uint2) * L.maxcells);
  L.bbox = o;  o = al(o + 8 * sizeof(uint32_t));
  L.grid = o;  o = al(o + sizeof(KnnGrid));
  L.status = o; o = al(o + sizeof(uint32_t));
  L.total = o;
  return L;
}

struct RegScratch {
  size_t speed, sgn, cnt, pe, pc, total;
  int nb;
};

static RegScratch reg_layout(int64_t n) {
  RegScratch L{};
  L.nb = static_cast<int>((n + kKnnBlock - 1) / kKnnBlock);
  size_t o = 0;
  L.speed = o; o = al(o + 16 * n);
  L.sgn = o;   o = al(o + 4 * n);
  L.cnt = o;   o = al(o + 8 * n);
  L.pe = o;    o = al(o + 4 * (L.nb + 1));
  L.pc = o;    o = al(o + 4 * (L.nb + 1));
  L.total = o;
  return L;
}

}  // namespace r4g

using namespace r4g;

namespace {
r4g_status failc(r4g_status st, const char* msg) {
  set_last_error(msg);
  return st;
}
bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
}  // namespace

extern "C" {

r4g_status r4g_knn_scratch_bytes(int64_t n, size_t* bytes) {
  if (!bytes || n < 0 || n > (int64_t(1) << 28)) return failc(R4G_EINVAL, "n out of range (0..2^28)");
  *bytes = knn_layout(n).total;
  return R4G_OK;
}

r4g_status r4g_knn4d(const float* means, int64_t n, float scale_xyz, float scale_t, int32_t k, int32_t* out_idx,
                     float* out_dist2, void* scratch, size_t scratch_bytes, void* stream) {
  if (n < 0 || n > (int64_t(1) << 28)) return failc(R4G_EINVAL, "n out of range (0..2^28)");
  if (k != 4 && k != 8 && k != 16) return failc(R4G_EINVAL, "k must be 4, 8 or 16");
  if (n <= k) return failc(R4G_EINVAL, "need more than k points");
  if (!(scale_xyz > 0.0f) || !(scale_t > 0.0f) || !std::isfinite(scale_xyz) || !std::isfinite(scale_t))
    return failc(R4G_EINVAL, "scene scales must be positive and finite");
  if (!means || !out_idx || !scratch) return failc(R4G_EINVAL, "NULL argument");
  if (!al16(means) || (reinterpret_cast<uintptr_t>(scratch) & 255)) return failc(R4G_EINVAL, "misaligned buffer");
  const KnnScratch L = knn_layout(n);
  if (scratch_bytes < L.total) return failc(R4G_EWORKSPACE, "scratch smaller than r4g_knn_scratch_bytes");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ni = static_cast<int>(n);
  const int nb = (ni + kKnnBlock - 1) / kKnnBlock;
  float4* q = at<float4>(scratch, L.q);
  uint32_t* bbox = at<uint32_t>(scratch, L.bbox);
  KnnGrid* grid = at<KnnGrid>(scratch, L.grid);
  uint32_t* status = at<uint32_t>(scratch, L.status);
  cudaError_t e = cudaMemsetAsync(bbox, 0xff, 4 * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bbox + 4, 0, 4 * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(at<char>(scratch, L.cells), 0, sizeof(uint2) * L.maxcells, s);
  if (e != cudaSuccess) return failc(R4G_ECUDA, cudaGetErrorString(e));
  knn_scale_kernel<<<nb, kKnnBlock, 0, s>>>(reinterpret_cast<const float4*>(means), ni, 1.0f / scale_xyz,
                                            1.0f / scale_t, q, bbox);
  knn_grid_kernel<<<1, 1, 0, s>>>(bbox, ni, L.maxcells, grid);
  knn_keys_kernel<<<nb, kKnnBlock, 0, s>>>(q, ni, grid, at<uint32_t>(scratch, L.keys0));
  int which = 0;
  e = launch_onesweep(at<uint32_t>(scratch, L.keys0), nullptr, at<uint32_t>(scratch, L.keys1),
                      at<uint32_t>(scratch, L.vals1), at<uint32_t>(scratch, L.keys0), at<uint32_t>(scratch, L.vals0),
                      nullptr, static_cast<uint32_t>(n), n, L.bits, at<void>(scratch, L.sort), status, s, &which);
  if (e != cudaSuccess) return failc(R4G_ECUDA, cudaGetErrorString(e));
  const uint32_t* sk = at<uint32_t>(scratch, which == 1 ? L.keys1 : L.keys0);
  const uint32_t* sv = at<uint32_t>(scratch, which == 1 ? L.vals1 : L.vals0);
  float4* qs = at<float4>(scratch, L.qs);
  uint2* cells = at<uint2>(scratch, L.cells);
  knn_cells_kernel<<<nb, kKnnBlock, 0, s>>>(sk, sv, q, ni, cells, qs);
  if (k == 4) knn_query_kernel<4><<<nb, kKnnBlock, 0, s>>>(sk, sv, qs, cells, ni, grid, out_idx, out_dist2);
  else if (k == 8) knn_query_kernel<8><<<nb, kKnnBlock, 0, s>>>(sk, sv, qs, cells, ni, grid, out_idx, out_dist2);
  else knn_query_kernel<16><<<nb, kKnnBlock, 0, s>>>(sk, sv, qs, cells, ni, grid, out_idx, out_dist2);
  e = cudaGetLastError();
  if (e != cudaSuccess) return failc(R4G_ECUDA, cudaGetErrorString(e));
  return R4G_OK;
}

r4g_status r4g_knn_status(const void* scratch, int64_t n, void* stream) {
  if (!scratch || n < 0 || n > (int64_t(1) << 28)) return failc(R4G_EINVAL, "bad argument");
  uint32_t st = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&st, static_cast<const char*>(scratch) + knn_layout(n).status, sizeof(st),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return failc(R4G_ECUDA, cudaGetErrorString(e));
  if (st & 2u) return failc(R4G_ETIMEOUT, "a radix-sort look-back wait hit its iteration limit");
  return R4G_OK;
}

r4g_status r4g_regularizers_scratch_bytes(int64_t n, size_t* bytes) {
  if (!bytes || n < 0 || n > (int64_t(1) << 28)) return failc(R4G_EINVAL, "n out of range (0..2^28)");
  *bytes = reg_layout(n).total;
  return R4G_OK;
}

r4g_status r4g_regularizers(const r4g_gaussians* g, const int32_t* knn_idx, int32_t k, float lambda_entropy,
                            float lambda_consistency, float* out_loss, r4g_grads* grads, void* scratch,
                            size_t scratch_bytes, void* stream) {
  if (!g || !knn_idx || !out_loss || !scratch) return failc(R4G_EINVAL, "NULL argument");
  if (g->n <= k || g->n > (int64_t(1) << 28)) return failc(R4G_EINVAL, "need k < n <= 2^28");
  if (k != 4 && k != 8 && k != 16) return failc(R4G_EINVAL, "k must be 4, 8 or 16");
  if (g->scale_dtype != R4G_F32 && g->scale_dtype != R4G_BF16) return failc(R4G_EINVAL, "unknown dtype");
  if (!g->mean || !g->rotor || !g->logscale || !g->logit) return failc(R4G_EINVAL, "a parameter pointer is NULL");
  if (grads && (!grads->rotor || !grads->logscale || !grads->logit || !al16(grads->rotor) || !al16(grads->logscale)))
    return failc(R4G_EINVAL, "gradient buffers must be non-NULL and 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(scratch) & 255) return failc(R4G_EINVAL, "scratch must be 256-byte aligned");
  const RegScratch L = reg_layout(g->n);
  if (scratch_bytes < L.total) return failc(R4G_EWORKSPACE, "scratch smaller than r4g_regularizers_scratch_bytes");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float4* speed = at<float4>(scratch, L.speed);
  uint32_t* sgn = at<uint32_t>(scratch, L.sgn);
  unsigned long long* cnt = at<unsigned long long>(scratch, L.cnt);
  float* pe = at<float>(scratch, L.pe);
  float* pc = at<float>(scratch, L.pc);
  cudaError_t e = cudaMemsetAsync(cnt, 0, 8 * g->n, s);
  if (e != cudaSuccess) return failc(R4G_ECUDA, cudaGetErrorString(e));
  const bool bf = g->scale_dtype == R4G_BF16;
  const int nb = L.nb;
  float* glogit = grads ? grads->logit : nullptr;
  if (bf) reg_speed_kernel<true><<<nb, kKnnBlock, 0, s>>>(*g, lambda_entropy, speed, pe, glogit);
  else reg_speed_kernel<false><<<nb, kKnnBlock, 0, s>>>(*g, lambda_entropy, speed, pe, glogit);
  const int ni = static_cast<int>(g->n);
#define R4G_RC(K_)                                                                               \
  reg_consistency_kernel<K_><<<nb, kKnnBlock, 0, s>>>(knn_idx, ni, speed, sgn, cnt, pc);       \
  if (grads) {                                                                                 \
    if (bf) reg_grad_kernel<K_, true><<<nb, kKnnBlock, 0, s>>>(*g, lambda_consistency, sgn, cnt, *grads); \
    else reg_grad_kernel<K_, false><<<nb, kKnnBlock, 0, s>>>(*g, lambda_consistency, sgn, cnt, *grads); \
  }
  if (k == 4) { R4G_RC(4) } else if (k == 8) { R4G_RC(8) } else { R4G_RC(16) }
#undef R4G_RC
  reg_final_kernel<<<1, 256, 0, s>>>(pe, pc, nb, ni, out_loss);
  e = cudaGetLastError();
  if (e != cudaSuccess) return failc(R4G_ECUDA, cudaGetErrorString(e));
  return R4G_OK;
}

}  // extern "C"
