// Adaptive density control of the 4D Gaussians on the GPU (Sec. 4.2: the
// duplication and pruning of the Gaussians run in CUDA; densification by the
// view-space positional gradient with the thresholds and schedule of 3D
// Gaussian Splatting, which the paper follows).
//
// One densify-and-prune step is a plan and an apply:
//   plan    one thread per Gaussian decides keep / clone / split and which of
//           its output rows survive the prune, then a block scan and a scan of
//           the block totals give every Gaussian its first output row;
//   apply   one thread per Gaussian writes its surviving rows (a split draws
//           its children's means from the Gaussian's 4D distribution).
// The output is a compacted copy: rows of Gaussian i precede those of i + 1,
// so the result is deterministic. Every decision is taken in double
// precision on the FP32 inputs against thresholds the host derives once, so
// it is exact (the products grad_threshold * count of two floats are exact in
// double; the logarithms are monotone).
#include <cmath>
#include <limits>

#include <cuda_runtime.h>

#include "r4g_math.cuh"

namespace r4g {

constexpr int kDensBlock = 256;
constexpr int kDensScanThreads = 1024;

// Thresholds of one step, derived on the host from r4g_densify_config.
struct DensRule {
  double grad_thr;       // grad_threshold
  double log_dense;      // ln(dense_scale): clone when the largest spatial log-scale <= this
  double logit_min;      // ln(m / (1 - m)): rows with logit below this are pruned (-inf: none)
  double log_max_scale;  // ln(max_scale): rows with a larger spatial log-scale are pruned (+inf: off)
  float max_radius;      // rows continuing a Gaussian with a larger screen radius are pruned (+inf: off)
  float ls_shift;        // ln(split_divisor) rounded to FP32: a child's log-scale is logscale - ls_shift
};

// Decision byte of a Gaussian: bits 0-1 the kind (0 keep, 1 clone, 2 split),
// bit 2 output row 0 survives, bit 3 output row 1 survives.
constexpr uint32_t kKeep = 0, kClone = 1, kSplit = 2;

__device__ __forceinline__ uint32_t dens_decide(const r4g_gaussians& g, const float* __restrict__ vs_grad,
                                                const float* __restrict__ vs_count,
                                                const float* __restrict__ max_radius, const DensRule& r, int i) {
  const float4 ls = __ldg(reinterpret_cast<const float4*>(g.logscale) + i);
  const float logit = __ldg(g.logit + i);
  const float cnt = __ldg(vs_count + i);
  const float gs = __ldg(vs_grad + i);
  const float rad = max_radius ? __ldg(max_radius + i) : 0.0f;
  const bool dens = cnt > 0.0f && static_cast<double>(gs) >= r.grad_thr * static_cast<double>(cnt);
  const float lmax = fmaxf(fmaxf(ls.x, ls.y), ls.z);
  const uint32_t kind = !dens ? kKeep : (static_cast<double>(lmax) <= r.log_dense ? kClone : kSplit);
  const bool opaque = static_cast<double>(logit) >= r.logit_min;
  uint32_t rows;
  if (kind == kSplit) {
    // the children's log-scales, rounded as apply writes them
    const float cmax = fmaxf(fmaxf(ls.x - r.ls_shift, ls.y - r.ls_shift), ls.z - r.ls_shift);
    const bool ok = opaque && static_cast<double>(cmax) <= r.log_max_scale;
    rows = ok ? 3u : 0u;
  } else {
    const bool small = static_cast<double>(lmax) <= r.log_max_scale;
    const bool row0 = opaque && small && !(rad > r.max_radius);  // continues Gaussian i
    const bool row1 = kind == kClone && opaque && small;         // the new copy has no screen history
    rows = (row0 ? 1u : 0u) | (row1 ? 2u : 0u);
  }
  return kind | (rows << 2);
}

// Plan: decisions, per-block exclusive offsets of the output rows, block totals.
__global__ void __launch_bounds__(kDensBlock)
    dens_plan_kernel(r4g_gaussians g, const float* __restrict__ vs_grad, const float* __restrict__ vs_count,
                     const float* __restrict__ max_radius, DensRule rule, uint8_t* __restrict__ code,
                     uint32_t* __restrict__ loc, uint32_t* __restrict__ blocksum) {
  __shared__ uint32_t s_warp[kDensBlock / 32];
  const int i = blockIdx.x * kDensBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t c = 0, rows = 0;
  if (i < g.n) {
    c = dens_decide(g, vs_grad, vs_count, max_radius, rule, i);
    rows = __popc(c >> 2);
    code[i] = static_cast<uint8_t>(c);
  }
  uint32_t x = rows;  // inclusive warp scan
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kDensBlock / 32 ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < kDensBlock / 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kDensBlock / 32) s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const uint32_t base = warp ? s_warp[warp - 1] : 0u;
  if (i < g.n) loc[i] = base + x - rows;
  if (threadIdx.x == kDensBlock - 1) blocksum[blockIdx.x] = base + x;
}

// Exclusive scan of the block totals in one CTA (each thread a contiguous
// chunk), and the number of output rows.
__global__ void __launch_bounds__(kDensScanThreads)
    dens_scan_kernel(const uint32_t* __restrict__ blocksum, uint32_t* __restrict__ blockoff, int nb,
                     long long* __restrict__ out_count) {
  __shared__ uint32_t s_warp[kDensScanThreads / 32];
  const int per = (nb + kDensScanThreads - 1) / kDensScanThreads;
  const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
  uint32_t sum = 0;
  for (int b = b0; b < b1; ++b) sum += blocksum[b];
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
  for (int b = b0; b < b1; ++b) {
    blockoff[b] = run;
    run += blocksum[b];
  }
  if (threadIdx.x == kDensScanThreads - 1) *out_count = static_cast<long long>(s_warp[31]);
}

__device__ __forceinline__ void copy_row(const r4g_gaussians& g, int i, const r4g_params_out& o, int64_t j) {
  reinterpret_cast<float4*>(o.mean)[j] = __ldg(reinterpret_cast<const float4*>(g.mean) + i);
  const float4* r = reinterpret_cast<const float4*>(g.rotor) + 2 * static_cast<int64_t>(i);
  float4* ro = reinterpret_cast<float4*>(o.rotor) + 2 * j;
  ro[0] = __ldg(r);
  ro[1] = __ldg(r + 1);
  reinterpret_cast<float4*>(o.logscale)[j] = __ldg(reinterpret_cast<const float4*>(g.logscale) + i);
  o.logit[j] = __ldg(g.logit + i);
  const float4* sh = reinterpret_cast<const float4*>(g.sh) + 12 * static_cast<int64_t>(i);
  float4* sho = reinterpret_cast<float4*>(o.sh) + 12 * j;
#pragma unroll
  for (int v = 0; v < 12; ++v) sho[v] = ld_nc_f4(sh + v);
}

// Apply: write the surviving rows of every Gaussian at its planned offset.
__global__ void __launch_bounds__(kDensBlock)
    dens_apply_kernel(r4g_gaussians g, const float* __restrict__ z, DensRule rule,
                      const uint8_t* __restrict__ code, const uint32_t* __restrict__ loc,
                      const uint32_t* __restrict__ blockoff, r4g_params_out out, int64_t capacity,
                      int32_t* __restrict__ out_src) {
  const int i = blockIdx.x * kDensBlock + threadIdx.x;
  if (i >= g.n) return;
  const uint32_t c = code[i];
  const uint32_t kind = c & 3u, rows = c >> 2;
  if (!rows) return;
  int64_t j = static_cast<int64_t>(blockoff[blockIdx.x]) + loc[i];
  if (kind != kSplit) {
    for (int q = 0; q < 2; ++q) {
      if (!((rows >> q) & 1u)) continue;
      if (j < capacity) {
        copy_row(g, i, out, j);
        if (out_src) out_src[j] = q == 0 ? i : -(i + 1);
      }
      ++j;
    }
    return;
  }
  // split: two children from N(mean, Sigma4), mean_c = mean + R diag(s) z_c
  Params p;
  load_params<false>(g, i, p);
  RotorNorm<float> rn;
  rotor_normalize<float>(p.rot, rn);
  float R[16];
  rotor_matrix<float>(rn.r, R);
  const float s[4] = {expf(p.ls[0]), expf(p.ls[1]), expf(p.ls[2]), expf(p.ls[3])};
  const float4 lsc = make_float4(p.ls[0] - rule.ls_shift, p.ls[1] - rule.ls_shift, p.ls[2] - rule.ls_shift,
                                 p.ls[3] - rule.ls_shift);
  for (int q = 0; q < 2; ++q, ++j) {
    if (j >= capacity) continue;
    const float4 zz = __ldg(reinterpret_cast<const float4*>(z) + 2 * static_cast<int64_t>(i) + q);
    const float u[4] = {s[0] * zz.x, s[1] * zz.y, s[2] * zz.z, s[3] * zz.w};
    float m[4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
      m[a] = p.mean[a] + (R[4 * a] * u[0] + R[4 * a + 1] * u[1] + R[4 * a + 2] * u[2] + R[4 * a + 3] * u[3]);
    reinterpret_cast<float4*>(out.mean)[j] = make_float4(m[0], m[1], m[2], m[3]);
    float4* ro = reinterpret_cast<float4*>(out.rotor) + 2 * j;
    ro[0] = make_float4(p.rot[0], p.rot[1], p.rot[2], p.rot[3]);
    ro[1] = make_float4(p.rot[4], p.rot[5], p.rot[6], p.rot[7]);
    reinterpret_cast<float4*>(out.logscale)[j] = lsc;
    out.logit[j] = p.logit;
    const float4* sh = reinterpret_cast<const float4*>(g.sh) + 12 * static_cast<int64_t>(i);
    float4* sho = reinterpret_cast<float4*>(out.sh) + 12 * j;
#pragma unroll
    for (int v = 0; v < 12; ++v) sho[v] = ld_nc_f4(sh + v);
    if (out_src) out_src[j] = -(i + 1);
  }
}

__global__ void opacity_reset_kernel(float* __restrict__ logit, int64_t n, float cap) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) logit[i] = fminf(logit[i], cap);
}

struct DensScratch {
  size_t code, loc, blocksum, blockoff, total;
  int nb;
};

static size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

static DensScratch dens_layout(int64_t n) {
  DensScratch L{};
  L.nb = static_cast<int>((n + kDensBlock - 1) / kDensBlock);
  size_t o = 0;
  L.code = o;     o = al256(o + static_cast<size_t>(n));
  L.loc = o;      o = al256(o + 4 * static_cast<size_t>(n));
  L.blocksum = o; o = al256(o + 4 * static_cast<size_t>(L.nb + 1));
  L.blockoff = o; o = al256(o + 4 * static_cast<size_t>(L.nb + 1));
  L.total = o;
  return L;
}

}  // namespace r4g

using namespace r4g;

namespace {
r4g_status faild(r4g_status st, const char* msg) {
  set_last_error(msg);
  return st;
}
bool aligned_to(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

r4g_status check_config(const r4g_densify_config* c) {
  if (!c) return faild(R4G_EINVAL, "cfg is NULL");
  if (!(c->grad_threshold >= 0.0f) || !std::isfinite(c->grad_threshold))
    return faild(R4G_EINVAL, "grad_threshold must be finite and >= 0");
  if (!(c->dense_scale > 0.0f) || !std::isfinite(c->dense_scale))
    return faild(R4G_EINVAL, "dense_scale must be finite and > 0");
  if (!(c->split_divisor > 1.0f) || !std::isfinite(c->split_divisor))
    return faild(R4G_EINVAL, "split_divisor must be finite and > 1");
  if (!(c->min_opacity >= 0.0f && c->min_opacity < 1.0f)) return faild(R4G_EINVAL, "min_opacity must be in [0, 1)");
  if (!(c->max_scale >= 0.0f) || !std::isfinite(c->max_scale))
    return faild(R4G_EINVAL, "max_scale must be finite and >= 0");
  if (!(c->max_screen_radius >= 0.0f) || !std::isfinite(c->max_screen_radius))
    return faild(R4G_EINVAL, "max_screen_radius must be finite and >= 0");
  return R4G_OK;
}

DensRule make_rule(const r4g_densify_config& c) {
  DensRule r;
  const double inf = std::numeric_limits<double>::infinity();
  r.grad_thr = static_cast<double>(c.grad_threshold);
  r.log_dense = std::log(static_cast<double>(c.dense_scale));
  const double m = static_cast<double>(c.min_opacity);
  r.logit_min = m > 0.0 ? std::log(m / (1.0 - m)) : -inf;
  r.log_max_scale = c.max_scale > 0.0f ? std::log(static_cast<double>(c.max_scale)) : inf;
  r.max_radius = c.max_screen_radius > 0.0f ? c.max_screen_radius : std::numeric_limits<float>::infinity();
  r.ls_shift = static_cast<float>(std::log(static_cast<double>(c.split_divisor)));
  return r;
}

r4g_status check_params(const r4g_gaussians* g) {
  if (!g) return faild(R4G_EINVAL, "g is NULL");
  if (g->n < 0 || g->n > (int64_t(1) << 28)) return faild(R4G_EINVAL, "n out of range (0..2^28)");
  if (g->scale_dtype != R4G_F32 || g->sh_dtype != R4G_F32)
    return faild(R4G_EINVAL, "density control takes FP32 scales and SH");
  if (g->n > 0 && (!g->mean || !g->rotor || !g->logscale || !g->logit || !g->sh))
    return faild(R4G_EINVAL, "a parameter pointer is NULL");
  if (g->n > 0 && (!aligned_to(g->mean, 16) || !aligned_to(g->rotor, 16) || !aligned_to(g->logscale, 16) ||
                   !aligned_to(g->sh, 16) || !aligned_to(g->logit, 4)))
    return faild(R4G_EINVAL, "parameter rows must be 16-byte aligned");
  return R4G_OK;
}
}  // namespace

extern "C" {

r4g_status r4g_densify_scratch_bytes(int64_t n, size_t* bytes) {
  if (!bytes || n < 0 || n > (int64_t(1) << 28)) return faild(R4G_EINVAL, "n out of range (0..2^28)");
  *bytes = dens_layout(n).total;
  return R4G_OK;
}

r4g_status r4g_densify_plan(const r4g_gaussians* g, const float* vs_grad, const float* vs_count,
                            const float* max_radius, const r4g_densify_config* cfg, void* scratch,
                            size_t scratch_bytes, int64_t* out_count, void* stream) {
  r4g_status st = check_params(g);
  if (st != R4G_OK) return st;
  if ((st = check_config(cfg)) != R4G_OK) return st;
  if (!out_count || !scratch) return faild(R4G_EINVAL, "NULL argument");
  if (g->n > 0 && (!vs_grad || !vs_count)) return faild(R4G_EINVAL, "vs_grad and vs_count are required");
  if (!aligned_to(scratch, 256)) return faild(R4G_EINVAL, "scratch must be 256-byte aligned");
  if (!aligned_to(out_count, 8)) return faild(R4G_EINVAL, "out_count must be 8-byte aligned");
  const DensScratch L = dens_layout(g->n);
  if (scratch_bytes < L.total) return faild(R4G_EWORKSPACE, "scratch smaller than r4g_densify_scratch_bytes");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const DensRule rule = make_rule(*cfg);
  uint32_t* blocksum = at<uint32_t>(scratch, L.blocksum);
  if (L.nb > 0)
    dens_plan_kernel<<<L.nb, kDensBlock, 0, s>>>(*g, vs_grad, vs_count, max_radius, rule,
                                                 at<uint8_t>(scratch, L.code), at<uint32_t>(scratch, L.loc),
                                                 blocksum);
  dens_scan_kernel<<<1, kDensScanThreads, 0, s>>>(blocksum, at<uint32_t>(scratch, L.blockoff), L.nb,
                                                  reinterpret_cast<long long*>(out_count));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return faild(R4G_ECUDA, cudaGetErrorString(e));
  return R4G_OK;
}

r4g_status r4g_densify_apply(const r4g_gaussians* g, const float* z, const r4g_densify_config* cfg,
                             const void* scratch, size_t scratch_bytes, r4g_params_out* out, int64_t capacity,
                             int32_t* out_src, void* stream) {
  r4g_status st = check_params(g);
  if (st != R4G_OK) return st;
  if ((st = check_config(cfg)) != R4G_OK) return st;
  if (!scratch || !out) return faild(R4G_EINVAL, "NULL argument");
  if (g->n > 0 && !z) return faild(R4G_EINVAL, "z is required");
  if (capacity < 0) return faild(R4G_EINVAL, "capacity must be >= 0");
  if (g->n > 0 && !aligned_to(z, 16)) return faild(R4G_EINVAL, "z must be 16-byte aligned");
  if (capacity > 0 && (!out->mean || !out->rotor || !out->logscale || !out->logit || !out->sh))
    return faild(R4G_EINVAL, "an output pointer is NULL");
  if (capacity > 0 && (!aligned_to(out->mean, 16) || !aligned_to(out->rotor, 16) ||
                       !aligned_to(out->logscale, 16) || !aligned_to(out->sh, 16) || !aligned_to(out->logit, 4)))
    return faild(R4G_EINVAL, "output rows must be 16-byte aligned");
  if (!aligned_to(scratch, 256)) return faild(R4G_EINVAL, "scratch must be 256-byte aligned");
  const DensScratch L = dens_layout(g->n);
  if (scratch_bytes < L.total) return faild(R4G_EWORKSPACE, "scratch smaller than r4g_densify_scratch_bytes");
  if (L.nb == 0) return R4G_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* sc = const_cast<void*>(scratch);
  dens_apply_kernel<<<L.nb, kDensBlock, 0, s>>>(*g, z, make_rule(*cfg), at<uint8_t>(sc, L.code),
                                                at<uint32_t>(sc, L.loc), at<uint32_t>(sc, L.blockoff), *out,
                                                capacity, out_src);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return faild(R4G_ECUDA, cudaGetErrorString(e));
  return R4G_OK;
}

r4g_status r4g_opacity_reset(float* logit, int64_t n, float max_opacity, void* stream) {
  if (n < 0) return faild(R4G_EINVAL, "n must be >= 0");
  if (n > 0 && !logit) return faild(R4G_EINVAL, "logit is NULL");
  if (!(max_opacity > 0.0f && max_opacity < 1.0f)) return faild(R4G_EINVAL, "max_opacity must be in (0, 1)");
  if (n == 0) return R4G_OK;
  const double m = static_cast<double>(max_opacity);
  const float cap = static_cast<float>(std::log(m / (1.0 - m)));
  const int64_t nb = (n + 255) / 256;
  opacity_reset_kernel<<<static_cast<unsigned>(nb), 256, 0, static_cast<cudaStream_t>(stream)>>>(logit, n, cap);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return faild(R4G_ECUDA, cudaGetErrorString(e));
  return R4G_OK;
}

}  // extern "C"
