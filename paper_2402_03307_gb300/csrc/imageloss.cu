// The image loss of the optimisation (Sec. 3.3 total loss, as in 3D
// Gaussian Splatting): L = (1 - lambda) L1 + lambda (1 - SSIM), with SSIM
// over an 11 x 11 Gaussian window (sigma 1.5, zero padding, C1 = 0.01^2,
// C2 = 0.03^2) averaged over every pixel and channel, and its gradient with
// respect to the rendered image.
//
// Forward: per 32 x 32 output tile (plus a 5-pixel halo in shared memory),
// the five windowed moments (mu_x, mu_y, E[x^2], E[y^2], E[xy]) by two
// separable 11-tap passes; from them the SSIM value and the three per-pixel
// adjoint coefficients a = dL/dmu_x, b = dL/dE[x^2], c = dL/dE[xy].
// Backward: dL/dx = G * a + 2 x (G * b) + y (G * c) + (1 - lambda) sign(x - y) / P,
// G * being the same zero-padded window (it is symmetric, so it is its own
// adjoint). Sums of the loss parts are reduced in a fixed order.
#include <cuda_runtime.h>

#include <cmath>

#include "r4g_internal.cuh"

namespace r4g {

constexpr int kSsimT = 32;               // output tile edge
constexpr int kSsimR = 5;                // window radius
constexpr int kSsimE = kSsimT + 2 * kSsimR;  // tile edge with the halo (42)
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct SsimWin {
  float g[2 * kSsimR + 1];
};

// (B, H) halo tile of one channel, zero outside the image.
__device__ __forceinline__ void load_tile(float (*dst)[kSsimE + 1], const float* __restrict__ src, int x0, int y0,
                                          int W, int H) {
  for (int k = threadIdx.y * blockDim.x + threadIdx.x; k < kSsimE * kSsimE; k += blockDim.x * blockDim.y) {
    const int r = k / kSsimE, c = k % kSsimE;
    const int yy = y0 + r - kSsimR, xx = x0 + c - kSsimR;
    dst[r][c] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? src[static_cast<size_t>(yy) * W + xx] : 0.0f;
  }
}

__global__ void __launch_bounds__(256)
    ssim_fwd_kernel(const float* __restrict__ x, const float* __restrict__ y, int W, int H, size_t P, SsimWin win,
                    float gscale, float* __restrict__ coef, float* __restrict__ part) {
  __shared__ float sx[kSsimE][kSsimE + 1], sy[kSsimE][kSsimE + 1];
  __shared__ float hm[5][kSsimE][kSsimT + 1];  // horizontal pass of x, y, x^2, y^2, xy
  __shared__ float s_red[2][8];
  const int ch = blockIdx.z;
  const int x0 = blockIdx.x * kSsimT, y0 = blockIdx.y * kSsimT;
  const size_t plane = static_cast<size_t>(W) * H;
  const float* xc = x + ch * plane;
  const float* yc = y + ch * plane;
  load_tile(sx, xc, x0, y0, W, H);
  load_tile(sy, yc, x0, y0, W, H);
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < kSsimE; r += 8) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kSsimR; ++k) {
      const float xv = sx[r][tx + k], yv = sy[r][tx + k], w = win.g[k];
      a0 += w * xv;
      a1 += w * yv;
      a2 += w * xv * xv;
      a3 += w * yv * yv;
      a4 += w * xv * yv;
    }
    hm[0][r][tx] = a0;
    hm[1][r][tx] = a1;
    hm[2][r][tx] = a2;
    hm[3][r][tx] = a3;
    hm[4][r][tx] = a4;
  }
  __syncthreads();
  float msum = 0.f, l1sum = 0.f;
  for (int r = ty; r < kSsimT; r += 8) {
    const int py = y0 + r, px = x0 + tx;
    float mx = 0.f, my = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kSsimR; ++k) {
      const float w = win.g[k];
      mx += w * hm[0][r + k][tx];
      my += w * hm[1][r + k][tx];
      sxx += w * hm[2][r + k][tx];
      syy += w * hm[3][r + k][tx];
      sxy += w * hm[4][r + k][tx];
    }
    if (px < W && py < H) {
      const float vx = sxx - mx * mx, vy = syy - my * my, cxy = sxy - mx * my;
      const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cxy + kC2;
      const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
      const float iB = 1.0f / (B1 * B2);
      const float m = A1 * A2 * iB;
      msum += m;
      l1sum += fabsf(sx[r + kSsimR][tx + kSsimR] - sy[r + kSsimR][tx + kSsimR]);
      // dm/dmu_x, dm/dE[x^2], dm/dE[xy], scaled by dL/dm
      const float dmx = 2.f * my * (A2 - A1) * iB - 2.f * mx * m * (1.0f / B1 - 1.0f / B2);
      const float dsxx = -m / B2;
      const float dsxy = 2.f * A1 * iB;
      const size_t pix = ch * plane + static_cast<size_t>(py) * W + px;
      coef[pix] = gscale * dmx;  // three maps of P = C H W values
      coef[P + pix] = gscale * dsxx;
      coef[2 * P + pix] = gscale * dsxy;
    }
  }
  // fixed-order block sums
  float a = msum, b = l1sum;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (tx == 0) {
    s_red[0][ty] = a;
    s_red[1][ty] = b;
  }
  __syncthreads();
  if (tx == 0 && ty == 0) {
    float ta = 0.f, tb = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      ta += s_red[0][k];
      tb += s_red[1][k];
    }
    const int blk = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    part[2 * blk] = ta;
    part[2 * blk + 1] = tb;
  }
}

__global__ void __launch_bounds__(256)
    ssim_bwd_kernel(const float* __restrict__ x, const float* __restrict__ y, const float* __restrict__ coef, int W,
                    int H, size_t P, SsimWin win, float l1scale, float* __restrict__ grad) {
  __shared__ float sc[3][kSsimE][kSsimE + 1];
  __shared__ float hm[3][kSsimE][kSsimT + 1];
  const int ch = blockIdx.z;
  const int x0 = blockIdx.x * kSsimT, y0 = blockIdx.y * kSsimT;
  const size_t plane = static_cast<size_t>(W) * H;
#pragma unroll
  for (int q = 0; q < 3; ++q) load_tile(sc[q], coef + q * P + ch * plane, x0, y0, W, H);
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < kSsimE; r += 8) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kSsimR; ++k) {
      const float w = win.g[k];
      a0 += w * sc[0][r][tx + k];
      a1 += w * sc[1][r][tx + k];
      a2 += w * sc[2][r][tx + k];
    }
    hm[0][r][tx] = a0;
    hm[1][r][tx] = a1;
    hm[2][r][tx] = a2;
  }
  __syncthreads();
  for (int r = ty; r < kSsimT; r += 8) {
    const int py = y0 + r, px = x0 + tx;
    if (px >= W || py >= H) continue;
    float ga = 0.f, gb = 0.f, gc = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kSsimR; ++k) {
      const float w = win.g[k];
      ga += w * hm[0][r + k][tx];
      gb += w * hm[1][r + k][tx];
      gc += w * hm[2][r + k][tx];
    }
    const size_t pix = ch * plane + static_cast<size_t>(py) * W + px;
    const float xv = x[pix], yv = y[pix];
    const float d = xv - yv;
    const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    grad[pix] = ga + 2.f * xv * gb + yv * gc + l1scale * sg;
  }
}

// out[0] = L, out[1] = L1, out[2] = mean SSIM.
__global__ void ssim_final_kernel(const float* __restrict__ part, int nb, double inv_p, float lam,
                                  float* __restrict__ out) {
  __shared__ double s[2][256];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nb; k += 256) {
    a += part[2 * k];
    b += part[2 * k + 1];
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
    const double ssim = ta * inv_p, l1 = tb * inv_p;
    out[0] = static_cast<float>((1.0 - lam) * l1 + lam * (1.0 - ssim));
    out[1] = static_cast<float>(l1);
    out[2] = static_cast<float>(ssim);
  }
}

}  // namespace r4g

using namespace r4g;

namespace {
size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
int ssim_blocks(int C, int H, int W) {
  return ((W + kSsimT - 1) / kSsimT) * ((H + kSsimT - 1) / kSsimT) * C;
}
}  // namespace

extern "C" {

r4g_status r4g_image_loss_scratch_bytes(int32_t channels, int32_t height, int32_t width, size_t* bytes) {
  if (!bytes || channels < 1 || channels > 64 || height < 1 || width < 1 || height > 32768 || width > 32768) {
    set_last_error("bad image size");
    return R4G_EINVAL;
  }
  const size_t p = static_cast<size_t>(channels) * height * width;
  *bytes = al256(3 * p * sizeof(float)) + al256(2 * sizeof(float) * (ssim_blocks(channels, height, width) + 1));
  return R4G_OK;
}

r4g_status r4g_image_loss(const float* image, const float* target, int32_t channels, int32_t height,
                          int32_t width, float lambda_ssim, float* out_loss, float* grad_image, void* scratch,
                          size_t scratch_bytes, void* stream) {
  size_t need = 0;
  r4g_status st = r4g_image_loss_scratch_bytes(channels, height, width, &need);
  if (st != R4G_OK) return st;
  if (!image || !target || !out_loss || !scratch) {
    set_last_error("NULL argument");
    return R4G_EINVAL;
  }
  if (!(lambda_ssim >= 0.0f && lambda_ssim <= 1.0f)) {
    set_last_error("lambda_ssim must be in [0, 1]");
    return R4G_EINVAL;
  }
  if (scratch_bytes < need || (reinterpret_cast<uintptr_t>(scratch) & 255)) {
    set_last_error("scratch smaller than r4g_image_loss_scratch_bytes or not 256-byte aligned");
    return R4G_EWORKSPACE;
  }
  SsimWin win;
  double sum = 0.0;
  for (int k = 0; k <= 2 * kSsimR; ++k) sum += std::exp(-(k - kSsimR) * (k - kSsimR) / (2.0 * 1.5 * 1.5));
  for (int k = 0; k <= 2 * kSsimR; ++k)
    win.g[k] = static_cast<float>(std::exp(-(k - kSsimR) * (k - kSsimR) / (2.0 * 1.5 * 1.5)) / sum);
  const size_t P = static_cast<size_t>(channels) * height * width;
  float* coef = static_cast<float*>(scratch);
  float* part = reinterpret_cast<float*>(static_cast<char*>(scratch) + al256(3 * P * sizeof(float)));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const dim3 grid((width + kSsimT - 1) / kSsimT, (height + kSsimT - 1) / kSsimT, channels), block(32, 8);
  const float gscale = static_cast<float>(-static_cast<double>(lambda_ssim) / P);  // dL/dm
  ssim_fwd_kernel<<<grid, block, 0, s>>>(image, target, width, height, P, win, gscale, coef, part);
  if (grad_image)
    ssim_bwd_kernel<<<grid, block, 0, s>>>(image, target, coef, width, height, P, win,
                                           static_cast<float>((1.0 - lambda_ssim) / P), grad_image);
  ssim_final_kernel<<<1, 256, 0, s>>>(part, ssim_blocks(channels, height, width), 1.0 / P, lambda_ssim, out_loss);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return R4G_ECUDA;
  }
  return R4G_OK;
}

}  // extern "C"
