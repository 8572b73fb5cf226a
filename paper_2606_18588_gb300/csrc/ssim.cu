// Photometric loss with the structural term (Sec. 2, step 4: L = L_RGB + L_D-SSIM, read as
// L = (1 - lam) L1 + lam (1 - SSIM), lam = 0.2 in 3DGS practice) over the concatenated
// views of a batch, and its gradient with respect to the rendered images.
//
// SSIM per channel uses an 11 x 11 Gaussian window (sigma 1.5, weights w_i w_j) with zero
// padding, C1 = 0.01^2, C2 = 0.03^2; both terms are means over all pixels and channels.
// With the local means mx, my, E[x^2], E[y^2], E[xy] of the window,
//   S = (2 mx my + C1)(2 cov + C2) / ((mx^2 + my^2 + C1)(vx + vy + C2)).
// k_ssim_fwd computes S and its partial derivatives with respect to mx, E[x^2] and E[xy]
// per pixel; since every pixel's statistics are windowed sums of x, x^2 and x y, the
// gradient of sum S is  w * dS/dmx + 2 x (w * dS/dE[x^2]) + y (w * dS/dE[xy])  (the window
// is symmetric, so the adjoint of the windowed sum is itself), which k_ssim_bwd forms and
// adds to the L1 term.  Both kernels work on 32 x 32 output tiles with a 5-pixel halo in
// shared memory and separable passes.
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace splx {

namespace {

constexpr int kT = 32;                // output tile side
constexpr int kR = 5;                 // window radius
constexpr int kS = kT + 2 * kR;       // staged side (42)
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// Normalised 11-tap Gaussian, sigma 1.5 (weights computed once on the host).
__constant__ float c_w[2 * kR + 1];

// Work item = (view, channel, tile): decoded from the global block index.
struct SsimItem {
  int v, ch, x0, y0, W, H;
  int64_t base;  // offset of the channel plane in the concatenated images
};

__device__ __forceinline__ SsimItem decode(const LossImgs& L, int64_t blk) {
  SsimItem it;
  it.v = view_of(L.blk_off, L.V, blk);
  const int64_t r = blk - L.blk_off[it.v];
  it.W = L.W[it.v];
  it.H = L.H[it.v];
  const int tx = (it.W + kT - 1) / kT, ty = (it.H + kT - 1) / kT;
  const int64_t per = (int64_t)tx * ty;
  it.ch = (int)(r / per);
  const int64_t t = r - (int64_t)it.ch * per;
  it.x0 = (int)(t % tx) * kT;
  it.y0 = (int)(t / tx) * kT;
  it.base = 3 * L.pix_off[it.v] + (int64_t)it.ch * it.W * it.H;
  return it;
}

// Stages a (kS x kS) window of plane `a` around the tile (zero outside the image).
__device__ __forceinline__ void stage(const float* __restrict__ a, const SsimItem& it,
                                      float (*s)[kS]) {
  for (int i = threadIdx.x; i < kS * kS; i += blockDim.x) {
    const int r = i / kS, c = i - r * kS;
    const int y = it.y0 + r - kR, x = it.x0 + c - kR;
    s[r][c] = (x >= 0 && x < it.W && y >= 0 && y < it.H) ? a[it.base + (int64_t)y * it.W + x] : 0.0f;
  }
}

__device__ __forceinline__ float hsum(const float (*s)[kS], int r, int c) {
  float acc = 0.0f;
#pragma unroll
  for (int k = 0; k <= 2 * kR; ++k) acc = fmaf(c_w[k], s[r][c + k], acc);
  return acc;
}

template <int NM>
__device__ __forceinline__ void vsum(const float (*h)[kS][kT], int r, int c, float* out) {
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) acc = fmaf(c_w[k], h[m][r + k][c], acc);
    out[m] = acc;
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

}  // namespace

__global__ void __launch_bounds__(256) k_ssim_fwd(const LossImgs L, const float* __restrict__ x,
                                                  const float* __restrict__ y, float* __restrict__ dmx,
                                                  float* __restrict__ dexx, float* __restrict__ dexy,
                                                  double* __restrict__ sums) {
  __shared__ float sx[kS][kS], sy[kS][kS];
  __shared__ float h[5][kS][kT];  // horizontal sums of x, y, x^2, y^2, x y
  __shared__ double red[8];
  const SsimItem it = decode(L, blockIdx.x);
  stage(x, it, sx);
  stage(y, it, sy);
  __syncthreads();
  for (int i = threadIdx.x; i < kS * kT; i += blockDim.x) {
    const int r = i / kT, c = i - r * kT;
    float a[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const float xv = sx[r][c + k], yv = sy[r][c + k], wk = c_w[k];
      a[0] = fmaf(wk, xv, a[0]);
      a[1] = fmaf(wk, yv, a[1]);
      a[2] = fmaf(wk, xv * xv, a[2]);
      a[3] = fmaf(wk, yv * yv, a[3]);
      a[4] = fmaf(wk, xv * yv, a[4]);
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) h[m][r][c] = a[m];
  }
  __syncthreads();
  double s_sum = 0.0, l1_sum = 0.0;
  for (int i = threadIdx.x; i < kT * kT; i += blockDim.x) {
    const int r = i / kT, c = i - r * kT;
    const int px = it.x0 + c, py = it.y0 + r;
    if (px >= it.W || py >= it.H) continue;
    float st[5];
    vsum<5>(h, r, c, st);
    const float mx = st[0], my = st[1];
    const float vx = st[2] - mx * mx, vy = st[3] - my * my, cxy = st[4] - mx * my;
    const float a1 = 2.0f * mx * my + kC1, a2 = 2.0f * cxy + kC2;
    const float b1 = mx * mx + my * my + kC1, b2 = vx + vy + kC2;
    const float ib = 1.0f / (b1 * b2);
    const float S = a1 * a2 * ib;
    const int64_t q = it.base + (int64_t)py * it.W + px;
    dmx[q] = 2.0f * my * (a2 - a1) * ib - 2.0f * mx * S / b1 + 2.0f * mx * S / b2;
    dexx[q] = -S / b2;
    dexy[q] = 2.0f * a1 * ib;
    s_sum += S;
    l1_sum += fabsf(sx[r + kR][c + kR] - sy[r + kR][c + kR]);
  }
  const double ts = block_sum(s_sum, red);
  __syncthreads();
  const double tl = block_sum(l1_sum, red);
  if (threadIdx.x == 0) {
    atomicAdd(sums, ts);
    atomicAdd(sums + 1, tl);
  }
}

__global__ void __launch_bounds__(256) k_ssim_bwd(const LossImgs L, const float* __restrict__ x,
                                                  const float* __restrict__ y,
                                                  const float* __restrict__ dmx,
                                                  const float* __restrict__ dexx,
                                                  const float* __restrict__ dexy, float lam,
                                                  double inv_n, float* __restrict__ dL) {
  __shared__ float sd[3][kS][kS];
  __shared__ float h[3][kS][kT];
  const SsimItem it = decode(L, blockIdx.x);
  stage(dmx, it, sd[0]);
  stage(dexx, it, sd[1]);
  stage(dexy, it, sd[2]);
  __syncthreads();
  for (int i = threadIdx.x; i < kS * kT; i += blockDim.x) {
    const int r = i / kT, c = i - r * kT;
#pragma unroll
    for (int m = 0; m < 3; ++m) h[m][r][c] = hsum(sd[m], r, c);
  }
  __syncthreads();
  const float a = (float)((1.0 - lam) * inv_n), bcoef = (float)(lam * inv_n);
  for (int i = threadIdx.x; i < kT * kT; i += blockDim.x) {
    const int r = i / kT, c = i - r * kT;
    const int px = it.x0 + c, py = it.y0 + r;
    if (px >= it.W || py >= it.H) continue;
    float cv[3];
    vsum<3>(h, r, c, cv);
    const int64_t q = it.base + (int64_t)py * it.W + px;
    const float xv = x[q], yv = y[q];
    const float d = xv - yv;
    const float sgn = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
    dL[q] = a * sgn - bcoef * (cv[0] + 2.0f * xv * cv[1] + yv * cv[2]);
  }
}

__global__ void k_ssim_loss(const double* __restrict__ sums, double inv_n, float lam, float* loss) {
  *loss = (float)((1.0 - lam) * sums[1] * inv_n + lam * (1.0 - sums[0] * inv_n));
}

// Host side ----------------------------------------------------------------------
// Uploads the window weights to the current device (synchronous; called when a context is
// created, never inside a stream capture).
int ssim_init() {
  float w[2 * kR + 1];
  double sum = 0.0, wd[2 * kR + 1];
  for (int k = 0; k <= 2 * kR; ++k) {
    const double t = (double)(k - kR);
    wd[k] = std::exp(-t * t / (2.0 * 1.5 * 1.5));
    sum += wd[k];
  }
  for (int k = 0; k <= 2 * kR; ++k) w[k] = (float)(wd[k] / sum);
  return cudaMemcpyToSymbol(c_w, w, sizeof(w)) == cudaSuccess ? 0 : -1;
}

int64_t ssim_blocks(const LossImgs& L) { return L.blk_off[L.V]; }

void launch_loss_l1_dssim(const LossImgs& L, const float* x, const float* y, float lam,
                          float* dmx, float* dexx, float* dexy, double* sums, float* loss,
                          float* dL, cudaStream_t s) {
  const int64_t blocks = ssim_blocks(L);
  if (blocks == 0) return;
  const double inv_n = 1.0 / (3.0 * (double)L.pix_off[L.V]);
  cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
  k_ssim_fwd<<<(unsigned)blocks, 256, 0, s>>>(L, x, y, dmx, dexx, dexy, sums);
  k_ssim_bwd<<<(unsigned)blocks, 256, 0, s>>>(L, x, y, dmx, dexx, dexy, lam, inv_n, dL);
  k_ssim_loss<<<1, 1, 0, s>>>(sums, inv_n, lam, loss);
  count_launch();
  count_launch();
  count_launch();
}

LossImgs make_loss_imgs(int V, const int* W, const int* H) {
  LossImgs L;
  std::memset(&L, 0, sizeof(L));
  L.V = V;
  for (int v = 0; v < V; ++v) {
    L.W[v] = W[v];
    L.H[v] = H[v];
    L.pix_off[v + 1] = L.pix_off[v] + (int64_t)W[v] * H[v];
    L.blk_off[v + 1] = L.blk_off[v] + 3 * (int64_t)((W[v] + kT - 1) / kT) * ((H[v] + kT - 1) / kT);
  }
  return L;
}

}  // namespace splx
