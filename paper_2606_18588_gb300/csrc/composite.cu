// Global composition (Eq. 5) and its adjoint (Eq. 6-7), one thread per pixel of every
// view of the batch, plus the L1 photometric loss.
//
// Order: subsets sorted per pixel by the normalised depth D^m / (1 - T^m), a convex
// combination of the subset's contributor depths (Eq. 4 read as D = sum d alpha T);
// ties go to the lower subset index and subsets with no contributor (T^m = 1) go last.
// Forward: C = sum_j C^{m_j} P_j + bg P_L with P_j = prod_{i<j} T^{m_i}, stopping once
// P_j < eps_comp (saturation, Sec. 4.2).  Adjoint per included subset m_j:
//   dL/dC^{m_j} = g P_j,  dL/dT^{m_j} = <g, P_j S_j> + gT P_j prod_{i>j} T^{m_i},
// with the suffix S_j = C^{m_{j+1}} + T^{m_{j+1}} S_{j+1}, S_{L-1} = bg.  Subsets after
// the cut get zero.
#include "common.cuh"

namespace splx {

template <int MK>
struct PixOrder {
  float T[MK], key[MK];
  int ord[MK];
  int K;
  uint64_t outside;  // bit m: the pixel's tile lies outside subset m's visible region

  // Partials of subsets whose visible region misses the pixel's tile were never written:
  // they are empty (C = 0, T = 1, D = 0) and are not read.
  __device__ __forceinline__ void load(const BatchDev& b, int v, int64_t p, int W) {
    K = b.K;
    outside = 0;
    int tx = 0, ty = 0;
    if (b.omega) {
      const int sh = __ffs(b.tile) - 1;  // the tile side is a power of two
      const uint32_t py = (uint32_t)p / (uint32_t)W;
      tx = (int)(((uint32_t)p - py * (uint32_t)W) >> sh);
      ty = (int)(py >> sh);
    }
#pragma unroll
    for (int m = 0; m < MK; ++m) {
      if (m < K) {
        if (!in_omega(b, v, m, tx, ty)) {
          outside |= 1ull << m;
          T[m] = 1.0f;
          key[m] = __int_as_float(0x7f800000);
          continue;
        }
        const ImgDev& im = b.imgs[v * b.K + m];
        const float t = im.T[p];
        const float d = im.D[p];
        T[m] = t;
        key[m] = t < 1.0f ? d / (1.0f - t) : __int_as_float(0x7f800000);
      }
    }
    // insertion sort of indices by (key, index): stable
    for (int m = 0; m < K; ++m) {
      int j = m;
      const float km = key[m];
      while (j > 0 && key[ord[j - 1]] > km) {
        ord[j] = ord[j - 1];
        --j;
      }
      ord[j] = m;
    }
  }
};

template <int MK>
__global__ void __launch_bounds__(256) k_composite(const BatchDev b, int64_t total) {
  const int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gp >= total) return;
  const int v = view_of(b.pix_off, b.V, gp);
  const ViewDev& cam = b.views[v];
  const int64_t HW = (int64_t)cam.W * cam.H;
  const int64_t p = gp - b.pix_off[v];
  PixOrder<MK> po;
  po.load(b, v, p, cam.W);
  float P = 1.0f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  for (int j = 0; j < po.K; ++j) {
    if (P < b.eps_comp) break;
    const int m = po.ord[j];
    if ((po.outside >> m) & 1ull) continue;  // empty: adds nothing, T = 1
    const float* rgb = b.imgs[v * b.K + m].rgb;
    c0 = fmaf(rgb[p], P, c0);
    c1 = fmaf(rgb[HW + p], P, c1);
    c2 = fmaf(rgb[2 * HW + p], P, c2);
    P *= po.T[m];
  }
  float* orgb = b.out_rgb + 3 * b.pix_off[v];
  orgb[p] = fmaf(b.bg[0], P, c0);
  orgb[HW + p] = fmaf(b.bg[1], P, c1);
  orgb[2 * HW + p] = fmaf(b.bg[2], P, c2);
  if (b.out_T) b.out_T[b.pix_off[v] + p] = P;
}

template <int MK>
__global__ void __launch_bounds__(256) k_composite_bwd(const BatchDev b, int64_t total) {
  const int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gp >= total) return;
  const int v = view_of(b.pix_off, b.V, gp);
  const ViewDev& cam = b.views[v];
  const int64_t HW = (int64_t)cam.W * cam.H;
  const int64_t p = gp - b.pix_off[v];
  PixOrder<MK> po;
  po.load(b, v, p, cam.W);
  float Pj[MK];
  float P = 1.0f;
  int L = 0;
  for (int j = 0; j < po.K; ++j) {
    if (P < b.eps_comp) break;
    Pj[j] = P;
    P *= po.T[po.ord[j]];
    ++L;
  }
  const float* dl = b.dL_drgb + 3 * b.pix_off[v];
  const float g0 = dl[p], g1 = dl[HW + p], g2 = dl[2 * HW + p];
  const float gT = b.dL_dT ? b.dL_dT[b.pix_off[v] + p] : 0.0f;
  float S0 = b.bg[0], S1 = b.bg[1], S2 = b.bg[2], Rt = 1.0f;
  for (int j = po.K - 1; j >= 0; --j) {
    const int m = po.ord[j];
    const ImgDev& im = b.imgs[v * b.K + m];
    if ((po.outside >> m) & 1ull) continue;  // empty and never rendered: T = 1, C = 0
    if (j >= L) {
      im.gCT[p] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float Pm = Pj[j];
    const float gTm = (g0 * S0 + g1 * S1 + g2 * S2) * Pm + gT * Pm * Rt;
    im.gCT[p] = make_float4(g0 * Pm, g1 * Pm, g2 * Pm, gTm);
    const float Tm = po.T[m];
    S0 = fmaf(Tm, S0, im.rgb[p]);
    S1 = fmaf(Tm, S1, im.rgb[HW + p]);
    S2 = fmaf(Tm, S2, im.rgb[2 * HW + p]);
    Rt *= Tm;
  }
}

template <int MK>
static void launch_c(const BatchDev& b, int64_t total, bool bwd, cudaStream_t s) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((total + threads - 1) / threads);
  if (bwd) k_composite_bwd<MK><<<blocks, threads, 0, s>>>(b, total);
  else k_composite<MK><<<blocks, threads, 0, s>>>(b, total);
}

static void dispatch(const BatchDev& b, int64_t total, bool bwd, cudaStream_t s) {
  if (total <= 0) return;
  if (b.K <= 1) launch_c<1>(b, total, bwd, s);
  else if (b.K <= 4) launch_c<4>(b, total, bwd, s);
  else if (b.K <= 8) launch_c<8>(b, total, bwd, s);
  else if (b.K <= 16) launch_c<16>(b, total, bwd, s);
  else if (b.K <= 32) launch_c<32>(b, total, bwd, s);
  else launch_c<64>(b, total, bwd, s);
  count_launch();
}

void launch_composite(const BatchDev& b, int64_t total, cudaStream_t s) { dispatch(b, total, false, s); }
void launch_composite_bwd(const BatchDev& b, int64_t total, cudaStream_t s) { dispatch(b, total, true, s); }

// ---------------------------------------------------------------- stale saturation state
// Sec. 4.2 step 2: the composition of this visit finds the pixels where the subsets in
// front have saturated; in the view's next visit the subsets behind leave those pixels.
// Per pixel: the prefix product of the partial transmittances in the view's front-to-back
// order (FP32, multiplied in that order, as the exact waves do), over the ranks below the
// old state (ranks at or beyond it were left empty); the new state is the first rank whose
// prefix before it is below eps_comp, or 255 (none).  Ranks pruned by the old state count
// as transparent, so where the prefix no longer saturates they all come back.  Subsets
// whose visible region leaves the pixel's tile out have no partial there (transparent).
__global__ void __launch_bounds__(256) k_sat_update(const BatchDev b,
                                                    const int32_t* __restrict__ order,
                                                    int64_t total) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int v = view_of(b.pix_off, b.V, q);
    const int64_t p = q - b.pix_off[v];
    const ViewDev& cam = b.views[v];
    const int px = (int)(p % cam.W), py = (int)(p / cam.W);
    const int tx = px / b.tile, ty = py / b.tile;
    uint8_t* sp = b.sat[v];
    const int lim = min((int)sp[p], b.K);
    float prefix = 1.0f;
    int out = 255;
    for (int r = 0; r < lim; ++r) {
      const int k = order[v * b.K + r];
      if (!in_omega(b, v, k, tx, ty)) continue;
      prefix *= b.imgs[v * b.K + k].T[p];
      if (prefix < b.eps_comp) {
        out = r + 1 < b.K ? r + 1 : 255;
        break;
      }
    }
    sp[p] = (uint8_t)out;
  }
}

void launch_sat_update(const BatchDev& b, const int32_t* order, int64_t total, cudaStream_t s) {
  if (total <= 0 || !b.sat) return;
  int64_t blocks = (total + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * 16;
  if (blocks > cap) blocks = cap;
  k_sat_update<<<(unsigned)blocks, 256, 0, s>>>(b, order, total);
  count_launch();
}

// ---------------------------------------------------------------- L1 loss
__global__ void __launch_bounds__(256) k_loss_l1(const float* __restrict__ img, const float* __restrict__ tgt,
                                                 int64_t n, float* loss, float* __restrict__ dL) {
  __shared__ float sw[8];
  const float inv = 1.0f / (float)n;
  float acc = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = img[i] - tgt[i];
    acc += fabsf(d);
    if (dL) dL[i] = d > 0.0f ? inv : (d < 0.0f ? -inv : 0.0f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sw[w];
    atomicAdd(loss, t * inv);
  }
}

void launch_loss_l1(const float* img, const float* target, int64_t n, float* loss, float* dL,
                    cudaStream_t s) {
  cudaMemsetAsync(loss, 0, sizeof(float), s);
  if (n <= 0) return;
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * 16;
  if (blocks > cap) blocks = cap;
  k_loss_l1<<<(unsigned)blocks, 256, 0, s>>>(img, target, n, loss, dL);
  count_launch();
}

}  // namespace splx
