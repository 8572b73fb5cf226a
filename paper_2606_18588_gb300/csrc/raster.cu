// Local rendering of every (view, subset) tile: forward (Eq. 1-4) and backward.
//
// One CTA per image tile (TS x TS pixels, one pixel per thread).  The tile's sorted
// list is walked in batches of TS*TS entries: each thread gathers one 64-byte record
// into shared memory, then every pixel blends the batch front to back.  A pixel takes a
// Gaussian only inside its integer 3-sigma rectangle (so the result does not depend on
// TS), with alpha = min(alpha_max, o 2^(p2)) >= alpha_min, and stops before the
// Gaussian that would take its transmittance below eps_T.  The CTA leaves the list
// once every pixel has stopped (__syncthreads_count).
//
// The backward walks the same list back to front from each pixel's last blended
// entry, recovering T_i = T_{i+1} / (1 - alpha_i) from the stored final T^m, and
// applies the adjoint of Eq. 3-4 with the composite adjoint (dL/dC^m, dL/dT^m of
// Eq. 6-7) as input:
//   dC^m/dc_i = alpha_i T_i,  dC^m/dalpha_i = c_i T_i - B_i / (1 - alpha_i),
//   dT^m/dalpha_i = -T^m / (1 - alpha_i),  B_i = sum_{j>i} c_j alpha_j T_j.
// Per-Gaussian sums over the tile's pixels are reduced with warp shuffles and added to
// the per-(view, Gaussian) 2-D gradient with float4 atomics.
#include "common.cuh"

namespace splx {

// alpha of record (a, b) at pixel centre (pcx, pcy); identical code in forward and
// backward so both take bit-identical decisions.  Returns false if the Gaussian is
// skipped at this pixel.
__device__ __forceinline__ bool eval_alpha(const float4 a, const float4 b, float pcx, float pcy,
                                           float amin, float amax, float& alpha, float& ex,
                                           float& dx, float& dy, bool& clamped) {
  dx = __fsub_rn(pcx, a.x);
  dy = __fsub_rn(pcy, a.y);
  const float t1 = __fmul_rn(a.w, __fmul_rn(dx, dy));
  const float t2 = __fmaf_rn(__fmul_rn(b.x, dy), dy, t1);
  const float p2 = __fmaf_rn(__fmul_rn(a.z, dx), dx, t2);
  if (p2 > 0.0f) return false;
  ex = exp2f(p2);
  const float raw = __fmul_rn(b.y, ex);
  clamped = raw > amax;
  alpha = clamped ? amax : raw;
  return alpha >= amin;
}

__device__ __forceinline__ bool in_rect(uint32_t rx, uint32_t ry, int px, int py) {
  const int x0 = (int)(rx & 0xFFFFu), x1 = (int)(rx >> 16);
  const int y0 = (int)(ry & 0xFFFFu), y1 = (int)(ry >> 16);
  return px >= x0 && px <= x1 && py >= y0 && py <= y1;
}

// Adds per-thread counts into counters[slot] with one atomic per warp.
__device__ __forceinline__ void flush_counter(unsigned long long* counters, int slot, unsigned v) {
  if (!counters) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(counters + slot, (unsigned long long)v);
}

struct TileInfo {
  int v, k, px, py, W, H;
  int64_t t;
};

__device__ __forceinline__ TileInfo decode_tile(const BatchDev& b, int64_t id, int TS) {
  TileInfo ti;
  ti.v = view_of(b.tile_base, b.V, id);
  const ViewDev& cam = b.views[ti.v];
  const int64_t nt = (int64_t)cam.tiles_x * cam.tiles_y;
  const int64_t rem = id - b.tile_base[ti.v];
  ti.k = (int)(rem / nt);
  ti.t = rem - (int64_t)ti.k * nt;
  const int tx = (int)(ti.t % cam.tiles_x), ty = (int)(ti.t / cam.tiles_x);
  ti.px = tx * TS + (int)(threadIdx.x % TS);
  ti.py = ty * TS + (int)(threadIdx.x / TS);
  ti.W = cam.W;
  ti.H = cam.H;
  return ti;
}

template <int TS>
__global__ void __launch_bounds__(TS * TS) k_raster_fwd(const BatchDev b, const uint32_t* __restrict__ vals) {
  constexpr int NT = TS * TS;
  constexpr int NB = NT > 512 ? 512 : NT;  // records staged per batch
  __shared__ float4 sA[NB], sB[NB], sC[NB];
  const int64_t id = blockIdx.x;
  const TileInfo ti = decode_tile(b, id, TS);
  const bool inside = ti.px < ti.W && ti.py < ti.H;
  const uint2 rg = b.ranges[id];
  const int64_t start = rg.x, end = rg.y > rg.x ? rg.y : rg.x;
  const Rec* rec = b.rec + (int64_t)ti.v * b.N;
  const float pcx = (float)ti.px + 0.5f, pcy = (float)ti.py + 0.5f;
  const float amin = b.alpha_min, amax = b.alpha_max, epsT = b.eps_T;
  float T = 1.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, D = 0.0f;
  int last = -1;
  bool done = !inside;
  unsigned n_eval = 0, n_blend = 0;
  for (int64_t base = start; base < end; base += NB) {
    if (__syncthreads_count(done) == NT) break;
    const int64_t j = base + threadIdx.x;
    if (threadIdx.x < NB && j < end) {
      uint32_t g = vals[j];
      if (g >= (uint32_t)b.N) { atomicOr(b.status, ST_BOUNDS); g = 0; }
      const Rec* r = rec + g;
      sA[threadIdx.x] = r->a;
      sB[threadIdx.x] = r->b;
      sC[threadIdx.x] = r->c;
    }
    __syncthreads();
    if (!done) {
      const int cnt = (int)((end - base) < NB ? (end - base) : NB);
      int jj = 0;
      for (; jj < cnt; ++jj) {
        const float4 B = sB[jj];
        const float4 C = sC[jj];
        if (!in_rect(__float_as_uint(B.w), __float_as_uint(C.w), ti.px, ti.py)) continue;
        const float4 A = sA[jj];
        float alpha, ex, dx, dy;
        bool cl;
        if (!eval_alpha(A, B, pcx, pcy, amin, amax, alpha, ex, dx, dy, cl)) continue;
        const float Tn = T * (1.0f - alpha);
        if (Tn < epsT) { done = true; ++jj; break; }
        const float w = alpha * T;
        c0 = fmaf(C.x, w, c0);
        c1 = fmaf(C.y, w, c1);
        c2 = fmaf(C.z, w, c2);
        D = fmaf(B.z, w, D);
        T = Tn;
        last = (int)(base - start) + jj;
        ++n_blend;
      }
      n_eval += (unsigned)jj;
    }
  }
  flush_counter(b.counters, 0, n_eval);
  flush_counter(b.counters, 1, n_blend);
  if (inside) {
    const ImgDev im = b.imgs[ti.v * b.K + ti.k];
    const int64_t HW = (int64_t)ti.W * ti.H;
    const int64_t p = (int64_t)ti.py * ti.W + ti.px;
    im.rgb[p] = c0;
    im.rgb[HW + p] = c1;
    im.rgb[2 * HW + p] = c2;
    im.T[p] = T;
    im.D[p] = D;
    im.last[p] = last;
  }
}

template <int TS>
__global__ void __launch_bounds__(TS * TS) k_raster_bwd(const BatchDev b, const uint32_t* __restrict__ vals) {
  constexpr int NB = TS * TS > 512 ? 512 : TS * TS;  // records staged per batch
  __shared__ float4 sA[NB], sB[NB], sC[NB];
  __shared__ uint32_t sG[NB];
  __shared__ int s_maxlast;
  const int64_t id = blockIdx.x;
  const TileInfo ti = decode_tile(b, id, TS);
  const bool inside = ti.px < ti.W && ti.py < ti.H;
  const uint2 rg = b.ranges[id];
  const int64_t start = rg.x;
  const ImgDev im = b.imgs[ti.v * b.K + ti.k];
  const int64_t p = (int64_t)ti.py * ti.W + ti.px;
  float4 gct = make_float4(0.f, 0.f, 0.f, 0.f);
  float Tf = 1.0f;
  int mylast = -1;
  if (inside) {
    gct = im.gCT[p];
    Tf = im.T[p];
    mylast = im.last[p];
    if (gct.x == 0.0f && gct.y == 0.0f && gct.z == 0.0f && gct.w == 0.0f) mylast = -1;
  }
  if (threadIdx.x == 0) s_maxlast = -1;
  __syncthreads();
  if (mylast >= 0) atomicMax(&s_maxlast, mylast);
  __syncthreads();
  const int maxlast = s_maxlast;
  if (maxlast < 0) return;

  const Rec* rec = b.rec + (int64_t)ti.v * b.N;
  float4* g2 = b.grad2d + (int64_t)ti.v * b.N * 3;
  const float pcx = (float)ti.px + 0.5f, pcy = (float)ti.py + 0.5f;
  const float amin = b.alpha_min, amax = b.alpha_max;
  float T = Tf;
  float B0 = 0.f, B1 = 0.f, B2 = 0.f;
  const float ninvTf = -Tf * gct.w;
  const int lane = threadIdx.x & 31;
  unsigned n_evalb = 0;

  for (int top = maxlast; top >= 0; top -= NB) {
    const int lo = top - NB + 1 > 0 ? top - NB + 1 : 0;
    __syncthreads();
    {
      const int j = top - (int)threadIdx.x;  // shared slot t holds entry top - t
      if ((int)threadIdx.x < NB && j >= lo) {
        uint32_t g = vals[start + j];
        if (g >= (uint32_t)b.N) { atomicOr(b.status, ST_BOUNDS); g = 0; }
        const Rec* r = rec + g;
        sA[threadIdx.x] = r->a;
        sB[threadIdx.x] = r->b;
        sC[threadIdx.x] = r->c;
        sG[threadIdx.x] = g;
      }
    }
    __syncthreads();
    const int cnt = top - lo + 1;
    if (mylast >= lo) n_evalb += (unsigned)((mylast < top ? mylast : top) - lo + 1);
    for (int jj = 0; jj < cnt; ++jj) {
      const int j = top - jj;
      float gu = 0.f, gv = 0.f, gA = 0.f, gB = 0.f, gC = 0.f, go = 0.f, gr = 0.f, gg = 0.f, gb = 0.f;
      bool act = false;
      if (j <= mylast) {
        const float4 Bv = sB[jj];
        const float4 Cv = sC[jj];
        if (in_rect(__float_as_uint(Bv.w), __float_as_uint(Cv.w), ti.px, ti.py)) {
          const float4 Av = sA[jj];
          float alpha, ex, dx, dy;
          bool cl;
          if (eval_alpha(Av, Bv, pcx, pcy, amin, amax, alpha, ex, dx, dy, cl)) {
            act = true;
            const float om = 1.0f - alpha;
            const float rinv = 1.0f / om;
            const float Ti = T * rinv;
            const float aT = alpha * Ti;
            gr = gct.x * aT;
            gg = gct.y * aT;
            gb = gct.z * aT;
            float ga = gct.x * (Cv.x * Ti - B0 * rinv) + gct.y * (Cv.y * Ti - B1 * rinv) +
                       gct.z * (Cv.z * Ti - B2 * rinv) + ninvTf * rinv;
            if (!cl) {
              go = ga * ex;
              const float gp = ga * alpha;  // dL/dpower
              // conic (A, B, C) recovered from the scaled record: A = -2 ln2 qa, ...
              const float A_ = -2.0f * kLn2 * Av.z, Bc = -kLn2 * Av.w, C_ = -2.0f * kLn2 * Bv.x;
              gu = (A_ * dx + Bc * dy) * gp;
              gv = (C_ * dy + Bc * dx) * gp;
              gA = -0.5f * dx * dx * gp;
              gB = -dx * dy * gp;
              gC = -0.5f * dy * dy * gp;
            }
            B0 = fmaf(Cv.x, aT, B0);
            B1 = fmaf(Cv.y, aT, B1);
            B2 = fmaf(Cv.z, aT, B2);
            T = Ti;
          }
        }
      }
      if (__any_sync(0xffffffffu, act)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          gu += __shfl_xor_sync(0xffffffffu, gu, o);
          gv += __shfl_xor_sync(0xffffffffu, gv, o);
          gA += __shfl_xor_sync(0xffffffffu, gA, o);
          gB += __shfl_xor_sync(0xffffffffu, gB, o);
          gC += __shfl_xor_sync(0xffffffffu, gC, o);
          go += __shfl_xor_sync(0xffffffffu, go, o);
          gr += __shfl_xor_sync(0xffffffffu, gr, o);
          gg += __shfl_xor_sync(0xffffffffu, gg, o);
          gb += __shfl_xor_sync(0xffffffffu, gb, o);
        }
        if (lane == 0) {
          float4* dst = g2 + (int64_t)sG[jj] * 3;
          atomicAdd(dst, make_float4(gu, gv, gA, gB));
          atomicAdd(dst + 1, make_float4(gC, go, gr, gg));
          atomicAdd(&dst[2].x, gb);
        }
      }
    }
  }
  flush_counter(b.counters, 2, n_evalb);
}

template <int TS>
static void launch_fwd_t(const BatchDev& b, const uint32_t* vals, cudaStream_t s) {
  k_raster_fwd<TS><<<(unsigned)b.n_tiles, TS * TS, 0, s>>>(b, vals);
}
template <int TS>
static void launch_bwd_t(const BatchDev& b, const uint32_t* vals, cudaStream_t s) {
  k_raster_bwd<TS><<<(unsigned)b.n_tiles, TS * TS, 0, s>>>(b, vals);
}

void launch_raster_fwd(const BatchDev& b, const uint32_t* vals, cudaStream_t s) {
  if (b.n_tiles == 0) return;
  switch (b.tile) {
    case 8: launch_fwd_t<8>(b, vals, s); break;
    case 32: launch_fwd_t<32>(b, vals, s); break;
    default: launch_fwd_t<16>(b, vals, s); break;
  }
  count_launch();
}

void launch_raster_bwd(const BatchDev& b, const uint32_t* vals, cudaStream_t s) {
  if (b.n_tiles == 0) return;
  switch (b.tile) {
    case 8: launch_bwd_t<8>(b, vals, s); break;
    case 32: launch_bwd_t<32>(b, vals, s); break;
    default: launch_bwd_t<16>(b, vals, s); break;
  }
  count_launch();
}

}  // namespace splx
