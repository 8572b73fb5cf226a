// Binning and per-tile depth sort (Sec. 2 step 2 "Sorting"), bucketed by tile.
//
// The projection kernel counts the (Gaussian, tile) pairs of every image tile with
// atomics; an exclusive scan of those counts gives each tile's segment.  fill writes one
// key per pair into its tile's segment, key = FP32 depth bits << 32 | Gaussian index,
// taking its slot by counting the tile's counter back down (the counters end at zero).
// Keys are unique within a tile, so sorting each segment by the full 64-bit key yields the
// (depth, index) order exactly, whatever order fill placed them in.  Segments are sorted
// in shared memory (bitonic network) by one CTA each: up to 2048 keys in a 256-thread CTA,
// up to 16384 in a 1024-thread CTA; longer segments use an in-CTA stable LSD radix sort in
// global memory.  Every pair is read and written a handful of times instead of once per
// 8-bit pass over 50+ key bits.
#include "common.cuh"

namespace splx {

namespace {

constexpr int kSmallKeys = 2048;
constexpr int kSmallThreads = 256;
constexpr int kBigKeys = 16384;
constexpr int kBigThreads = 1024;

__device__ __forceinline__ int next_pow2(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

// Ascending bitonic sort of s[0, P) in shared memory (P a power of two), NT threads.
template <int NT>
__device__ __forceinline__ void bitonic_smem(uint64_t* s, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < (P >> 1); i += NT) {
        const int lo = 2 * j * (i / j) + (i % j);
        const int hi = lo + j;
        const uint64_t a = s[lo], c = s[hi];
        const bool up = (lo & k) == 0;
        if ((a > c) == up) {
          s[lo] = c;
          s[hi] = a;
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ void segment_of(const BatchDev& b, int64_t t, uint32_t& s, uint32_t& e) {
  const uint64_t cap = (uint64_t)b.capacity;
  uint64_t s64 = b.tile_start[t], e64 = b.tile_start[t + 1];
  if (s64 > cap) s64 = cap;
  if (e64 > cap) e64 = cap;
  if (e64 < s64) e64 = s64;
  s = (uint32_t)s64;
  e = (uint32_t)e64;
}

}  // namespace

// ---------------------------------------------------------------- fill
__global__ void __launch_bounds__(256) k_fill(const BatchDev b) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)b.V * b.N) return;
  if (b.counts[idx] == 0) return;
  const int v = (int)(idx / b.N);
  const int64_t g = idx - (int64_t)v * b.N;
  const int k = subset_of(b, g);
  const ViewDev& cam = b.views[v];
  const Rec* r = b.rec + idx;
  const float4 rb = r->b;
  const uint32_t rx = __float_as_uint(rb.w), ry = __float_as_uint(r->c.w);
  const int B_ = b.tile;
  const int tx0 = (int)(rx & 0xFFFFu) / B_, tx1 = (int)(rx >> 16) / B_;
  const int ty0 = (int)(ry & 0xFFFFu) / B_, ty1 = (int)(ry >> 16) / B_;
  const uint64_t key_hi = (uint64_t)__float_as_uint(rb.z) << 32;
  const int64_t base = b.tile_base[v] + (int64_t)k * cam.tiles_x * cam.tiles_y;
  bool overflow = false;
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) {
      const int64_t t = base + (int64_t)ty * cam.tiles_x + tx;
      const uint64_t pos = (uint64_t)b.tile_start[t] + (atomicSub(&b.tile_cnt[t], 1u) - 1u);
      if (pos < (uint64_t)b.capacity) b.keys[pos] = key_hi | (uint64_t)(uint32_t)g;
      else overflow = true;
    }
  if (overflow) atomicOr(b.status, ST_CAPACITY);
}

void launch_fill(const BatchDev& b, cudaStream_t s) {
  const int64_t n = (int64_t)b.V * b.N;
  const int64_t blocks = (n + 255) / 256;
  if (blocks == 0) return;
  k_fill<<<(unsigned)blocks, 256, 0, s>>>(b);
  count_launch();
}

// ---------------------------------------------------------------- segment sorts
__global__ void __launch_bounds__(kSmallThreads) k_seg_sort_small(const BatchDev b) {
  __shared__ uint64_t sk[kSmallKeys];
  const int64_t t = blockIdx.x;
  uint32_t s, e;
  segment_of(b, t, s, e);
  if (threadIdx.x == 0) b.ranges[t] = make_uint2(s, e);
  const int n = (int)(e - s);
  if (n <= 1) return;
  if (n > kSmallKeys) {
    if (threadIdx.x == 0) {
      const unsigned i = atomicAdd(b.big_count, 1u);
      b.big_list[i] = (uint32_t)t;
    }
    return;
  }
  const int P = next_pow2(n);
  uint64_t* keys = b.keys + s;
  for (int i = threadIdx.x; i < P; i += kSmallThreads) sk[i] = i < n ? keys[i] : ~0ull;
  __syncthreads();
  bitonic_smem<kSmallThreads>(sk, P);
  for (int i = threadIdx.x; i < n; i += kSmallThreads) keys[i] = sk[i];
}

namespace {

// In-CTA stable LSD radix sort of a[0, n) by the full 64-bit key (8 passes of 8 bits),
// ping-ponging with tmp; the result ends in a.  smem: 32 x 256 warp counters + 2 x 256.
__device__ void cta_lsd_sort(uint64_t* a, uint64_t* tmp, int n, uint32_t* sm) {
  constexpr int NW = kBigThreads / 32;
  uint32_t* wcnt = sm;                    // [NW][256]
  uint32_t* base = sm + NW * 256;         // [256] running output offset of each digit
  uint32_t* ctot = base + 256;            // [256] digit totals of the current chunk
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 8 * pass;
    const uint64_t* src = (pass & 1) ? tmp : a;
    uint64_t* dst = (pass & 1) ? a : tmp;
    for (int d = threadIdx.x; d < 256; d += kBigThreads) base[d] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kBigThreads) atomicAdd(&base[(src[i] >> shift) & 0xFFu], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      for (int d = 0; d < 256; ++d) {
        const uint32_t c = base[d];
        base[d] = run;
        run += c;
      }
    }
    __syncthreads();
    // chunks of 4 x 1024 keys in order; warp w owns 128 consecutive keys of a chunk
    for (int c0 = 0; c0 < n; c0 += 4 * kBigThreads) {
      for (int d = threadIdx.x; d < NW * 256; d += kBigThreads) wcnt[d] = 0;
      __syncthreads();
      uint64_t kv[4];
      uint32_t rk[4], dg[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = c0 + w * 128 + r * 32 + lane;
        const bool valid = i < n;
        kv[r] = valid ? src[i] : 0ull;
        const uint32_t d = valid ? (uint32_t)(kv[r] >> shift) & 0xFFu : 0x100u;
        dg[r] = d;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (valid) before = wcnt[w * 256 + d];
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[w * 256 + d] = before + __popc(peers);
        __syncwarp();
        rk[r] = before + __popc(peers & lt);
      }
      __syncthreads();
      for (int d = threadIdx.x; d < 256; d += kBigThreads) {
        uint32_t run = 0;
        for (int ww = 0; ww < NW; ++ww) {
          const uint32_t c = wcnt[ww * 256 + d];
          wcnt[ww * 256 + d] = run;
          run += c;
        }
        ctot[d] = run;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (dg[r] < 0x100u) dst[base[dg[r]] + wcnt[w * 256 + dg[r]] + rk[r]] = kv[r];
      __syncthreads();
      for (int d = threadIdx.x; d < 256; d += kBigThreads) base[d] += ctot[d];
      __syncthreads();
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(kBigThreads) k_seg_sort_big(const BatchDev b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(smem_raw);
  const unsigned count = *b.big_count;
  for (unsigned i = blockIdx.x; i < count; i += gridDim.x) {
    const int64_t t = b.big_list[i];
    if (t >= b.n_tiles) continue;
    uint32_t s, e;
    segment_of(b, t, s, e);
    const int n = (int)(e - s);
    uint64_t* keys = b.keys + s;
    if (n <= kBigKeys) {
      const int P = next_pow2(n);
      for (int j = threadIdx.x; j < P; j += kBigThreads) sk[j] = j < n ? keys[j] : ~0ull;
      __syncthreads();
      bitonic_smem<kBigThreads>(sk, P);
      for (int j = threadIdx.x; j < n; j += kBigThreads) keys[j] = sk[j];
    } else {
      cta_lsd_sort(keys, b.keys_alt + s, n, reinterpret_cast<uint32_t*>(smem_raw));
    }
    __syncthreads();
  }
}

size_t seg_sort_big_smem() { return (size_t)kBigKeys * sizeof(uint64_t); }

void launch_seg_sort(const BatchDev& b, cudaStream_t s) {
  if (b.n_tiles == 0) return;
  k_seg_sort_small<<<(unsigned)b.n_tiles, kSmallThreads, 0, s>>>(b);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_seg_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)seg_sort_big_smem());
    attr = true;
  }
  k_seg_sort_big<<<2 * 152, kBigThreads, seg_sort_big_smem(), s>>>(b);
  count_launch(2);
}

}  // namespace splx
