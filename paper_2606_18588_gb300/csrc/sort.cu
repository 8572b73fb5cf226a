// Device-wide exclusive scan and stable LSD radix sort of (u64 key, u32 value) pairs.
//
// Sort (Sec. 2 step 2 "Sorting"): keys are image-tile id << 32 | FP32 depth bits, so a
// stable sort of pairs emitted in Gaussian-index order yields every tile's list ordered
// by (depth, index).  Each 8-bit pass runs three kernels: per-block digit histograms
// (digit-major), an exclusive scan of those histograms, and a scatter in which each
// block ranks its 4096 keys stably (warp match + per-warp digit counters), stages them
// digit-sorted in shared memory and writes each digit run contiguously.  The item count
// is read on the device (capacity-sized grids), so the sequence is graph-capturable.
#include "common.cuh"

namespace splx {

namespace {

constexpr int kThreads = 256;
constexpr int kIPT = 16;
constexpr int kTile = kThreads * kIPT;  // 4096
constexpr int kRadix = 256;
constexpr int kWarps = kThreads / 32;

// ---------------------------------------------------------------- block scan helpers
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive scan of one value per thread across the block; returns the block total.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T& total, T* sw /* [kWarps] */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const T inc = warp_inclusive_scan(x);
  if (lane == 31) sw[w] = inc;
  __syncthreads();
  if (w == 0) {
    T s = lane < kWarps ? sw[lane] : T(0);
    s = warp_inclusive_scan(s);
    if (lane < kWarps) sw[lane] = s;
  }
  __syncthreads();
  const T wbase = w ? sw[w - 1] : T(0);
  total = sw[kWarps - 1];
  __syncthreads();
  return wbase + inc - x;
}

// ---------------------------------------------------------------- scan kernels
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kThreads) k_scan_reduce(const TIn* __restrict__ in, int64_t n,
                                                          TOut* __restrict__ sums) {
  __shared__ TOut sw[kWarps];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  TOut acc = 0;
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    const int64_t i = base + j * kThreads + threadIdx.x;
    if (i < n) acc += (TOut)in[i];
  }
  TOut total;
  block_exclusive_scan<TOut>(acc, total, sw);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// out[i] = offset[block] + exclusive prefix within the block; out[n] = grand total when
// the block holds the last element.
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kThreads) k_scan_down(const TIn* __restrict__ in, TOut* __restrict__ out,
                                                        int64_t n, const TOut* __restrict__ offs,
                                                        bool write_total) {
  __shared__ TOut tile[kTile];
  __shared__ TOut sw[kWarps];
  const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    const int64_t i = base + j * kThreads + threadIdx.x;
    tile[j * kThreads + threadIdx.x] = i < n ? (TOut)in[i] : TOut(0);
  }
  __syncthreads();
  TOut v[kIPT];
  TOut acc = 0;
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    v[j] = tile[threadIdx.x * kIPT + j];
    acc += v[j];
  }
  TOut total;
  TOut run = block_exclusive_scan<TOut>(acc, total, sw) + (offs ? offs[blockIdx.x] : TOut(0));
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    tile[threadIdx.x * kIPT + j] = run;
    run += v[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    const int64_t i = base + j * kThreads + threadIdx.x;
    if (i < n) out[i] = tile[j * kThreads + threadIdx.x];
  }
  if (write_total && threadIdx.x == kThreads - 1 && base + kTile >= n)
    out[n] = (offs ? offs[blockIdx.x] : TOut(0)) + total;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// bytes of temporary storage for scanning n items (all recursion levels)
size_t scan_levels_bytes(int64_t n, size_t elem) {
  size_t bytes = 0;
  int64_t m = ceil_div(n, kTile);
  while (m > 1) {
    bytes += 2 * (size_t)m * elem + 256;
    m = ceil_div(m, kTile);
  }
  return bytes + 2 * elem + 512;
}

// Exclusive scan in -> out (n items, out[n] written if write_total), recursive on the
// block sums.  temp must hold scan_levels_bytes(n, sizeof(TOut)).
template <typename TIn, typename TOut>
void scan_rec(const TIn* in, TOut* out, int64_t n, bool write_total, char* temp, cudaStream_t s) {
  const int64_t blocks = ceil_div(n, kTile);
  if (blocks <= 1) {
    k_scan_down<TIn, TOut><<<1, kThreads, 0, s>>>(in, out, n, nullptr, write_total);
    count_launch();
    return;
  }
  TOut* sums = reinterpret_cast<TOut*>(temp);
  TOut* offs = sums + blocks;
  char* rest = temp + (((size_t)2 * blocks * sizeof(TOut) + 255) & ~(size_t)255);
  k_scan_reduce<TIn, TOut><<<(unsigned)blocks, kThreads, 0, s>>>(in, n, sums);
  count_launch();
  scan_rec<TOut, TOut>(sums, offs, blocks, false, rest, s);
  k_scan_down<TIn, TOut><<<(unsigned)blocks, kThreads, 0, s>>>(in, out, n, offs, write_total);
  count_launch();
}

// ---------------------------------------------------------------- radix sort kernels
__device__ __forceinline__ int64_t clamp_n(const uint64_t* n_dev, int64_t cap) {
  const uint64_t n = *n_dev;
  return n < (uint64_t)cap ? (int64_t)n : cap;
}

__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint64_t* __restrict__ keys,
                                                         const uint64_t* n_dev, int64_t cap, int shift,
                                                         uint32_t* __restrict__ hist, int64_t nblocks) {
  __shared__ uint32_t cnt[kRadix];
  const int64_t n = clamp_n(n_dev, cap);
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (base < n) {
#pragma unroll
    for (int j = 0; j < kIPT; ++j) {
      const int64_t i = base + j * kThreads + threadIdx.x;
      if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & 0xFFu], 1u);
    }
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

struct ScatterSmem {
  uint64_t keys[kTile];
  uint32_t vals[kTile];
  uint32_t wcnt[kWarps][kRadix];
  uint32_t dstart[kRadix];
  uint32_t gbase[kRadix];
  uint32_t sw[kWarps];
};

__global__ void __launch_bounds__(kThreads) k_radix_scatter(const uint64_t* __restrict__ kin,
                                                            const uint32_t* __restrict__ vin,
                                                            uint64_t* __restrict__ kout,
                                                            uint32_t* __restrict__ vout,
                                                            const uint64_t* n_dev, int64_t cap,
                                                            int shift, const uint32_t* __restrict__ hist,
                                                            int64_t nblocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem& sm = *reinterpret_cast<ScatterSmem*>(smem_raw);
  const int64_t n = clamp_n(n_dev, cap);
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (base >= n) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kWarps * kRadix; d += kThreads) (&sm.wcnt[0][0])[d] = 0;
  __syncthreads();

  // Warp w owns items [w*512, (w+1)*512) of the tile, 32 per round, in index order.
  uint64_t k[kIPT];
  uint32_t val[kIPT];
  uint32_t rank[kIPT];
  uint32_t dig[kIPT];
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    const int64_t i = base + (int64_t)w * (32 * kIPT) + r * 32 + lane;
    const bool valid = i < n;
    k[r] = valid ? kin[i] : 0ull;
    val[r] = valid ? vin[i] : 0u;
    const uint32_t d = valid ? (uint32_t)(k[r] >> shift) & 0xFFu : 0x100u;
    dig[r] = d;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = 0;
    if (valid) before = sm.wcnt[w][d];
    __syncwarp();
    if (valid && (peers & lt) == 0) sm.wcnt[w][d] = before + __popc(peers);
    __syncwarp();
    rank[r] = before + __popc(peers & lt);
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, then over digits (block-local start)
  {
    const int d = threadIdx.x;  // kThreads == kRadix
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
      const uint32_t c = sm.wcnt[ww][d];
      sm.wcnt[ww][d] = run;
      run += c;
    }
    uint32_t total;
    const uint32_t start = block_exclusive_scan<uint32_t>(run, total, sm.sw);
    sm.dstart[d] = start;
    sm.gbase[d] = hist[(int64_t)d * nblocks + blockIdx.x];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    if (dig[r] < 0x100u) {
      const uint32_t pos = sm.dstart[dig[r]] + sm.wcnt[w][dig[r]] + rank[r];
      sm.keys[pos] = k[r];
      sm.vals[pos] = val[r];
    }
  }
  __syncthreads();
  const int64_t cnt = (n - base) < kTile ? (n - base) : kTile;
  for (int j = threadIdx.x; j < cnt; j += kThreads) {
    const uint64_t kk = sm.keys[j];
    const uint32_t d = (uint32_t)(kk >> shift) & 0xFFu;
    const uint64_t dst = (uint64_t)sm.gbase[d] + (uint64_t)(j - sm.dstart[d]);
    kout[dst] = kk;
    vout[dst] = sm.vals[j];
  }
}

}  // namespace

size_t scan_u32_u64_temp_bytes(int64_t n) { return scan_levels_bytes(n, sizeof(uint64_t)); }

void scan_u32_u64(const uint32_t* in, uint64_t* out, int64_t n, void* temp, cudaStream_t s) {
  scan_rec<uint32_t, uint64_t>(in, out, n, true, static_cast<char*>(temp), s);
}

size_t radix_sort_temp_bytes(int64_t capacity) {
  const int64_t nblocks = ceil_div(capacity > 0 ? capacity : 1, kTile);
  const int64_t hn = nblocks * kRadix;
  return 2 * (size_t)hn * sizeof(uint32_t) + scan_levels_bytes(hn, sizeof(uint32_t)) + 1024;
}

bool radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                      const uint64_t* n_dev, int64_t capacity, int bits, void* temp,
                      cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(ScatterSmem));
    attr_set = true;
  }
  const int64_t nblocks = ceil_div(capacity > 0 ? capacity : 1, kTile);
  const int64_t hn = nblocks * kRadix;
  uint32_t* hist = static_cast<uint32_t*>(temp);
  uint32_t* hscan = hist + hn;
  char* stemp = reinterpret_cast<char*>(hscan + hn);
  stemp = reinterpret_cast<char*>(((uintptr_t)stemp + 255) & ~(uintptr_t)255);
  bool alt = false;
  for (int shift = 0; shift < bits; shift += 8) {
    const uint64_t* kin = alt ? keys_alt : keys;
    const uint32_t* vin = alt ? vals_alt : vals;
    uint64_t* kout = alt ? keys : keys_alt;
    uint32_t* vout = alt ? vals : vals_alt;
    k_radix_hist<<<(unsigned)nblocks, kThreads, 0, s>>>(kin, n_dev, capacity, shift, hist, nblocks);
    count_launch();
    scan_rec<uint32_t, uint32_t>(hist, hscan, hn, false, stemp, s);
    k_radix_scatter<<<(unsigned)nblocks, kThreads, sizeof(ScatterSmem), s>>>(
        kin, vin, kout, vout, n_dev, capacity, shift, hscan, nblocks);
    count_launch();
    alt = !alt;
  }
  return alt;
}

}  // namespace splx
