// Device-wide exclusive scan of u32 counts (reduce-then-scan, recursive on block sums).
// Used to turn per-tile pair counts into per-tile segment starts.
#include "common.cuh"

namespace splx {

namespace {

constexpr int kThreads = 256;
constexpr int kIPT = 16;
constexpr int kTile = kThreads * kIPT;  // 4096
constexpr int kWarps = kThreads / 32;

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

// Exclusive scan of one value per thread across the block; also returns the total.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T& total, T* sw) {
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

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const uint32_t* __restrict__ in, int64_t n,
                                                          uint32_t* __restrict__ sums) {
  __shared__ uint32_t sw[kWarps];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    const int64_t i = base + j * kThreads + threadIdx.x;
    if (i < n) acc += in[i];
  }
  uint32_t total;
  block_exclusive_scan<uint32_t>(acc, total, sw);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// out[i] = offs[block] + exclusive prefix within the block; out[n] = grand total when
// write_total and the block holds the end of the input.
__global__ void __launch_bounds__(kThreads) k_scan_down(const uint32_t* __restrict__ in,
                                                        uint32_t* __restrict__ out, int64_t n,
                                                        const uint32_t* __restrict__ offs,
                                                        bool write_total) {
  __shared__ uint32_t tile[kTile];
  __shared__ uint32_t sw[kWarps];
  const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    const int64_t i = base + j * kThreads + threadIdx.x;
    tile[j * kThreads + threadIdx.x] = i < n ? in[i] : 0u;
  }
  __syncthreads();
  uint32_t v[kIPT];
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    v[j] = tile[threadIdx.x * kIPT + j];
    acc += v[j];
  }
  uint32_t total;
  const uint32_t off = offs ? offs[blockIdx.x] : 0u;
  uint32_t run = block_exclusive_scan<uint32_t>(acc, total, sw) + off;
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
  if (write_total && threadIdx.x == kThreads - 1 && base + kTile >= n) out[n] = off + total;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

void scan_rec(const uint32_t* in, uint32_t* out, int64_t n, bool write_total, char* temp,
              cudaStream_t s) {
  const int64_t blocks = ceil_div(n, kTile);
  if (blocks <= 1) {
    k_scan_down<<<1, kThreads, 0, s>>>(in, out, n, nullptr, write_total);
    count_launch();
    return;
  }
  uint32_t* sums = reinterpret_cast<uint32_t*>(temp);
  uint32_t* offs = sums + blocks;
  char* rest = temp + (((size_t)2 * blocks * sizeof(uint32_t) + 255) & ~(size_t)255);
  k_scan_reduce<<<(unsigned)blocks, kThreads, 0, s>>>(in, n, sums);
  count_launch();
  scan_rec(sums, offs, blocks, false, rest, s);
  k_scan_down<<<(unsigned)blocks, kThreads, 0, s>>>(in, out, n, offs, write_total);
  count_launch();
}

}  // namespace

size_t scan_u32_temp_bytes(int64_t n) {
  size_t bytes = 0;
  int64_t m = ceil_div(n, kTile);
  while (m > 1) {
    bytes += (((size_t)2 * m * sizeof(uint32_t) + 255) & ~(size_t)255);
    m = ceil_div(m, kTile);
  }
  return bytes + 512;
}

void scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* temp, cudaStream_t s) {
  scan_rec(in, out, n, true, static_cast<char*>(temp), s);
}

}  // namespace splx

namespace splx {

// Number of nonzero entries of a[0, n) added into *out (a grid-stride count, one atomic
// per warp).
__global__ void __launch_bounds__(256) k_count_nonzero(const uint32_t* __restrict__ a, int64_t n,
                                                       unsigned long long* out) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c += a[i] != 0u ? 1ull : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

void count_nonzero_u32(const uint32_t* a, int64_t n, unsigned long long* out, cudaStream_t s) {
  if (n <= 0) return;
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * 8;
  if (blocks > cap) blocks = cap;
  k_count_nonzero<<<(unsigned)blocks, 256, 0, s>>>(a, n, out);
  count_launch();
}

}  // namespace splx
