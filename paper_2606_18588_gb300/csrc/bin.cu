// Binning and per-tile depth sort (Sec. 2 step 2 "Sorting"), bucketed by tile.
//
// The projection kernel counts the (Gaussian, tile) pairs of every image tile; an
// exclusive scan of those counts gives each tile's segment.  fill writes one key per pair
// into its tile's segment, key = FP32 depth bits << 32 | Gaussian index, taking slots by
// counting the tile's counter back down (lanes of a warp that hit the same tile take a
// block of slots with one atomic; the counters end at zero).  Keys are unique within a
// tile, so sorting each segment by the full 64-bit key yields the (depth, index) order
// exactly, whatever order fill placed them in.  With cross-boundary filtering on, a pair
// the filter removes keeps its slot with depth bits 0xFFFFFFFF, so it sorts last, and the
// tile's range ends before it.
//
// Sorting: a segment of up to 2048 keys is sorted in shared memory by one CTA of 256
// threads (8 keys per thread by a transposition network, then merge-path merges of runs).
// Longer segments are cut into 4096-key chunks, each sorted the same way by a CTA of 512
// threads, and then merged pairwise in rounds (run width 4096, 8192, ...) with merge-path
// partitioning, one CTA per 4096 outputs, ping-ponging between the key buffer and its
// twin; segments that end in the twin are copied back.  Every pair is read and written a
// few times instead of once per 8-bit pass over 50+ key bits.
#include "common.cuh"
#include "spec.cuh"
#include "walk.cuh"

namespace splx {

namespace {

constexpr int kChunk = 2048;     // a segment up to this long is sorted by one CTA
constexpr int kSortThreads = 256;
constexpr int kBig = 4096;       // chunk of a longer segment (sorted, then merged)
constexpr int kBigThreads = 512;

__device__ __forceinline__ int next_pow2(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

constexpr int kItems = kChunk / kSortThreads;  // 8 keys per thread
static_assert(kBig / kBigThreads == kItems, "both sorts hold 8 keys per thread");

__device__ __forceinline__ void cas(uint64_t& a, uint64_t& b) {
  const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
  a = lo;
  b = hi;
}

// Shared buffers hold one spare slot per 8 keys, so that the 8-key runs a warp touches
// with stride 8 fall into different banks.
__device__ __forceinline__ int pad(int i) { return i + (i >> 3); }
constexpr int kPadded = kChunk + kChunk / 8;
constexpr int kBigPadded = kBig + kBig / 8;

// Number of elements taken from A = s[pad(a0 + i)] among the first d of merge(A, B) with
// B = s[pad(b0 + j)], in shared memory.
__device__ __forceinline__ int merge_path_smem(const uint64_t* s, int a0, int na, int b0, int nb,
                                               int d) {
  int lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s[pad(a0 + mid)] < s[pad(b0 + d - 1 - mid)]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Sorts in[0, n) into out[0, n) (n <= CH; out may be in) with TH threads: each thread sorts kItems keys in
// registers (odd-even transposition network), then runs of 8, 16, ... are merged pairwise
// through two shared buffers, every thread producing kItems outputs located by merge path.
// The array is padded to a power of two P >= 8 with ~0 keys.  sa, sb: CH + CH/8 keys each.
template <int TH>
__device__ __forceinline__ void sort_chunk(const uint64_t* in, uint64_t* out, int n, uint64_t* sa,
                                           uint64_t* sb) {
  int P = next_pow2(n);
  if (P < kItems) P = kItems;
  for (int i = threadIdx.x; i < P; i += TH) sa[pad(i)] = i < n ? in[i] : ~0ull;
  __syncthreads();
  const int active = P / kItems;  // threads holding keys
  const int t = threadIdx.x;
  if (t < active) {
    uint64_t v[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) v[r] = sa[pad(t * kItems + r)];
#pragma unroll
    for (int pass = 0; pass < kItems; ++pass)
#pragma unroll
      for (int r = pass & 1; r + 1 < kItems; r += 2) cas(v[r], v[r + 1]);
#pragma unroll
    for (int r = 0; r < kItems; ++r) sa[pad(t * kItems + r)] = v[r];
  }
  __syncthreads();
  uint64_t* src = sa;
  uint64_t* dst = sb;
  for (int w = kItems; w < P; w <<= 1) {
    if (t < active) {
      const int o = t * kItems;
      const int p0 = (o / (2 * w)) * (2 * w);
      const int d = o - p0;
      int ia = merge_path_smem(src, p0, w, p0 + w, w, d);
      int ib = d - ia;
      // heads of both runs in registers (~0 past a run's end; a key is below ~0 (its index
      // is below 2^32 - 1), and the ~0 padding keys are equal, so their order does not
      // matter); each output reloads only the head it consumed
      uint64_t va = ia < w ? src[pad(p0 + ia)] : ~0ull;
      uint64_t vb = ib < w ? src[pad(p0 + w + ib)] : ~0ull;
#pragma unroll
      for (int r = 0; r < kItems; ++r) {
        const bool takeA = va < vb;
        dst[pad(o + r)] = takeA ? va : vb;
        if (r + 1 < kItems) {
          ia += takeA ? 1 : 0;
          ib += takeA ? 0 : 1;
          const bool more = takeA ? ia < w : ib < w;
          const uint64_t nv = more ? src[takeA ? pad(p0 + ia) : pad(p0 + w + ib)] : ~0ull;
          va = takeA ? nv : va;
          vb = takeA ? vb : nv;
        }
      }
    }
    __syncthreads();
    uint64_t* tmp = src;
    src = dst;
    dst = tmp;
  }
  for (int i = threadIdx.x; i < n; i += TH) out[i] = src[pad(i)];
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

// Merge rounds a segment of n keys needs: ceil(log2(number of chunks)).
__device__ __forceinline__ int rounds_for(uint32_t n) {
  const uint32_t nch = (n + kBig - 1) / kBig;
  int r = 0;
  while ((1u << r) < nch) ++r;
  return r;
}

// Number of elements taken from A among the first d of merge(A, B) (unique keys), found
// by one warp with 32 probes per step (a 33-ary search over global memory).
__device__ __forceinline__ uint32_t merge_path_warp(const uint64_t* A, uint32_t na,
                                                    const uint64_t* B, uint32_t nb, uint32_t d) {
  const unsigned lane = threadIdx.x & 31u;
  uint32_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    const uint32_t span = hi - lo;
    const uint32_t m = lo + (uint32_t)(((uint64_t)span * (lane + 1)) / 33u);
    const bool pred = A[m] < B[d - 1 - m];  // true exactly for m below the answer
    const unsigned bal = __ballot_sync(0xffffffffu, pred);
    const int nt = __popc(bal);
    const uint32_t m_last_true = __shfl_sync(0xffffffffu, m, nt > 0 ? nt - 1 : 0);
    const uint32_t m_first_false = __shfl_sync(0xffffffffu, m, nt < 32 ? nt : 31);
    if (nt > 0) lo = m_last_true + 1;
    if (nt < 32) hi = m_first_false;
  }
  return lo;
}

// ---- selected-prefix sort (BatchDev::sel) ----
constexpr int kHistBins = 4096;
constexpr int kHistPer = kHistBins / kSortThreads;  // bins per thread in the boundary scan

// With base + (all keys counted in hist) > cap: the bin j whose keys take the running
// count base + (keys in bins below j) from at most cap to above it.  Writes j to s_tmp[8]
// and base + (keys below j) to s_tmp[9]; s_tmp[0..7] hold the warps' totals.  Whole-CTA
// call; the results are valid after it returns.
__device__ __forceinline__ void hist_boundary(const unsigned* hist, unsigned base, unsigned cap,
                                              unsigned* s_tmp) {
  const int t = (int)threadIdx.x, lane = t & 31, w = t >> 5;
  if (t == 0) { s_tmp[8] = 0u; s_tmp[9] = base; }  // (always overwritten below)
  unsigned v[kHistPer];
  unsigned sum = 0;
#pragma unroll
  for (int r = 0; r < kHistPer; ++r) {
    v[r] = hist[t * kHistPer + r];
    sum += v[r];
  }
  unsigned inc = sum;  // inclusive prefix over the warp's threads
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_tmp[w] = inc;
  __syncthreads();
  unsigned before = base + inc - sum;
  for (int i = 0; i < w; ++i) before += s_tmp[i];
#pragma unroll
  for (int r = 0; r < kHistPer; ++r) {
    if (before <= cap && cap < before + v[r]) {  // true for exactly one bin
      s_tmp[8] = (unsigned)(t * kHistPer + r);
      s_tmp[9] = before;
    }
    before += v[r];
  }
  __syncthreads();
}

// Sorts the S <= kSelCap smallest keys of the segment [s, e) (n > kChunk keys) into
// keys_alt[s, s + S) and records S in sel[t] and ranges[t] = [capacity + s, capacity + s
// + S), which indexes keys_alt through keys (keys_alt = keys + capacity with sel on);
// keys[s, e) stays as the fill left it.  S is the number of keys below a threshold found
// from a histogram of key bits 62..51 (the depth's exponent and 4 mantissa bits; bit 63,
// its sign, is 0), refined by one of bits 50..39 inside the bin the threshold falls in:
// the keys below the threshold are exactly the S smallest.  If even the nearest bin holds
// more than kSelCap keys, sel[t] = kSelNone and the forward hands the item straight to
// the full sort.
__device__ __forceinline__ void select_prefix(const BatchDev& b, int64_t t, uint32_t s,
                                              uint32_t e, uint64_t* sa, uint64_t* sb,
                                              unsigned* s_tmp) {
  const uint64_t* in = b.keys + s;
  const int n = (int)(e - s);
  unsigned* hist = reinterpret_cast<unsigned*>(sa);  // 16 KB of sa's 18 KB
  for (int i = threadIdx.x; i < kHistBins; i += kSortThreads) hist[i] = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kSortThreads)
    atomicAdd(&hist[(unsigned)(in[i] >> 51) & (kHistBins - 1)], 1u);
  __syncthreads();
  hist_boundary(hist, 0u, (unsigned)kSelCap, s_tmp);
  const unsigned b1 = s_tmp[8];
  unsigned S = s_tmp[9];
  uint64_t thr = (uint64_t)b1 << 51;
  if (8u * ((unsigned)kSelCap - S) > (unsigned)kSelCap) {
    // more than an eighth of the prefix left: refine inside bin b1
    for (int i = threadIdx.x; i < kHistBins; i += kSortThreads) hist[i] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kSortThreads) {
      const uint64_t k = in[i];
      if ((unsigned)(k >> 51) == b1) atomicAdd(&hist[(unsigned)(k >> 39) & (kHistBins - 1)], 1u);
    }
    __syncthreads();
    hist_boundary(hist, S, (unsigned)kSelCap, s_tmp);
    thr |= (uint64_t)s_tmp[8] << 39;
    S = s_tmp[9];
  }
  if (S == 0) {
    if (threadIdx.x == 0) b.sel[t] = kSelNone;
    return;
  }
  if (threadIdx.x == 0) s_tmp[10] = 0u;
  __syncthreads();
  // the keys below thr, in any order, then sorted (sort_chunk reads them before it
  // writes sb)
  for (int i = threadIdx.x; i < n; i += kSortThreads) {
    const uint64_t k = in[i];
    if (k < thr) {
      const unsigned pos = atomicAdd(&s_tmp[10], 1u);
      if (pos < S) sb[pos] = k;
    }
  }
  __syncthreads();
  if (s_tmp[10] != S) {  // not reachable for keys of positive depths; kept as a check
    if (threadIdx.x == 0) { atomicOr(b.status, ST_BOUNDS); b.sel[t] = kSelNone; }
    return;
  }
  sort_chunk<kSortThreads>(sb, b.keys_alt + s, (int)S, sa, sb);
  if (threadIdx.x == 0) {
    b.sel[t] = S;
    const uint32_t off = (uint32_t)b.capacity + s;
    b.ranges[t] = make_uint2(off, off + S);
  }
}

}  // namespace

// ---------------------------------------------------------------- fill
constexpr int kFillThreads = 256;
constexpr int kFillFields = 18;  // per lane: tile test (8), rect x, rect y, tile base, width,
                                 // 1/width, tiles per row, pass bits, key (2), tiles

__global__ void __launch_bounds__(kFillThreads, 8) k_fill(const BatchDev b) {
  __shared__ float s_walk[kFillThreads / 32][kFillFields][32];
  __shared__ int s_own[kFillThreads / 32][32];
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lanes = __ballot_sync(0xffffffffu, idx < (int64_t)b.V * b.N);
  if (idx >= (int64_t)b.V * b.N) return;
  const uint32_t tiles = b.counts[idx];
  const int v = (int)(idx / b.N);
  const int64_t g = idx - (int64_t)v * b.N;
  int tw = 1, tiles_x = 0, rx0 = 0, rx1 = 0, ry0 = 0, ry1 = 0;
  int64_t tbase = 0;
  uint64_t key = 0;
  TileCull tc = tile_cull_prep(0.f, 0.f, 1.f, 0.f, 1.f, -1.0f);
  uint32_t hits = 0;
  if (tiles) {
    const int k = subset_of(b, g);
    const ViewDev& cam = b.views[v];
    const Rec* r = b.rec + idx;
    const float4 rb = r->b;
    const uint32_t rx = __float_as_uint(rb.w), ry = __float_as_uint(r->c.w);
    const int B_ = b.tile;
    rx0 = (int)(rx & 0xFFFFu); rx1 = (int)(rx >> 16);
    ry0 = (int)(ry & 0xFFFFu); ry1 = (int)(ry >> 16);
    const int tx0 = rx0 / B_, ty0 = ry0 / B_;
    tw = rx1 / B_ - tx0 + 1;
    const float4 rd = r->d;  // the tile test's pass bits, or its inputs (> 32 tiles)
    if (tiles <= 32u) {
      hits = __float_as_uint(rd.w);
    } else {
      // the test centres on the specification's 2-D mean (the record holds the blend's)
      const SubsetDev S = b.subsets[k];
      const int64_t i = g - S.goff;
      const float m[3] = {__ldg(S.means + 3 * i), __ldg(S.means + 3 * i + 1),
                          __ldg(S.means + 3 * i + 2)};
      float tcam[3], terr[3], su, sv;
      spec_camera(m, cam.R, cam.t, tcam, terr);
      spec_center(tcam[0], tcam[1], tcam[2], cam.fx, cam.fy, cam.cx, cam.cy, su, sv);
      tc = tile_cull_prep(su, sv, rd.x, rd.y, rd.z, rd.w);
    }
    tiles_x = cam.tiles_x;
    tbase = b.tile_base[v] + (int64_t)k * cam.tiles_x * cam.tiles_y + (int64_t)ty0 * cam.tiles_x + tx0;
    key = ((uint64_t)__float_as_uint(rb.z) << 32) | (uint64_t)(uint32_t)g;
  }
  const int warp = (int)(threadIdx.x >> 5);
  const unsigned lane = threadIdx.x & 31u, lt = (1u << lane) - 1u;
  bool overflow = false;
  // one (tile, key) candidate per lane: aggregate per tile, take slots, write the keys
  auto place = [&](unsigned t, uint64_t k) {
    if (b.cross && t != 0xFFFFFFFFu) {
      // cross-boundary filtering: a removed pair keeps its slot with the largest depth
      const unsigned long long c = b.cross[(uint32_t)k];
      if (c) {
        const int v = view_of(b.tile_base, b.V, (int64_t)t);
        const ViewDev& cam = b.views[v];
        const int64_t nt = (int64_t)cam.tiles_x * cam.tiles_y;
        const int64_t rem = (int64_t)t - b.tile_base[v];
        const int km = (int)(rem / nt);
        const int loc = (int)(rem - (int64_t)km * nt);
        if (cross_removed(b, v, km, c, loc % cam.tiles_x, loc / cam.tiles_x,
                          (uint32_t)(k >> 32))) {
          k = (0xFFFFFFFFull << 32) | (k & 0xFFFFFFFFull);
          atomicAdd(&b.removed[t], 1u);
        }
      }
    }
    const unsigned peers = __match_any_sync(lanes, t);
    const int leader = __ffs(peers) - 1;
    unsigned old = 0;
    if (t != 0xFFFFFFFFu && (int)lane == leader) old = atomicSub(&b.tile_cnt[t], (unsigned)__popc(peers));
    old = __shfl_sync(lanes, old, leader);
    if (t != 0xFFFFFFFFu) {
      const uint64_t pos = (uint64_t)b.tile_start[t] + (old - 1u - (unsigned)__popc(peers & lt));
      if (pos < (uint64_t)b.capacity) b.keys[pos] = k;
      else overflow = true;
    }
  };
  // the warp's (Gaussian, tile) candidates spread evenly over its lanes (see walk.cuh;
  // here the whole list: a head walked in lockstep measured slower for this kernel)
  {
    float(*f)[32] = s_walk[warp];
    f[0][lane] = tc.u; f[1][lane] = tc.v; f[2][lane] = tc.A; f[3][lane] = tc.B;
    f[4][lane] = tc.C; f[5][lane] = tc.qmax; f[6][lane] = tc.rBC; f[7][lane] = tc.rBA;
    f[8][lane] = __uint_as_float((uint32_t)rx0 | ((uint32_t)rx1 << 16));
    f[9][lane] = __uint_as_float((uint32_t)ry0 | ((uint32_t)ry1 << 16));
    f[10][lane] = __uint_as_float((uint32_t)tbase);
    f[11][lane] = __int_as_float(tw);
    f[12][lane] = 1.0f / (float)tw;
    f[13][lane] = __int_as_float(tiles_x);
    f[14][lane] = __uint_as_float(hits);
    f[15][lane] = __uint_as_float((uint32_t)key);
    f[16][lane] = __uint_as_float((uint32_t)(key >> 32));
    f[17][lane] = __uint_as_float(tiles);
    // a rectangle of at most 32 tiles walks only the tiles its pass bits name (the test is
    // already taken); a larger one walks them all and takes the test
    const int cand = tiles <= 32u ? __popc(hits) : (int)tiles;
    const WarpWalk walk = warp_walk_begin(lanes, cand);
    for (int base = 0; base < walk.total; base += walk.nact) {
      int j;
      const int o = warp_walk_owner(walk, base, s_own[warp], j);
      unsigned t = 0xFFFFFFFFu;
      uint64_t okey = 0;
      if (o >= 0) {
        int jx, jy;
        bool pass;
        if (__float_as_uint(f[17][o]) <= 32u) {
          // the j-th set pass bit
          unsigned m = __float_as_uint(f[14][o]);
          for (int q = 0; q < j; ++q) m &= m - 1u;
          walk_tile(__ffs(m) - 1, __float_as_int(f[11][o]), f[12][o], jx, jy);
          pass = true;
        } else {
          walk_tile(j, __float_as_int(f[11][o]), f[12][o], jx, jy);
          TileCull oc;
          oc.u = f[0][o]; oc.v = f[1][o]; oc.A = f[2][o]; oc.B = f[3][o];
          oc.C = f[4][o]; oc.qmax = f[5][o]; oc.rBC = f[6][o]; oc.rBA = f[7][o];
          const uint32_t rx = __float_as_uint(f[8][o]), ry = __float_as_uint(f[9][o]);
          const int x0 = (int)(rx & 0xFFFFu), x1 = (int)(rx >> 16);
          const int y0 = (int)(ry & 0xFFFFu), y1 = (int)(ry >> 16);
          pass = tile_hits_spec(oc, x0, x1, y0, y1, x0 / b.tile + jx, y0 / b.tile + jy, b.tile);
        }
        if (pass) {
          t = __float_as_uint(f[10][o]) + (unsigned)(jy * __float_as_int(f[13][o]) + jx);
          okey = ((uint64_t)__float_as_uint(f[16][o]) << 32) | __float_as_uint(f[15][o]);
        }
      }
      place(t, okey);
    }
  }
  if (overflow) atomicOr(b.status, ST_CAPACITY);
}

void launch_fill(const BatchDev& b, cudaStream_t s) {
  const int64_t n = (int64_t)b.V * b.N;
  const int64_t blocks = (n + kFillThreads - 1) / kFillThreads;
  if (blocks == 0) return;
  k_fill<<<(unsigned)blocks, kFillThreads, 0, s>>>(b);
  count_launch();
}

// ---------------------------------------------------------------- segment sorts
// One CTA per tile: ranges, then either the whole segment (<= kChunk keys) or, for a
// longer one, its registration as chunk work items (segment list index, chunk index).
__global__ void __launch_bounds__(kSortThreads) k_seg_sort_small(const BatchDev b) {
  __shared__ uint64_t sk[2][kPadded];
  __shared__ unsigned s_base[2];
  __shared__ unsigned s_tmp[11];
  const int64_t t = item_of(b, blockIdx.x);
  uint32_t s, e;
  segment_of(b, t, s, e);
  // the pairs the cross-boundary filter removed sort last and stay out of the range
  if (threadIdx.x == 0) {
    const uint32_t cut = b.removed ? min(b.removed[t], e - s) : 0u;
    b.ranges[t] = make_uint2(s, e - cut);
    if (b.sel) b.sel[t] = 0u;
  }
  const int n = (int)(e - s);
  if (n <= 1) return;
  // saturation-skipping waves sort only what the wave's rasteriser will walk
  if (b.order && b.wave > 0 && item_saturated(b, t)) return;
  // likewise with a stale saturation state: a tile pruned at every pixel stays unsorted
  if (b.sat && item_pruned(b, t)) return;
  if (n > kChunk && b.sel) {
    select_prefix(b, t, s, e, sk[0], sk[1], s_tmp);
    return;
  }
  if (n > kChunk) {
    const unsigned nch = (unsigned)((n + kBig - 1) / kBig);
    if (threadIdx.x == 0) {
      s_base[0] = atomicAdd(b.big_count, 1u);
      s_base[1] = atomicAdd(b.chunk_count, nch);
      atomicMax(b.big_count + 1, nch);
    }
    __syncthreads();
    const unsigned i = s_base[0];
    if (threadIdx.x == 0) b.big_list[i] = (uint32_t)t;
    for (unsigned c = threadIdx.x; c < nch; c += kSortThreads) b.chunks[s_base[1] + c] = make_uint2(i, c);
    return;
  }
  sort_chunk<kSortThreads>(b.keys + s, b.keys + s, n, sk[0], sk[1]);
}

// Sorts every 4096-key chunk of the long segments (grid-stride over the chunk list); two
// shared buffers of kBigPadded keys in dynamic shared memory.
__global__ void __launch_bounds__(kBigThreads) k_chunk_sort(const BatchDev b) {
  extern __shared__ uint64_t sk_dyn[];
  uint64_t* sa = sk_dyn;
  uint64_t* sb = sk_dyn + kBigPadded;
  const unsigned count = *b.chunk_count;
  for (unsigned w = blockIdx.x; w < count; w += gridDim.x) {
    const uint2 ch = b.chunks[w];
    const int64_t t = b.big_list[ch.x];
    uint32_t s, e;
    segment_of(b, t, s, e);
    const uint32_t c0 = s + ch.y * kBig;
    if (c0 >= e) continue;
    const uint32_t c1 = c0 + kBig < e ? c0 + kBig : e;
    // a segment merged in R rounds starts them in keys_alt when R is odd, so that its
    // last round writes keys
    uint64_t* out = ((rounds_for(e - s) & 1) ? b.keys_alt : b.keys) + c0;
    sort_chunk<kBigThreads>(b.keys + c0, out, (int)(c1 - c0), sa, sb);
    __syncthreads();
  }
}

// Merge round r (run width 4096 << r): each chunk work item produces 4096 outputs of the
// merge of the two runs its output range falls in.  A segment merged in R rounds holds the
// input of round r in keys_alt when R - r is odd and in keys otherwise, so its last round
// writes keys.
__global__ void __launch_bounds__(kBigThreads) k_merge_round(const BatchDev b, int r) {
  __shared__ uint64_t sm[kBigPadded];
  __shared__ uint32_t s_split[4];
  constexpr int PER = kBig / kBigThreads;  // outputs per thread
  // a round is needed only while some segment holds more than 2^r chunks (the launches
  // cover the bound for the largest subset; most rounds of a wave find nothing to do)
  if ((1u << r) >= b.big_count[1]) return;
  const unsigned count = *b.chunk_count;
  const uint32_t w = (uint32_t)kBig << r;
  for (unsigned wi = blockIdx.x; wi < count; wi += gridDim.x) {
    const uint2 ch = b.chunks[wi];
    const int64_t t = b.big_list[ch.x];
    uint32_t s, e;
    segment_of(b, t, s, e);
    const uint32_t n = e - s;
    if (n <= w) continue;  // this segment needs no merge at this width
    // round r of a segment merged in R rounds reads keys_alt when R - r is odd (see the
    // chunk sort), so its last round writes keys
    const bool from_alt = ((rounds_for(n) - r) & 1) != 0;
    const uint64_t* src = (from_alt ? b.keys_alt : b.keys) + s;
    uint64_t* dst = (from_alt ? b.keys : b.keys_alt) + s;
    const uint32_t o0 = ch.y * kBig;
    if (o0 >= n) continue;
    const uint32_t o1 = o0 + kBig < n ? o0 + kBig : n;
    const uint32_t p0 = (o0 / (2 * w)) * (2 * w);
    const uint32_t na = (p0 + w < n ? p0 + w : n) - p0;
    const uint32_t nb = (p0 + 2 * w < n ? p0 + 2 * w : n) - (p0 + na);
    const uint64_t* A = src + p0;
    const uint64_t* B = A + na;
    // warp 0 finds the split at the block's first output, warp 1 at its end
    if (threadIdx.x < 64) {
      const uint32_t dd = (threadIdx.x < 32 ? o0 : o1) - p0;
      const uint32_t a = merge_path_warp(A, na, B, nb, dd);
      if ((threadIdx.x & 31) == 0) {
        s_split[threadIdx.x >> 5] = a;
        s_split[2 + (threadIdx.x >> 5)] = dd - a;
      }
    }
    __syncthreads();
    const uint32_t a0 = s_split[0], a1 = s_split[1], b0 = s_split[2], b1 = s_split[3];
    const int la = (int)(a1 - a0), lb = (int)(b1 - b0);
    for (int i = threadIdx.x; i < la; i += kBigThreads) sm[pad(i)] = A[a0 + i];
    for (int i = threadIdx.x; i < lb; i += kBigThreads) sm[pad(la + i)] = B[b0 + i];
    __syncthreads();
    // each thread merges PER consecutive outputs of sm[0,la) and sm[la,la+lb)
    const int d = threadIdx.x * PER;
    if (d < la + lb) {
      int ia = merge_path_smem(sm, 0, la, la, lb, d);
      int ib = d - ia;
      const int dend = d + PER < la + lb ? d + PER : la + lb;
      uint64_t va = ia < la ? sm[pad(ia)] : ~0ull;  // run heads (~0 past the end)
      uint64_t vb = ib < lb ? sm[pad(la + ib)] : ~0ull;
      for (int o = d; o < dend; ++o) {
        const bool takeA = va < vb;
        dst[o0 + o] = takeA ? va : vb;
        ia += takeA ? 1 : 0;
        ib += takeA ? 0 : 1;
        const bool more = takeA ? ia < la : ib < lb;
        const uint64_t nv = more ? sm[takeA ? pad(ia) : pad(la + ib)] : ~0ull;
        va = takeA ? nv : va;
        vb = takeA ? vb : nv;
      }
    }
    __syncthreads();
  }
}

// The items the forward handed back (b.retry): full segment ranges, sel = 0, and their
// segments registered as chunk work items for the long-segment sort.
__global__ void __launch_bounds__(128) k_retry_prep(const BatchDev b) {
  const unsigned n = *b.retry_count;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = b.retry[i];
    uint32_t s, e;
    segment_of(b, t, s, e);
    b.ranges[t] = make_uint2(s, e);
    // after a prefix the second forward resumes at the prefix's end (the whole sort puts
    // the prefix's keys first, in its order); without one it starts at the beginning
    const uint32_t sv = b.sel[t];
    b.sel[t] = sv != kSelNone && sv != 0u ? (kSelResume | sv) : 0u;
    const unsigned nch = (e - s + kBig - 1) / kBig;
    const unsigned bi = atomicAdd(b.big_count, 1u);
    const unsigned c0 = atomicAdd(b.chunk_count, nch);
    atomicMax(b.big_count + 1, nch);
    b.big_list[bi] = t;
    for (unsigned c = 0; c < nch; ++c) b.chunks[c0 + c] = make_uint2(bi, c);
  }
}

// Chunk sort and merge rounds of the segments registered in big_list / chunks.
static void launch_long_sort(const BatchDev& b, int max_rounds, cudaStream_t s) {
  const unsigned grid = (unsigned)device_sm_count() * 4;
  // 72 KB of dynamic shared memory: opted in once per device (a refused opt-in shows as
  // the launch's error, which the callers check).  Its grid-stride loop runs one wave of
  // resident CTAs (3 per SM at 72 KB), so that no CTA starts after the others have ended
  constexpr int kChunkSmem = 2 * kBigPadded * (int)sizeof(uint64_t);
  (void)opt_in_smem((const void*)k_chunk_sort, kChunkSmem, 0);
  const unsigned cgrid = (unsigned)device_sm_count() *
                         (unsigned)resident_ctas((const void*)k_chunk_sort, kBigThreads,
                                                 kChunkSmem, 0);
  k_chunk_sort<<<cgrid, kBigThreads, kChunkSmem, s>>>(b);
  for (int r = 0; r < max_rounds; ++r) k_merge_round<<<grid, kBigThreads, 0, s>>>(b, r);
  count_launch(1 + max_rounds);
}

void launch_seg_sort(const BatchDev& b, int max_rounds, cudaStream_t s) {
  if (b.n_tiles == 0) return;
  const int64_t items = b.order ? b.item_n : b.n_tiles;
  k_seg_sort_small<<<(unsigned)items, kSortThreads, 0, s>>>(b);
  count_launch();
  // with selected prefixes no segment is left to the long-segment sort before the forward
  if (!b.sel) launch_long_sort(b, max_rounds, s);
}

void launch_sort_retries(const BatchDev& b, int max_rounds, cudaStream_t s) {
  if (!b.sel || b.n_tiles == 0) return;
  cudaMemsetAsync(b.big_count, 0, 2 * sizeof(unsigned), s);
  cudaMemsetAsync(b.chunk_count, 0, sizeof(unsigned), s);
  k_retry_prep<<<(unsigned)device_sm_count(), 128, 0, s>>>(b);
  count_launch();
  launch_long_sort(b, max_rounds, s);
}

// Merge rounds that cover any segment of a batch whose largest subset has max_n Gaussians
// (a tile's segment holds at most one key per Gaussian of its subset).
int merge_rounds_bound(int64_t max_n) {
  const int64_t nch = (max_n + kBig - 1) / kBig;
  int r = 0;
  while ((int64_t(1) << r) < nch) ++r;
  return r;
}

}  // namespace splx
