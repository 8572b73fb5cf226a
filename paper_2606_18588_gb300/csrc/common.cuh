// Internal definitions shared by the libsplx kernels and the C-ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "splx.h"

namespace splx {

constexpr int kMaxK = 64;        // subsets per view
constexpr int kCounters = 10;    // work counters of a batch (BatchDev::counters)
constexpr int kMaxViews = 256;   // views per batch

// Concatenated views of the D-SSIM loss: view v's [3][H][W] image at 3 * pix_off[v];
// blk_off[v] = first (channel, 32 x 32 tile) work item of view v.
struct LossImgs {
  int V;
  int W[kMaxViews], H[kMaxViews];
  int64_t pix_off[kMaxViews + 1];
  int64_t blk_off[kMaxViews + 1];
};
LossImgs make_loss_imgs(int V, const int* W, const int* H);
int ssim_init();
void launch_loss_l1_dssim(const LossImgs& L, const float* x, const float* y, float lam,
                          float* dmx, float* dexx, float* dexy, double* sums, float* loss,
                          float* dL, cudaStream_t s);

// True while `s` is being captured into a CUDA graph.
inline bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  return cs != cudaStreamCaptureStatusNone;
}
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// Device status bits (OR-ed by kernels, read and cleared by the host).
enum : int { ST_CAPACITY = 1, ST_TIMEOUT = 2, ST_BOUNDS = 4 };

// One subset as seen by the kernels: parameters, gradient targets, global index base.
struct SubsetDev {
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const float* sh;
  float* g_means;
  float* g_log_scales;
  float* g_quats;
  float* g_opacity_logits;
  float* g_sh;
  int64_t n;
  int64_t goff;  // first global index of this subset
};

// One view: camera, image geometry, where its tiles and pixels live, its I/O planes.
struct ViewDev {
  float R[9], t[3];
  float fx, fy, cx, cy, near_plane;
  float eye[3];  // camera centre in world space
  int32_t W, H, tiles_x, tiles_y;
};

// Planes of one (view, subset) partial image.
struct ImgDev {
  float* rgb;      // [3][H][W]
  float* T;        // [H][W]
  float* D;        // [H][W]
  int32_t* last;   // [H][W]
  float4* gCT;     // [H][W] composite adjoint (dL/dC^m rgb, dL/dT^m)
};

// Projected record of one (view, Gaussian): 64 bytes, gathered by the rasterisers.
//   a = (u, v, qa, qb)      the blend's 2-D mean (double-float, see blend_center), conic
//                            scaled by -log2(e)/2 ... see project.cu
//   b = (qc, opacity, depth, rect_x)   rect_x = x0 | x1 << 16 (bit pattern)
//   c = (r, g, b, rect_y)              rect_y = y0 | y1 << 16
//   d = (A, B, C, q_max | hits)   conic and tile-test threshold in the binning
//                            specification; w holds instead the pass bits of the
//                            rectangle's tiles when it spans at most 32 (read by fill)
struct Rec {
  float4 a, b, c, d;
};

// Everything a batch kernel needs, passed by value.
struct BatchDev {
  int32_t V, K, sh_degree, nc;  // nc = (deg+1)^2
  int64_t N;                    // Gaussians over all subsets
  int32_t tile;                 // tile side
  int32_t tile_bits;            // bits of the image-tile id in a sort key
  int64_t n_tiles;              // image tiles over all (view, subset)
  int64_t capacity;             // pair capacity
  float eps_T, eps_comp, alpha_min, alpha_max;
  float bg[3];
  const SubsetDev* subsets;     // [K]
  const ViewDev* views;         // [V]
  const ImgDev* imgs;           // [V*K], image (v,k) at v*K+k
  Rec* rec;                     // [V][N]
  uint32_t* counts;             // [V*N] tiles touched
  uint32_t* tile_cnt;           // [n_tiles] pairs per image tile (zero between runs)
  uint32_t* tile_start;         // [n_tiles+1] exclusive scan of tile_cnt (last = total)
  uint64_t* keys;               // [capacity] depth bits << 32 | Gaussian index, by tile
  uint64_t* keys_alt;           // [capacity] scratch for the long-segment sort
  uint32_t* big_list;           // [n_tiles] tiles whose segment exceeds one sort chunk
  unsigned* big_count;          // [2]: tiles in big_list, most chunks of one of them
  uint2* chunks;                // [n_tiles + capacity/2048 + 1] (big_list index, chunk)
  unsigned* chunk_count;        // [1]
  uint2* ranges;                // [n_tiles] sorted [start, end)
  int64_t goff[kMaxK + 1];      // subset k = global indices [goff[k], goff[k+1])
  int64_t tile_base[kMaxViews + 1];  // view v's image tiles start at tile_base[v]
  int64_t pix_off[kMaxViews + 1];    // view v's pixels start at pix_off[v]
  // [V][N][3]: (sx, sy, sxx, sxy), (syy, go, gr, gg), (gb, 0, 0, 0): sums over pixels of
  // ge dx, ge dy, ge dx^2, ge dx dy, ge dy^2 (ge = dL/dpower / o), dL/do, dL/dcolour
  float4* grad2d;
  int* status;                  // device status word
  // work counters (nullable; kept by eager runs): forward [0] thread-entries examined,
  // [1] (pixel, entry) alpha evaluations, [2] blends; backward [3] thread-entries,
  // [4] alpha evaluations, [5] contributions (alpha >= alpha_min); [6] work items left
  // empty by saturation skipping; [7] work items outside their subset's visible region;
  // [8] work items the forward walked on a selected prefix, [9] of those, the ones it
  // handed to the full sort (see sel)
  unsigned long long* counters;
  // selected-prefix sort (sel != nullptr; the batched path, with keys_alt = keys +
  // capacity and 2 capacity < 2^32): a tile segment longer than one sort chunk gets only
  // its sel[t] smallest keys sorted, into keys_alt at the segment's offset, and ranges[t]
  // names them as keys[capacity + start, capacity + start + sel[t]) (keys keeps the
  // segment unsorted).
  // The forward walks that prefix; if a pixel of the tile is still blending at its end,
  // it renders nothing and appends the item to retry (retry_count of them), whose segments
  // are then sorted whole into keys (sel[t] = 0) and rendered again.  sel[t] = 0: the
  // segment is sorted whole in keys; kSelNone: no prefix was selected (straight to retry);
  // kSelResume | S: sorted whole after a prefix of S keys, whose forward state the planes
  // hold
  uint32_t* sel;
  uint32_t* retry;
  unsigned* retry_count;
  // spatial visibility (nullable): per (view, subset) the bounding tile rectangle of the
  // subset's (Gaussian, tile) pairs as (min tx, min ty, ~max tx, ~max ty), built by the
  // projection with atomicMin (all four start at 0xFFFFFFFF, i.e. empty).  Work items
  // outside it have no pairs; their partial planes are neither written nor read.
  uint32_t* omega;
  // cross-boundary per-ray filtering (cross != nullptr; needs omega): cells [K][6] = the
  // subsets' k-d boxes (lo x, y, z, hi x, y, z); cross [N] = per Gaussian the mask of other
  // cells its support box mu +- 3 s_max meets; zr [V][K][2] = per (view, subset) the depth
  // range of its kept Gaussians as (min bits, ~max bits), built by the projection with
  // atomicMin (both start at 0xFFFFFFFF, i.e. empty)
  const float* cells;
  unsigned long long* cross;
  uint32_t* zr;
  // per image tile, the pairs the filter removed: the fill gives them the largest depth,
  // so they sort last, and the tile's range ends before them (zero between runs)
  uint32_t* removed;
  // the cells the filter compares against: ncells boxes in `cells`, their visible regions
  // omega_x [V][ncells][4] and depth ranges zr_x [V][ncells][2] (the batch's own omega and
  // zr, ncells = K); cell_self >= 0 names the one cell a per-view render's single subset
  // belongs to (-1: subset k is cell k)
  const uint32_t* omega_x;
  const uint32_t* zr_x;
  int ncells;
  int cell_self;
  // saturation skipping (order != nullptr): the forward rasteriser runs in K waves; wave r
  // renders subset order[v * K + r] of every view v, and tpre [total pixels] holds the
  // product of the transmittances of the subsets rendered so far
  const int32_t* order;
  int wave;
  // a wave launch covers wave items [item_lo, item_lo + item_n) of the n_tiles / K (views
  // in order), so that groups of views can run their waves side by side
  int64_t item_lo, item_n;
  float* tpre;
  // stale saturation state (sat != nullptr, one launch per stage instead of waves): view
  // v's state sat[v] [H_v][W_v] prunes the subsets of rank >= sat[v][p] in its
  // front-to-back order at pixel p (values >= K prune nothing); rank [V][K] is the rank of
  // subset k in view v's order
  uint8_t* const* sat;
  const int32_t* rank;
  // persistent rasterisers: grid size (0 = one CTA per work item) and the two work
  // counters they take items from ([0] forward, [1] backward; reset before each launch)
  int persist_grid;
  unsigned long long* work_ctr;
  // concatenated per-view I/O: view v's rgb at 3*pix_off[v], its T plane at pix_off[v]
  float* out_rgb;
  float* out_T;                 // nullable
  const float* dL_drgb;
  const float* dL_dT;           // nullable
};

// Gradient targets of the K subsets (means, log_scales, quats, opacity_logits, sh).
struct GradTable {
  float* p[kMaxK][5];
};

// Adam state of the K subsets (parameters, first and second moments; arrays in the
// GradTable order) and its hyperparameters: lr[0..4] per array, lr[5] the SH coefficients
// above degree 0; the step number is *step_dev if non-NULL, else step.
struct AdamTable {
  float* p[kMaxK][5];
  float* m[kMaxK][5];
  float* v[kMaxK][5];
  float lr[6];
  float b1, b2, eps;
  int64_t step;
  const int64_t* step_dev;
  // optional, [ceil(N / 128)]: the fused projection adjoint leaves to a second, streaming
  // pass the 128-Gaussian blocks in which no Gaussian has a gradient (flag 1)
  uint8_t* defer;
};

__host__ __device__ inline int n_sh(int deg) { return (deg + 1) * (deg + 1); }

// BatchDev::sel value of a long segment with no selected prefix (its nearest depth bin
// alone holds more keys than a prefix may)
constexpr uint32_t kSelNone = 0xFFFFFFFFu;
// BatchDev::sel bit of a handed-back item whose segment is now sorted whole and whose
// second forward resumes after its first (sel & ~kSelResume) entries
constexpr uint32_t kSelResume = 0x80000000u;
// largest selected prefix: keys sorted in shared memory by one sort CTA
constexpr int kSelCap = 2048;

// ---- launch wrappers (defined in the .cu files) ------------------------------------
void launch_project(const BatchDev& b, cudaStream_t s);
void launch_fill(const BatchDev& b, cudaStream_t s);
// Sorts every tile segment; max_rounds = merge_rounds_bound(largest subset size).
void launch_seg_sort(const BatchDev& b, int max_rounds, cudaStream_t s);
int merge_rounds_bound(int64_t max_n);
inline int64_t chunk_list_capacity(int64_t n_tiles, int64_t capacity) {
  return n_tiles + capacity / 2048 + 1;
}
void launch_raster_fwd(const BatchDev& b, cudaStream_t s);
// The full sort of the segments the forward handed back (b.retry) and their second
// forward: no-ops when the retry list is empty (selected-prefix sort, b.sel != nullptr).
void launch_sort_retries(const BatchDev& b, int max_rounds, cudaStream_t s);
void launch_raster_fwd_retry(const BatchDev& b, cudaStream_t s);
void launch_composite(const BatchDev& b, int64_t total_pixels, cudaStream_t s);
void launch_composite_bwd(const BatchDev& b, int64_t total_pixels, cudaStream_t s);
// Re-evaluates every view's stale saturation state (b.sat) from the partials just rendered:
// order [V][K] is each view's front-to-back subset order.
void launch_sat_update(const BatchDev& b, const int32_t* order, int64_t total_pixels,
                       cudaStream_t s);
void launch_raster_bwd(const BatchDev& b, cudaStream_t s);
// Largest number of persistent rasteriser CTAs that fit on one SM (0 on error).
int raster_max_ctas_per_sm(int tile, bool bwd);
void launch_project_bwd(const BatchDev& b, const GradTable& gt, cudaStream_t s);
// The projection adjoint with Adam fused in: every Gaussian of the batch is updated from its
// gradient of this backward (zero where it has none) without materialising the gradient.
// Increments *at.step_dev first when it is set.
void launch_project_bwd_adam(const BatchDev& b, const AdamTable& at, cudaStream_t s);

// exclusive scan of n u32 values (out has n+1 entries; out[n] = total)
size_t scan_u32_temp_bytes(int64_t n);
void scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* temp, cudaStream_t s);
// *out += number of nonzero entries of a[0, n)
void count_nonzero_u32(const uint32_t* a, int64_t n, unsigned long long* out, cudaStream_t s);

// Adam over one parameter array.  The step number is `step` or, if step_dev is non-NULL,
// *step_dev read on the device.
void launch_adam(float* p, float* g, float* m, float* v, int64_t n, int64_t sh_stride,
                 float lr, float lr_rest, float b1, float b2, float eps, int64_t step,
                 const int64_t* step_dev, bool zero_grad, bool vec4, cudaStream_t s);
void launch_step_increment(int64_t* step_dev, cudaStream_t s);
void launch_loss_l1(const float* img, const float* target, int64_t n, float* loss,
                    float* dL, cudaStream_t s);

// Number of SMs of the current device (looked up once per device), for grids sized to the
// chip; 152 if the query fails.
int device_sm_count();
// Opts kernel `fn` into `bytes` of dynamic shared memory on the current device, once per
// device (function attributes belong to a device's context); returns the opt-in's result.
cudaError_t opt_in_smem(const void* fn, int bytes, int slot);
// CTAs of kernel fn (threads per CTA, dynamic shared memory bytes) resident on one SM of the
// current device, looked up once per device and slot (at least 1).
int resident_ctas(const void* fn, int threads, int smem, int slot);

// Counts kernel launches issued by the library (for reporting).
extern thread_local int64_t* g_launch_counter;
inline void count_launch(int n = 1) {
  if (g_launch_counter) *g_launch_counter += n;
}

}  // namespace splx

namespace splx {
// Subset of global Gaussian index g (binary search over the by-value offsets).
__device__ __forceinline__ int subset_of(const BatchDev& b, int64_t g) {
  int lo = 0, hi = b.K - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b.goff[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}
// View of global image-tile id / global pixel index.
__device__ __forceinline__ int view_of(const int64_t* base, int V, int64_t x) {
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Work item of a launch: every (view, subset, tile), or in a saturation-skipping wave the
// tiles of subset order[v][wave] of every view v (n_tiles / K items).
__device__ __forceinline__ int64_t item_of(const BatchDev& b, int64_t w) {
  if (!b.order) return w;
  w += b.item_lo;
  const int v = view_of(b.tile_base, b.V, w * b.K);
  const int64_t nt = (b.tile_base[v + 1] - b.tile_base[v]) / b.K;
  const int k = b.order[v * b.K + b.wave];
  return b.tile_base[v] + (int64_t)k * nt + (w - b.tile_base[v] / b.K);
}

__device__ __forceinline__ int64_t items_of_launch(const BatchDev& b) {
  return b.order ? b.item_n : b.n_tiles;
}

// Saturation skipping test of work item `id` in a wave after the first: true if every pixel
// of its tile has prefix transmittance below eps_comp.  Whole-CTA call (uses
// __syncthreads_or); the rasteriser and the segment sort take the same decision.
__device__ __forceinline__ bool item_saturated(const BatchDev& b, int64_t id) {
  const int v = view_of(b.tile_base, b.V, id);
  const ViewDev& cam = b.views[v];
  const int64_t nt = (int64_t)cam.tiles_x * cam.tiles_y;
  const int64_t t = (id - b.tile_base[v]) % nt;
  const int x0 = (int)(t % cam.tiles_x) * b.tile, y0 = (int)(t / cam.tiles_x) * b.tile;
  const float* tp = b.tpre + b.pix_off[v];
  bool open = false;
  for (int i = threadIdx.x; i < b.tile * b.tile; i += blockDim.x) {
    const int x = x0 + i % b.tile, y = y0 + i / b.tile;
    if (x < cam.W && y < cam.H) open |= tp[(int64_t)y * cam.W + x] >= b.eps_comp;
  }
  return !__syncthreads_or(open);
}

// Cross-boundary per-ray filtering (Sec. 8.1): whether a Gaussian of subset k whose support
// meets the other cells in mask c, at depth bits dbits, leaves the rays of tile (tx, ty) of
// view v: for some such cell s, the tile lies in subset s's visible region and the depth in
// the overlap of the two subsets' depth ranges.  (The tile holds a pair of the Gaussian, so
// it lies in k's.)
__device__ __forceinline__ bool cross_removed(const BatchDev& b, int v, int k,
                                              unsigned long long c, int tx, int ty,
                                              uint32_t dbits) {
  const int own = b.cell_self >= 0 ? b.cell_self : k;
  const uint32_t* zk = b.zr_x + 2 * ((int64_t)v * b.ncells + own);
  const uint32_t kmin = zk[0], kmax = ~zk[1];
  while (c) {
    const int s = __ffsll((long long)c) - 1;
    c &= c - 1ull;
    const uint4 o = reinterpret_cast<const uint4*>(b.omega_x)[v * b.ncells + s];
    const uint32_t x = (uint32_t)tx, y = (uint32_t)ty;
    if (x < o.x || y < o.y || x > ~o.z || y > ~o.w) continue;
    const uint32_t* zs = b.zr_x + 2 * ((int64_t)v * b.ncells + s);
    const uint32_t lo = max(kmin, zs[0]), hi = min(kmax, ~zs[1]);
    if (dbits >= lo && dbits <= hi) return true;
  }
  return false;
}

// Stale-state test of work item `id` (a whole tile of subset k in view v): true if every
// pixel of the tile has subset k pruned (its rank >= the pixel's state).  Whole-CTA call;
// the rasteriser and the segment sort take the same decision.
__device__ __forceinline__ bool item_pruned(const BatchDev& b, int64_t id) {
  const int v = view_of(b.tile_base, b.V, id);
  const ViewDev& cam = b.views[v];
  const int64_t nt = (int64_t)cam.tiles_x * cam.tiles_y;
  const int k = (int)((id - b.tile_base[v]) / nt);
  const int64_t t = (id - b.tile_base[v]) - (int64_t)k * nt;
  const int x0 = (int)(t % cam.tiles_x) * b.tile, y0 = (int)(t / cam.tiles_x) * b.tile;
  const uint8_t* sp = b.sat[v];
  const int rk = b.rank[v * b.K + k];
  bool open = false;
  for (int i = threadIdx.x; i < b.tile * b.tile; i += blockDim.x) {
    const int x = x0 + i % b.tile, y = y0 + i / b.tile;
    if (x < cam.W && y < cam.H) open |= (int)sp[(int64_t)y * cam.W + x] > rk;
  }
  return !__syncthreads_or(open);
}

// Asynchronous global -> shared copies (cp.async) of 16 or 4 bytes by the calling thread,
// grouped by commit; wait<N> returns once at most N of the thread's groups are pending, and
// then the thread's own copies of the older groups are visible to it.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Whether tile (tx, ty) of view v lies in subset k's visible region (always, if off).
__device__ __forceinline__ bool in_omega(const BatchDev& b, int v, int k, int tx, int ty) {
  if (!b.omega) return true;
  const uint4 o = reinterpret_cast<const uint4*>(b.omega)[v * b.K + k];
  const uint32_t x = (uint32_t)tx, y = (uint32_t)ty;
  return x >= o.x && y >= o.y && x <= ~o.z && y <= ~o.w;
}
}  // namespace splx
