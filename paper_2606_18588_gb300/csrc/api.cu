// C ABI of libsplx (declared in include/splx.h): context, per-view entry points, the
// batched V x K plan, CUDA-graph helpers and diagnostics.  Host code only; every step
// of the math runs in the kernels of project.cu, sort.cu, raster.cu, composite.cu and
// project_bwd.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace splx {
thread_local int64_t* g_launch_counter = nullptr;

namespace {
constexpr int kMaxDev = 64;
constexpr int kSmemSlots = 16;
std::mutex g_dev_mu;
int g_sm_count[kMaxDev] = {};
bool g_smem_done[kMaxDev][kSmemSlots] = {};
cudaError_t g_smem_result[kMaxDev][kSmemSlots] = {};
int g_ctas[kMaxDev][kSmemSlots] = {};
int current_device() {
  int d = 0;
  return cudaGetDevice(&d) == cudaSuccess && d >= 0 && d < kMaxDev ? d : 0;
}
}  // namespace

int device_sm_count() {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (!g_sm_count[d]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0)
      n = 152;
    g_sm_count[d] = n;
  }
  return g_sm_count[d];
}

int resident_ctas(const void* fn, int threads, int smem, int slot) {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (!g_ctas[d][slot]) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, (size_t)smem) !=
            cudaSuccess ||
        n <= 0)
      n = 1;
    g_ctas[d][slot] = n;
  }
  return g_ctas[d][slot];
}

cudaError_t opt_in_smem(const void* fn, int bytes, int slot) {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (!g_smem_done[d][slot]) {
    g_smem_result[d][slot] =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    g_smem_done[d][slot] = true;
  }
  return g_smem_result[d][slot];
}
}

using namespace splx;

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
  return SPLX_ERR_CUDA;
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

#define CK_LAUNCH()                                                     \
  do {                                                                  \
    cudaError_t e_ = cudaGetLastError();                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, "kernel launch");       \
  } while (0)

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

// ---------------------------------------------------------------- context
struct splx_ctx_s {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  cudaMemPool_t pool = nullptr;
  int* d_status = nullptr;
  int64_t launches = 0;
  std::mutex mu;
  std::unordered_map<void*, size_t> sizes;
};

namespace {

struct CtxScope {
  int prev = -1;
  explicit CtxScope(splx_ctx_t c) {
    g_launch_counter = &c->launches;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
  }
  ~CtxScope() {
    g_launch_counter = nullptr;
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

int ctx_alloc(splx_ctx_t c, void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->budget && c->in_use + bytes > c->budget) return SPLX_ERR_BUDGET;
    c->in_use += bytes;
  }
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, c->pool, s);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(c->mu);
    c->in_use -= bytes;
    return cuda_fail(e, "cudaMallocFromPoolAsync");
  }
  std::lock_guard<std::mutex> lk(c->mu);
  c->sizes[*p] = bytes;
  return SPLX_OK;
}

void ctx_free(splx_ctx_t c, void* p, cudaStream_t s) {
  if (!p) return;
  cudaFreeAsync(p, s);
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->sizes.find(p);
  if (it != c->sizes.end()) {
    c->in_use -= it->second;
    c->sizes.erase(it);
  }
}

template <typename T>
int ctx_alloc_t(splx_ctx_t c, T** p, size_t count, cudaStream_t s) {
  return ctx_alloc(c, reinterpret_cast<void**>(p), count * sizeof(T), s);
}

int check_opts(const splx_opts* o) {
  if (!o) return SPLX_ERR_INVALID;
  if (o->tile != 8 && o->tile != 16 && o->tile != 32) return SPLX_ERR_INVALID;
  if (!(o->alpha_min >= 0.0f) || !(o->alpha_max > 0.0f) || !(o->alpha_max < 1.0f)) return SPLX_ERR_INVALID;
  if (!(o->eps_T >= 0.0f) || !(o->eps_comp >= 0.0f)) return SPLX_ERR_INVALID;
  return SPLX_OK;
}

int check_cam(const splx_camera* c) {
  if (!c) return SPLX_ERR_INVALID;
  if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384) return SPLX_ERR_INVALID;
  if (!(c->fx > 0.0f) || !(c->fy > 0.0f)) return SPLX_ERR_INVALID;
  return SPLX_OK;
}

int check_gaussians(const splx_gaussians* g) {
  if (!g) return SPLX_ERR_INVALID;
  if (g->n < 0 || g->n >= (int64_t(1) << 31)) return SPLX_ERR_INVALID;
  if (g->sh_degree < 0 || g->sh_degree > 3) return SPLX_ERR_INVALID;
  if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
    return SPLX_ERR_INVALID;
  if (g->n > 0 && !aligned16(g->quats)) return SPLX_ERR_INVALID;
  return SPLX_OK;
}

ViewDev make_view(const splx_camera& c, int tile) {
  ViewDev v;
  std::memcpy(v.R, c.R, sizeof(v.R));
  std::memcpy(v.t, c.t, sizeof(v.t));
  v.fx = c.fx; v.fy = c.fy; v.cx = c.cx; v.cy = c.cy; v.near_plane = c.near_plane;
  // camera centre eye = -R^T t (double on the host, rounded once)
  for (int k = 0; k < 3; ++k)
    v.eye[k] = (float)(-((double)c.R[k] * c.t[0] + (double)c.R[3 + k] * c.t[1] +
                         (double)c.R[6 + k] * c.t[2]));
  v.W = c.width; v.H = c.height;
  v.tiles_x = (c.width + tile - 1) / tile;
  v.tiles_y = (c.height + tile - 1) / tile;
  return v;
}

int bits_for(int64_t n) {
  int b = 1;
  while (b < 62 && (int64_t(1) << b) < n) ++b;
  return b;
}

// A planned render of V views x K subsets.  The per-view entry points use V = 1 plans;
// the batch API uses one plan for the whole batch.
struct Plan {
  splx_ctx_t ctx = nullptr;
  int V = 0, K = 0, deg = 0, tile = 16;
  int64_t N = 0;
  std::vector<SubsetDev> subsets_h;
  std::vector<ViewDev> views_h;
  std::vector<ImgDev> imgs_h;
  SubsetDev* subsets_d = nullptr;
  ViewDev* views_d = nullptr;
  ImgDev* imgs_d = nullptr;
  Rec* rec = nullptr;
  uint32_t* counts = nullptr;
  uint32_t* tile_cnt = nullptr;
  uint32_t* tile_start = nullptr;
  uint64_t* keys = nullptr;
  uint64_t* keys_alt = nullptr;
  uint32_t* big_list = nullptr;
  unsigned* big_count = nullptr;
  uint2* chunks = nullptr;
  unsigned* chunk_count = nullptr;
  uint2* ranges = nullptr;
  float4* grad2d = nullptr;
  uint8_t* defer = nullptr;  // [ceil(N / 128)]: blocks left to the zero-gradient Adam pass
  unsigned long long* counters = nullptr;  // [kCounters]: see BatchDev::counters
  unsigned long long* work_ctr = nullptr;  // [2]: persistent rasterisers' work counters
  int persist_grid = 0;                    // persistent raster grid (0: one CTA per item)
  // saturation-skipping waves of view groups side by side (batches): group g > 0 runs on
  // side[g - 1] with its own long-segment lists; fork / join events
  static constexpr int kGroups = 4;
  bool split_views = false;
  cudaStream_t side[kGroups - 1] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kGroups - 1] = {};
  uint32_t* big_list_g[kGroups - 1] = {};
  unsigned* big_count_g[kGroups - 1] = {};
  uint2* chunks_g[kGroups - 1] = {};
  unsigned* chunk_count_g[kGroups - 1] = {};
  // selected-prefix sort of long segments (batches; see BatchDev::sel): per image tile the
  // prefix length, and per view group the forward's retry list and its count
  bool select_prefix = false;
  bool alt_in_keys = false;  // keys_alt = keys + capacity (one allocation, owned by keys)
  uint32_t* sel = nullptr;
  uint32_t* retry = nullptr;
  unsigned* retry_count = nullptr;
  uint32_t* retry_g[kGroups - 1] = {};
  unsigned* retry_count_g[kGroups - 1] = {};
  int32_t* order_d = nullptr;              // [V][K] front-to-back subset order (skipping on)
  int32_t* rank_d = nullptr;               // [V][K] rank of subset k in view v's order
  // stale saturation state (with order_d): device table of the V views' state planes;
  // the forward then runs one launch per stage and re-evaluates the states in place
  uint8_t** sat_d = nullptr;
  bool stale() const { return sat_d && order_d; }
  uint32_t* omega = nullptr;               // [V][K][4] visible regions (internal partials only)
  bool visibility = false;                 // use omega (batches and server launches)
  float* tpre = nullptr;                   // [total pixels] prefix transmittance of the waves
  float* cells_d = nullptr;                // [K][6] k-d boxes (cross-boundary filtering)
  unsigned long long* cross = nullptr;     // [N] cells each Gaussian's support meets
  uint32_t* zr = nullptr;                  // [V][K][2] depth ranges (min, ~max bits)
  uint32_t* removed = nullptr;             // [n_tiles] pairs the filter removed per tile
  bool cross_filter = false;               // filter cross-boundary Gaussians per ray
  bool depth_ranges = false;               // record depth ranges (zr) without filtering
  // a per-view render's filter: every cell's visible region [ncells][4] and depth range
  // [ncells][2] in this view (uploaded), and the cell of the plan's one subset
  uint32_t* omega_x = nullptr;
  uint32_t* zr_x = nullptr;
  int ncells = 0, cell_self = -1;
  void* scan_temp = nullptr;
  int64_t capacity = 0, n_tiles = 0, total_pixels = 0;
  splx_opts opts{};
  std::vector<int64_t> tile_base, pix_off;
  // per-kernel timing: events at the marks below, recorded as graph event nodes when
  // the stream is being captured.  Forward: 0 start, 1 project, 2 scan, 3 fill, 4 sort,
  // 5 raster_fwd, 6 composite; backward: 7 start, 8 composite_bwd, 9 raster_bwd,
  // 10 project_bwd.
  bool timing = false;
  cudaEvent_t ev[11] = {};
  // saturation-skipping waves: events before wave r's sort (2r), between its sort and its
  // rasteriser (2r + 1), and after the last rasteriser (2K)
  std::vector<cudaEvent_t> wev;

  void mark_wave(int i, cudaStream_t s) {
    if (!timing || i >= (int)wev.size() || !wev[i]) return;
    if (stream_capturing(s))
      cudaEventRecordWithFlags(wev[i], s, cudaEventRecordExternal);
    else
      cudaEventRecord(wev[i], s);
  }

  void mark(int i, cudaStream_t s) {
    if (!timing || !ev[i]) return;
    if (stream_capturing(s))
      cudaEventRecordWithFlags(ev[i], s, cudaEventRecordExternal);
    else
      cudaEventRecord(ev[i], s);
  }

  void layout() {
    tile_base.assign(V + 1, 0);
    pix_off.assign(V + 1, 0);
    for (int v = 0; v < V; ++v) {
      tile_base[v + 1] = tile_base[v] + (int64_t)K * views_h[v].tiles_x * views_h[v].tiles_y;
      pix_off[v + 1] = pix_off[v] + (int64_t)views_h[v].W * views_h[v].H;
    }
    n_tiles = tile_base[V];
    total_pixels = pix_off[V];
  }

  BatchDev dev() const {
    BatchDev b;
    std::memset(&b, 0, sizeof(b));
    b.V = V; b.K = K; b.sh_degree = deg; b.nc = n_sh(deg); b.N = N; b.tile = tile;
    b.n_tiles = n_tiles;
    b.tile_bits = bits_for(n_tiles + 1);
    b.capacity = capacity;
    b.eps_T = opts.eps_T; b.eps_comp = opts.eps_comp;
    b.alpha_min = opts.alpha_min; b.alpha_max = opts.alpha_max;
    for (int c = 0; c < 3; ++c) b.bg[c] = opts.bg[c];
    b.subsets = subsets_d; b.views = views_d; b.imgs = imgs_d;
    b.rec = rec; b.counts = counts; b.tile_cnt = tile_cnt; b.tile_start = tile_start;
    b.keys = keys; b.keys_alt = keys_alt; b.big_list = big_list; b.big_count = big_count;
    b.chunks = chunks; b.chunk_count = chunk_count;
    b.ranges = ranges; b.grad2d = grad2d;
    b.status = ctx->d_status;
    b.counters = counters;
    b.persist_grid = persist_grid;
    b.work_ctr = work_ctr;
    b.omega = visibility ? omega : nullptr;
    // the filter needs the cells' visible regions: the batch's own (visibility on) or, for a
    // per-view render, the uploaded ones
    const bool cf = cross_filter && (omega_x || (visibility && omega)) && cells_d && cross &&
                    zr && removed;
    b.cells = cf ? cells_d : nullptr;
    b.cross = cf ? cross : nullptr;
    b.zr = cf || (depth_ranges && zr) ? zr : nullptr;
    b.removed = cf ? removed : nullptr;
    b.omega_x = omega_x ? omega_x : omega;
    b.zr_x = zr_x ? zr_x : zr;
    b.ncells = ncells > 0 ? ncells : K;
    b.cell_self = cell_self;
    b.order = nullptr;  // set per launch by the forward's waves
    b.wave = 0;
    b.item_lo = 0;
    b.item_n = K > 0 ? n_tiles / K : 0;
    b.tpre = tpre;
    b.sat = stale() ? sat_d : nullptr;
    b.rank = rank_d;
    // (the cross-boundary filter's removed pairs keep the whole-segment sort)
    b.sel = select_prefix && alt_in_keys && sel && !b.removed ? sel : nullptr;
    b.retry = retry;
    b.retry_count = retry_count;
    // composite-only plans carry no subsets; their offsets are unused
    for (int k = 0; k <= K; ++k) b.goff[k] = k < (int)subsets_h.size() ? subsets_h[k].goff : N;
    for (int v = 0; v <= V; ++v) { b.tile_base[v] = tile_base[v]; b.pix_off[v] = pix_off[v]; }
    return b;
  }

  void free_ptr(void*& p, cudaStream_t s) {
    ctx_free(ctx, p, s);
    p = nullptr;
  }

  void release(cudaStream_t s) {
    if (alt_in_keys) {
      keys_alt = nullptr;  // part of keys' allocation
      alt_in_keys = false;
    }
    void** ps[] = {(void**)&subsets_d, (void**)&views_d, (void**)&imgs_d, (void**)&rec,
                   (void**)&counts, (void**)&tile_cnt, (void**)&tile_start, (void**)&keys,
                   (void**)&keys_alt, (void**)&big_list, (void**)&big_count, (void**)&chunks,
                   (void**)&chunk_count, (void**)&ranges,
                   (void**)&grad2d, (void**)&defer, (void**)&scan_temp, (void**)&counters, (void**)&work_ctr,
                   (void**)&order_d, (void**)&rank_d, (void**)&sat_d, (void**)&tpre,
                   (void**)&omega, (void**)&cells_d,
                   (void**)&cross, (void**)&zr, (void**)&removed, (void**)&omega_x,
                   (void**)&zr_x, (void**)&sel, (void**)&retry, (void**)&retry_count};
    for (void** p : ps) free_ptr(*p, s);
    for (int g = 0; g < kGroups - 1; ++g) {
      free_ptr((void*&)retry_g[g], s);
      free_ptr((void*&)retry_count_g[g], s);
      free_ptr((void*&)big_list_g[g], s);
      free_ptr((void*&)big_count_g[g], s);
      free_ptr((void*&)chunks_g[g], s);
      free_ptr((void*&)chunk_count_g[g], s);
      if (side[g]) { cudaStreamSynchronize(side[g]); cudaStreamDestroy(side[g]); side[g] = nullptr; }
      if (join_ev[g]) { cudaEventDestroy(join_ev[g]); join_ev[g] = nullptr; }
    }
    if (fork_ev) { cudaEventDestroy(fork_ev); fork_ev = nullptr; }
    for (auto& e : ev)
      if (e) { cudaEventDestroy(e); e = nullptr; }
    for (auto& e : wev)
      if (e) cudaEventDestroy(e);
    wev.clear();
  }

  // Project (counting pairs per tile) and scan the counts into segment starts.
  int project_and_count(cudaStream_t s) {
    const BatchDev b = dev();
    if (counters && !stream_capturing(s))
      CK(cudaMemsetAsync(counters, 0, kCounters * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(tile_cnt, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(n_tiles, 1), s));
    if (visibility && omega)
      CK(cudaMemsetAsync(omega, 0xFF, sizeof(uint32_t) * 4 * (size_t)V * K, s));
    if (b.zr) CK(cudaMemsetAsync(zr, 0xFF, sizeof(uint32_t) * 2 * (size_t)V * K, s));
    if (b.removed)
      CK(cudaMemsetAsync(removed, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(n_tiles, 1), s));
    CK(cudaMemsetAsync(big_count, 0, 2 * sizeof(unsigned), s));
    CK(cudaMemsetAsync(chunk_count, 0, sizeof(unsigned), s));
    mark(0, s);
    launch_project(b, s);
    CK_LAUNCH();
    mark(1, s);
    scan_u32(tile_cnt, tile_start, n_tiles, scan_temp, s);
    CK_LAUNCH();
    mark(2, s);
    return SPLX_OK;
  }

  // Fill the tile buckets and sort every segment (needs capacity > 0).
  int fill_and_sort(cudaStream_t s) {
    const BatchDev b = dev();
    launch_fill(b, s);
    CK_LAUNCH();
    mark(3, s);
    // with saturation-skipping waves each wave sorts its own segments; with a stale state
    // one sort covers the tiles it leaves open
    if (!order_d || stale()) {
      if (b.sel) CK(cudaMemsetAsync(retry_count, 0, sizeof(unsigned), s));
      launch_seg_sort(b, merge_rounds_bound(max_subset()), s);
      CK_LAUNCH();
    }
    mark(4, s);
    return SPLX_OK;
  }

  // Forward rasterisation with saturation skipping: per wave, sort the wave's segments
  // (those of saturated items are left unsorted) and render them.
  // Saturation skipping: K waves, wave r sorting and rendering subset order[v][r] of every
  // view v after the waves before it (the prefix transmittance it reads).  With
  // split_views the views form up to kGroups groups of about equal pixels whose waves run
  // on their own streams, so that one group's kernels fill the others' wave tails; the
  // groups share nothing but the read-only inputs.
  int waves(const BatchDev& b, cudaStream_t s) {
    const int64_t nw = n_tiles / K;
    // first view of each group; groups[G] = V
    int G = 1, first[kGroups + 1] = {0};
    if (split_views && persist_grid == 0 && V >= 2) {
      G = std::min(kGroups, V);
      for (int g = 1; g < G; ++g) {
        // the view whose start is nearest to g / G of the pixels, after the previous group's
        int v = first[g - 1] + 1;
        while (v < V - (G - g) && G * (pix_off[v] + pix_off[v + 1]) <= 2 * g * pix_off[V]) ++v;
        first[g] = v;
      }
    }
    first[G] = V;
    mark_wave(0, s);
    if (G > 1) {
      CK(cudaEventRecord(fork_ev, s));
      for (int g = 1; g < G; ++g) CK(cudaStreamWaitEvent(side[g - 1], fork_ev, 0));
    }
    for (int r = 0; r < K; ++r) {
      BatchDev bg[kGroups];
      for (int g = 0; g < G; ++g) {
        BatchDev& bw = bg[g];
        bw = b;
        bw.order = order_d;
        bw.wave = r;
        bw.item_lo = tile_base[first[g]] / K;
        bw.item_n = tile_base[first[g + 1]] / K - bw.item_lo;
        if (g > 0) {
          bw.big_list = big_list_g[g - 1]; bw.big_count = big_count_g[g - 1];
          bw.chunks = chunks_g[g - 1]; bw.chunk_count = chunk_count_g[g - 1];
          bw.retry = retry_g[g - 1]; bw.retry_count = retry_count_g[g - 1];
        }
      }
      if (r > 0) mark_wave(2 * r, s);
      const int rounds = merge_rounds_bound(max_subset());
      for (int g = 0; g < G; ++g) {
        cudaStream_t sg = g ? side[g - 1] : s;
        CK(cudaMemsetAsync(bg[g].big_count, 0, 2 * sizeof(unsigned), sg));
        CK(cudaMemsetAsync(bg[g].chunk_count, 0, sizeof(unsigned), sg));
        if (bg[g].sel) CK(cudaMemsetAsync(bg[g].retry_count, 0, sizeof(unsigned), sg));
        launch_seg_sort(bg[g], rounds, sg);
      }
      mark_wave(2 * r + 1, s);
      for (int g = 0; g < G; ++g) {
        cudaStream_t sg = g ? side[g - 1] : s;
        launch_raster_fwd(bg[g], sg);
        // items whose pixels were still open at the end of their selected prefix: full
        // sort, second forward
        launch_sort_retries(bg[g], rounds, sg);
        launch_raster_fwd_retry(bg[g], sg);
      }
      CK_LAUNCH();
    }
    for (int g = 1; g < G; ++g) {
      CK(cudaEventRecord(join_ev[g - 1], side[g - 1]));
      CK(cudaStreamWaitEvent(s, join_ev[g - 1], 0));
    }
    mark_wave(2 * K, s);
    (void)nw;
    return SPLX_OK;
  }

  int bin(cudaStream_t s) {
    int r;
    if ((r = project_and_count(s))) return r;
    if (capacity <= 0) return SPLX_OK;
    return fill_and_sort(s);
  }

  int alloc_pairs(int64_t cap, cudaStream_t s) {
    capacity = cap;
    int r;
    if (select_prefix && cap > 0 && 2 * cap < (int64_t(1) << 32)) {
      // selected prefixes are named by ranges into keys_alt through keys: one allocation
      if ((r = ctx_alloc_t(ctx, &keys, (size_t)(2 * cap), s))) return r;
      keys_alt = keys + cap;
      alt_in_keys = true;
    } else {
      if ((r = ctx_alloc_t(ctx, &keys, (size_t)std::max<int64_t>(cap, 1), s))) return r;
      if ((r = ctx_alloc_t(ctx, &keys_alt, (size_t)std::max<int64_t>(cap, 1), s))) return r;
    }
    if ((r = ctx_alloc_t(ctx, &chunks, (size_t)chunk_list_capacity(n_tiles, cap), s))) return r;
    if (split_views)
      for (int g = 0; g < kGroups - 1; ++g)
        if ((r = ctx_alloc_t(ctx, &chunks_g[g], (size_t)chunk_list_capacity(n_tiles, cap), s)))
          return r;
    return SPLX_OK;
  }

  // The other view groups' streams, events and long-segment lists (split_views).
  int alloc_split(cudaStream_t s) {
    int r;
    const size_t nt = (size_t)std::max<int64_t>(n_tiles, 1);
    for (int g = 0; g < kGroups - 1; ++g) {
      if ((r = ctx_alloc_t(ctx, &big_list_g[g], nt, s))) return r;
      if ((r = ctx_alloc_t(ctx, &big_count_g[g], 2, s))) return r;
      if ((r = ctx_alloc_t(ctx, &chunk_count_g[g], 1, s))) return r;
      CK(cudaStreamCreateWithFlags(&side[g], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&join_ev[g], cudaEventDisableTiming));
    }
    CK(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
    split_views = true;
    return SPLX_OK;
  }

  // Selected-prefix sort state (batches): per tile prefix lengths, retry lists per group.
  int alloc_select(cudaStream_t s) {
    int r;
    const size_t nt = (size_t)std::max<int64_t>(n_tiles, 1);
    if ((r = ctx_alloc_t(ctx, &sel, nt, s))) return r;
    if ((r = ctx_alloc_t(ctx, &retry, nt, s))) return r;
    if ((r = ctx_alloc_t(ctx, &retry_count, 1, s))) return r;
    if (split_views)
      for (int g = 0; g < kGroups - 1; ++g) {
        if ((r = ctx_alloc_t(ctx, &retry_g[g], nt, s))) return r;
        if ((r = ctx_alloc_t(ctx, &retry_count_g[g], 1, s))) return r;
      }
    CK(cudaMemsetAsync(sel, 0, sizeof(uint32_t) * nt, s));
    CK(cudaMemsetAsync(retry_count, 0, sizeof(unsigned), s));
    for (int g = 0; g < kGroups - 1; ++g)
      if (retry_count_g[g]) CK(cudaMemsetAsync(retry_count_g[g], 0, sizeof(unsigned), s));
    select_prefix = true;
    return SPLX_OK;
  }

  int alloc_common(cudaStream_t s) {
    int r;
    const size_t nt = (size_t)std::max<int64_t>(n_tiles, 1);
    if ((r = ctx_alloc_t(ctx, &subsets_d, std::max<size_t>(subsets_h.size(), 1), s))) return r;
    if ((r = ctx_alloc_t(ctx, &views_d, views_h.size(), s))) return r;
    if ((r = ctx_alloc_t(ctx, &imgs_d, std::max<size_t>(imgs_h.size(), 1), s))) return r;
    if ((r = ctx_alloc_t(ctx, &rec, (size_t)std::max<int64_t>((int64_t)V * N, 1), s))) return r;
    if ((r = ctx_alloc_t(ctx, &counts, (size_t)std::max<int64_t>((int64_t)V * N, 1), s))) return r;
    if ((r = ctx_alloc_t(ctx, &tile_cnt, nt, s))) return r;
    if ((r = ctx_alloc_t(ctx, &tile_start, nt + 1, s))) return r;
    if ((r = ctx_alloc_t(ctx, &big_list, nt, s))) return r;
    if ((r = ctx_alloc_t(ctx, &big_count, 2, s))) return r;  // count, most chunks of one
    if ((r = ctx_alloc_t(ctx, &chunk_count, 1, s))) return r;
    if ((r = ctx_alloc(ctx, &scan_temp, scan_u32_temp_bytes(n_tiles), s))) return r;
    if ((r = ctx_alloc_t(ctx, &ranges, nt, s))) return r;
    if (!subsets_h.empty())
      CK(cudaMemcpyAsync(subsets_d, subsets_h.data(), sizeof(SubsetDev) * subsets_h.size(),
                         cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(views_d, views_h.data(), sizeof(ViewDev) * views_h.size(),
                       cudaMemcpyHostToDevice, s));
    if (!imgs_h.empty())
      CK(cudaMemcpyAsync(imgs_d, imgs_h.data(), sizeof(ImgDev) * imgs_h.size(),
                         cudaMemcpyHostToDevice, s));
    return SPLX_OK;
  }

  int64_t max_subset() const {
    int64_t m = 0;
    for (const SubsetDev& d : subsets_h) m = std::max<int64_t>(m, d.n);
    return m;
  }

  // Pair count of the last projection (synchronises).
  int read_total(uint64_t* total, cudaStream_t s) {
    uint32_t t = 0;
    CK(cudaMemcpyAsync(&t, tile_start + n_tiles, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *total = t;
    return SPLX_OK;
  }
};

SubsetDev make_subset(const splx_gaussians& g, int64_t goff) {
  SubsetDev d;
  std::memset(&d, 0, sizeof(d));
  d.means = g.means; d.log_scales = g.log_scales; d.quats = g.quats;
  d.opacity_logits = g.opacity_logits; d.sh = g.sh; d.n = g.n; d.goff = goff;
  return d;
}

}  // namespace

struct splx_state_s {
  Plan plan;
  bool has_grad2d = false;
};

struct splx_batch_s {
  Plan plan;
  splx_camera* pinned_cams = nullptr;
  float4* gCT = nullptr;       // [K * total_pixels]
  float* partial = nullptr;    // rgb [3 K P], T [K P], D [K P] (P = total pixels)
  int32_t* last = nullptr;     // [K P]
  float* ssim_maps = nullptr;  // [3][3 P]: D-SSIM partial-derivative maps
  double* ssim_sums = nullptr; // [2]: sum of SSIM, sum of |x - y|
  bool forward_done = false;
};

struct splx_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // timing ring: the graph's event-record nodes, the events they captured, and per ring
  // slot the events they record instead on the launch that takes that slot
  std::vector<cudaGraphNode_t> ev_nodes;
  std::vector<cudaEvent_t> ev_orig;
  std::vector<cudaEvent_t> ring;  // [slots][ev_nodes.size()]
  int slots = 0, next = 0;

  // The event that stands for `e` in ring slot `slot` (e itself without a ring).
  cudaEvent_t in_slot(cudaEvent_t e, int slot) const {
    if (slots <= 0 || slot < 0 || slot >= slots) return e;
    for (size_t k = 0; k < ev_orig.size(); ++k)
      if (ev_orig[k] == e) return ring[(size_t)slot * ev_orig.size() + k];
    return e;
  }
};

extern "C" {

int splx_create(splx_ctx_t* out, int device, size_t hbm_budget_bytes) {
  if (!out) return SPLX_ERR_INVALID;
  *out = nullptr;
  int n = 0;
  CK(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return SPLX_ERR_INVALID;
  splx_ctx_t c = new (std::nothrow) splx_ctx_s();
  if (!c) return SPLX_ERR_BUDGET;
  c->device = device;
  c->budget = hbm_budget_bytes;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  cudaError_t e = cudaMemPoolCreate(&c->pool, &props);
  if (e == cudaSuccess) {
    uint64_t thr = ~0ull;
    e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
  if (e == cudaSuccess && ssim_init() != 0) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "splx_create");
  }
  *out = c;
  return SPLX_OK;
}

int splx_destroy(splx_ctx_t c) {
  if (!c) return SPLX_ERR_INVALID;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  cudaFree(c->d_status);
  cudaMemPoolDestroy(c->pool);
  cudaSetDevice(prev);
  delete c;
  return SPLX_OK;
}

size_t splx_scratch_bytes(splx_ctx_t c) {
  if (!c) return 0;
  std::lock_guard<std::mutex> lk(c->mu);
  return c->in_use;
}

// The filter of a per-view render (splx_render_partial_filtered): K cells, this subset's
// cell k, the cells' boxes and their visible regions and depth ranges in the view.
struct ViewFilter {
  int K, k;
  const float* cells;      // host [K][6]
  const uint32_t* regions; // host [K][6]
};

static int render_partial_impl(splx_ctx_t ctx, const splx_gaussians* subset,
                               const splx_camera* cam, const splx_opts* opts,
                               const splx_partial* out, splx_state_t* state_out,
                               splx_stream_t stream, const ViewFilter* vf) {
  if (!ctx || !out || !out->rgb || !out->T || !out->depth || !out->last) return SPLX_ERR_INVALID;
  int r;
  if ((r = check_gaussians(subset)) || (r = check_cam(cam)) || (r = check_opts(opts))) return r;
  if (state_out) *state_out = nullptr;
  CtxScope scope(ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  splx_state_s* st = new (std::nothrow) splx_state_s();
  if (!st) return SPLX_ERR_BUDGET;
  Plan& P = st->plan;
  P.ctx = ctx; P.V = 1; P.K = 1; P.deg = subset->sh_degree; P.tile = opts->tile; P.N = subset->n;
  P.opts = *opts;
  P.subsets_h.push_back(make_subset(*subset, 0));
  P.views_h.push_back(make_view(*cam, opts->tile));
  ImgDev im;
  im.rgb = out->rgb; im.T = out->T; im.D = out->depth; im.last = out->last; im.gCT = nullptr;
  P.imgs_h.push_back(im);
  P.layout();
  auto fail = [&](int code) {
    P.release(s);
    delete st;
    return code;
  };
  if ((r = P.alloc_common(s))) return fail(r);
  if (vf) {
    // the batch's filter with this subset as cell k of K, the cells' visible regions and
    // depth ranges from `regions`; every tile is rendered (tiles outside the subset's own
    // region have no pairs and come out empty, as the batch's composite reads them)
    if ((r = ctx_alloc_t(ctx, &P.cells_d, (size_t)6 * vf->K, s))) return fail(r);
    if ((r = ctx_alloc_t(ctx, &P.cross, (size_t)std::max<int64_t>(P.N, 1), s))) return fail(r);
    if ((r = ctx_alloc_t(ctx, &P.zr, 2, s))) return fail(r);
    if ((r = ctx_alloc_t(ctx, &P.removed, (size_t)std::max<int64_t>(P.n_tiles, 1), s)))
      return fail(r);
    if ((r = ctx_alloc_t(ctx, &P.omega_x, (size_t)4 * vf->K, s))) return fail(r);
    if ((r = ctx_alloc_t(ctx, &P.zr_x, (size_t)2 * vf->K, s))) return fail(r);
    std::vector<uint32_t> om((size_t)4 * vf->K), zr((size_t)2 * vf->K);
    for (int c = 0; c < vf->K; ++c) {
      for (int e = 0; e < 4; ++e) om[(size_t)4 * c + e] = vf->regions[(size_t)6 * c + e];
      for (int e = 0; e < 2; ++e) zr[(size_t)2 * c + e] = vf->regions[(size_t)6 * c + 4 + e];
    }
    CK(cudaMemcpyAsync(P.cells_d, vf->cells, sizeof(float) * 6 * vf->K, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.omega_x, om.data(), sizeof(uint32_t) * om.size(),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.zr_x, zr.data(), sizeof(uint32_t) * zr.size(), cudaMemcpyHostToDevice,
                       s));
    P.cross_filter = true;
    P.ncells = vf->K;
    P.cell_self = vf->k;
  }
  if ((r = P.project_and_count(s))) return fail(r);
  uint64_t total = 0;
  if ((r = P.read_total(&total, s))) return fail(r);
  if (total >= (uint64_t)UINT32_MAX) return fail(SPLX_ERR_CAPACITY);
  if ((r = P.alloc_pairs((int64_t)total, s))) return fail(r);
  if ((r = P.fill_and_sort(s))) return fail(r);
  launch_raster_fwd(P.dev(), s);
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(cuda_fail(e, "render_partial launch"));
  }
  // keep only what the backward needs (records, tile counts, sorted keys, ranges,
  // descriptors; a zero count marks a culled Gaussian, whose record is not written)
  P.free_ptr((void*&)P.scan_temp, s);
  P.free_ptr((void*&)P.keys_alt, s);
  P.free_ptr((void*&)P.tile_cnt, s);
  P.free_ptr((void*&)P.big_list, s);
  P.free_ptr((void*&)P.big_count, s);
  P.free_ptr((void*&)P.chunks, s);
  P.free_ptr((void*&)P.chunk_count, s);
  if (!state_out) return fail(SPLX_OK);
  *state_out = st;
  return SPLX_OK;
}

int splx_render_partial(splx_ctx_t ctx, const splx_gaussians* subset, const splx_camera* cam,
                        const splx_opts* opts, const splx_partial* out, splx_state_t* state_out,
                        splx_stream_t stream) {
  return render_partial_impl(ctx, subset, cam, opts, out, state_out, stream, nullptr);
}

int splx_render_partial_filtered(splx_ctx_t ctx, const splx_gaussians* subset, int32_t k,
                                 int32_t K, const float* cells, const uint32_t* regions,
                                 const splx_camera* cam, const splx_opts* opts,
                                 const splx_partial* out, splx_state_t* state_out,
                                 splx_stream_t stream) {
  if (!cells || !regions || K < 1 || K > 64 || k < 0 || k >= K) return SPLX_ERR_INVALID;
  for (int i = 0; i < 6 * K; ++i)
    if (std::isnan(cells[i])) return SPLX_ERR_INVALID;
  const ViewFilter vf{K, k, cells, regions};
  return render_partial_impl(ctx, subset, cam, opts, out, state_out, stream, &vf);
}

int splx_view_regions(splx_ctx_t ctx, const splx_gaussians* subsets, int32_t K,
                      const splx_camera* cam, const splx_opts* opts, uint32_t* regions_out,
                      splx_stream_t stream) {
  if (!ctx || !subsets || !regions_out || K < 1 || K > kMaxK) return SPLX_ERR_INVALID;
  int r;
  if ((r = check_cam(cam)) || (r = check_opts(opts))) return r;
  int64_t N = 0;
  for (int k = 0; k < K; ++k) {
    if ((r = check_gaussians(&subsets[k]))) return r;
    if (subsets[k].sh_degree != subsets[0].sh_degree) return SPLX_ERR_INVALID;
    N += subsets[k].n;
  }
  CtxScope scope(ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Plan P;
  P.ctx = ctx; P.V = 1; P.K = K; P.deg = subsets[0].sh_degree; P.tile = opts->tile; P.N = N;
  P.opts = *opts;
  int64_t goff = 0;
  for (int k = 0; k < K; ++k) {
    P.subsets_h.push_back(make_subset(subsets[k], goff));
    goff += subsets[k].n;
  }
  P.views_h.push_back(make_view(*cam, opts->tile));
  P.layout();
  for (int k = 0; k < K; ++k) {
    ImgDev im{};
    P.imgs_h.push_back(im);
  }
  auto done = [&](int code) {
    P.release(s);
    return code;
  };
  if ((r = P.alloc_common(s))) return done(r);
  if ((r = ctx_alloc_t(ctx, &P.omega, (size_t)4 * K, s))) return done(r);
  if ((r = ctx_alloc_t(ctx, &P.zr, (size_t)2 * K, s))) return done(r);
  P.visibility = true;
  P.depth_ranges = true;
  if ((r = P.project_and_count(s))) return done(r);
  std::vector<uint32_t> om((size_t)4 * K), zr((size_t)2 * K);
  cudaError_t e = cudaMemcpyAsync(om.data(), P.omega, sizeof(uint32_t) * om.size(),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(zr.data(), P.zr, sizeof(uint32_t) * zr.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return done(cuda_fail(e, "splx_view_regions"));
  for (int k = 0; k < K; ++k) {
    for (int i = 0; i < 4; ++i) regions_out[(size_t)6 * k + i] = om[(size_t)4 * k + i];
    for (int i = 0; i < 2; ++i) regions_out[(size_t)6 * k + 4 + i] = zr[(size_t)2 * k + i];
  }
  return done(SPLX_OK);
}

namespace splx {
// The projection writes no record for a culled Gaussian; the export shows it as documented
// (zeros, rectangle x0 = y0 = 0xFFFF > x1 = y1 = 0).
__global__ void k_export_culled(Rec* rec, const uint32_t* counts, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || counts[i]) return;
  Rec r;
  r.a = make_float4(0.f, 0.f, 0.f, 0.f);
  r.b = make_float4(0.f, 0.f, 0.f, __uint_as_float(0xFFFFu));
  r.c = make_float4(0.f, 0.f, 0.f, __uint_as_float(0xFFFFu));
  r.d = make_float4(0.f, 0.f, 0.f, 0.f);
  rec[i] = r;
}
}  // namespace splx

int splx_state_export(splx_ctx_t ctx, splx_state_t st, int64_t* n_pairs, int64_t* n_tiles,
                      uint32_t* ranges_out, uint64_t* keys_out, float* rec_out,
                      splx_stream_t stream) {
  if (!ctx || !st) return SPLX_ERR_INVALID;
  CtxScope scope(ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const Plan& P = st->plan;
  if (n_pairs) *n_pairs = P.capacity;
  if (n_tiles) *n_tiles = P.n_tiles;
  if (ranges_out && P.n_tiles > 0)
    CK(cudaMemcpyAsync(ranges_out, P.ranges, sizeof(uint2) * P.n_tiles, cudaMemcpyDeviceToDevice, s));
  if (keys_out && P.capacity > 0)
    CK(cudaMemcpyAsync(keys_out, P.keys, sizeof(uint64_t) * P.capacity, cudaMemcpyDeviceToDevice, s));
  if (rec_out && P.N > 0) {
    if (!P.counts) return SPLX_ERR_STATE;
    CK(cudaMemcpyAsync(rec_out, P.rec, sizeof(Rec) * P.N, cudaMemcpyDeviceToDevice, s));
    k_export_culled<<<(unsigned)((P.N + 255) / 256), 256, 0, s>>>(reinterpret_cast<Rec*>(rec_out),
                                                                  P.counts, P.N);
    CK_LAUNCH();
  }
  CK(cudaStreamSynchronize(s));
  return SPLX_OK;
}

int splx_state_release(splx_ctx_t ctx, splx_state_t st, splx_stream_t stream) {
  if (!ctx || !st) return SPLX_ERR_INVALID;
  CtxScope scope(ctx);
  st->plan.release(reinterpret_cast<cudaStream_t>(stream));
  delete st;
  return SPLX_OK;
}

int splx_composite(splx_ctx_t ctx, const splx_partial* parts, int32_t K, int32_t width,
                   int32_t height, const splx_opts* opts, float* out_rgb, float* out_T,
                   splx_stream_t stream) {
  if (!ctx || !parts || K < 1 || K > kMaxK || width < 1 || height < 1 || !out_rgb)
    return SPLX_ERR_INVALID;
  int r;
  if ((r = check_opts(opts))) return r;
  for (int k = 0; k < K; ++k)
    if (!parts[k].rgb || !parts[k].T || !parts[k].depth) return SPLX_ERR_INVALID;
  CtxScope scope(ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Plan P;
  P.ctx = ctx; P.V = 1; P.K = K; P.tile = opts->tile; P.opts = *opts;
  splx_camera cam;
  std::memset(&cam, 0, sizeof(cam));
  cam.width = width; cam.height = height; cam.fx = cam.fy = 1.0f;
  P.views_h.push_back(make_view(cam, opts->tile));
  for (int k = 0; k < K; ++k) {
    ImgDev im;
    im.rgb = parts[k].rgb; im.T = parts[k].T; im.D = parts[k].depth; im.last = parts[k].last;
    im.gCT = nullptr;
    P.imgs_h.push_back(im);
  }
  P.layout();
  if ((r = ctx_alloc_t(ctx, &P.views_d, 1, s))) return r;
  if ((r = ctx_alloc_t(ctx, &P.imgs_d, (size_t)K, s))) { P.release(s); return r; }
  cudaError_t e = cudaMemcpyAsync(P.views_d, P.views_h.data(), sizeof(ViewDev), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P.imgs_d, P.imgs_h.data(), sizeof(ImgDev) * K, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) { P.release(s); return cuda_fail(e, "composite upload"); }
  BatchDev b = P.dev();
  b.out_rgb = out_rgb;
  b.out_T = out_T;
  launch_composite(b, P.total_pixels, s);
  e = cudaGetLastError();
  P.release(s);
  if (e != cudaSuccess) return cuda_fail(e, "composite launch");
  return SPLX_OK;
}

int splx_backward(splx_ctx_t ctx, const splx_gaussians* subsets, int32_t K,
                  const splx_camera* cam, const splx_partial* parts, const splx_state_t* states,
                  const float* dL_drgb, const float* dL_dT, const splx_opts* opts,
                  const splx_params* grads, splx_stream_t stream) {
  if (!ctx || !subsets || K < 1 || K > kMaxK || !parts || !states || !dL_drgb || !grads)
    return SPLX_ERR_INVALID;
  int r;
  if ((r = check_cam(cam)) || (r = check_opts(opts))) return r;
  for (int k = 0; k < K; ++k) {
    if (!states[k] || (r = check_gaussians(&subsets[k]))) return r ? r : SPLX_ERR_INVALID;
    if (states[k]->plan.N != subsets[k].n || states[k]->plan.views_h[0].W != cam->width ||
        states[k]->plan.views_h[0].H != cam->height || states[k]->plan.tile != opts->tile)
      return SPLX_ERR_STATE;
    if (subsets[k].n > 0 && (!grads[k].means || !grads[k].log_scales || !grads[k].quats ||
                             !grads[k].opacity_logits || !grads[k].sh || !aligned16(grads[k].quats)))
      return SPLX_ERR_INVALID;
  }
  CtxScope scope(ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t HW = (int64_t)cam->width * cam->height;
  // 1. composite adjoint for all K subsets of this view
  Plan C;
  C.ctx = ctx; C.V = 1; C.K = K; C.tile = opts->tile; C.opts = *opts;
  C.views_h.push_back(make_view(*cam, opts->tile));
  float4* gCT = nullptr;
  if ((r = ctx_alloc_t(ctx, &gCT, (size_t)K * HW, s))) return r;
  for (int k = 0; k < K; ++k) {
    ImgDev im;
    im.rgb = parts[k].rgb; im.T = parts[k].T; im.D = parts[k].depth; im.last = parts[k].last;
    im.gCT = gCT + (int64_t)k * HW;
    C.imgs_h.push_back(im);
  }
  C.layout();
  auto cleanup = [&](int code) {
    C.release(s);
    ctx_free(ctx, gCT, s);
    return code;
  };
  if ((r = ctx_alloc_t(ctx, &C.views_d, 1, s))) return cleanup(r);
  if ((r = ctx_alloc_t(ctx, &C.imgs_d, (size_t)K, s))) return cleanup(r);
  cudaError_t e = cudaMemcpyAsync(C.views_d, C.views_h.data(), sizeof(ViewDev), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(C.imgs_d, C.imgs_h.data(), sizeof(ImgDev) * K, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "backward upload"));
  {
    BatchDev b = C.dev();
    b.dL_drgb = dL_drgb;
    b.dL_dT = dL_dT;
    launch_composite_bwd(b, C.total_pixels, s);
  }
  // 2. per subset: raster adjoint into per-Gaussian 2-D gradients, then projection adjoint
  for (int k = 0; k < K; ++k) {
    Plan& P = states[k]->plan;
    if (P.N == 0) continue;
    // refresh the image table with this view's adjoint plane
    P.imgs_h[0].rgb = parts[k].rgb; P.imgs_h[0].T = parts[k].T; P.imgs_h[0].D = parts[k].depth;
    P.imgs_h[0].last = parts[k].last; P.imgs_h[0].gCT = gCT + (int64_t)k * HW;
    e = cudaMemcpyAsync(P.imgs_d, P.imgs_h.data(), sizeof(ImgDev), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "backward upload"));
    if (!P.grad2d) {
      if ((r = ctx_alloc_t(ctx, &P.grad2d, (size_t)P.N * 3, s))) return cleanup(r);
      e = cudaMemsetAsync(P.grad2d, 0, sizeof(float4) * 3 * (size_t)P.N, s);
      if (e != cudaSuccess) return cleanup(cuda_fail(e, "memset grad2d"));
    }
    BatchDev b = P.dev();
    launch_raster_bwd(b, s);
    GradTable gt;
    std::memset(&gt, 0, sizeof(gt));
    gt.p[0][0] = grads[k].means; gt.p[0][1] = grads[k].log_scales; gt.p[0][2] = grads[k].quats;
    gt.p[0][3] = grads[k].opacity_logits; gt.p[0][4] = grads[k].sh;
    launch_project_bwd(b, gt, s);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "backward launch"));
  return cleanup(SPLX_OK);
}

namespace {
int adam_all(splx_ctx_t ctx, const splx_params* p, const splx_params* g, const splx_params* m,
             const splx_params* v, const splx_adam* hp, int64_t step, int64_t* step_dev,
             cudaStream_t s) {
  if (!p || !g || !m || !v || !hp) return SPLX_ERR_INVALID;
  if (p->n < 0 || p->sh_degree < 0 || p->sh_degree > 3) return SPLX_ERR_INVALID;
  if (g->n != p->n || m->n != p->n || v->n != p->n) return SPLX_ERR_INVALID;
  const int nc = n_sh(p->sh_degree);
  float* const P[5] = {p->means, p->log_scales, p->quats, p->opacity_logits, p->sh};
  float* const G[5] = {g->means, g->log_scales, g->quats, g->opacity_logits, g->sh};
  float* const M[5] = {m->means, m->log_scales, m->quats, m->opacity_logits, m->sh};
  float* const Vv[5] = {v->means, v->log_scales, v->quats, v->opacity_logits, v->sh};
  const int64_t cnt[5] = {3 * p->n, 3 * p->n, 4 * p->n, p->n, (int64_t)3 * nc * p->n};
  if (p->n == 0) return SPLX_OK;
  for (int i = 0; i < 5; ++i)
    if (!P[i] || !G[i] || !M[i] || !Vv[i]) return SPLX_ERR_INVALID;
  if (step_dev) launch_step_increment(step_dev, s);
  for (int i = 0; i < 5; ++i) {
    const bool vec = aligned16(P[i]) && aligned16(G[i]) && aligned16(M[i]) && aligned16(Vv[i]);
    const float lr = hp->lr[i < 4 ? i : 4];
    const float lr_rest = i == 4 ? hp->lr[5] : lr;
    launch_adam(P[i], G[i], M[i], Vv[i], cnt[i], i == 4 ? 3 * nc : 0, lr, lr_rest, hp->beta1,
                hp->beta2, hp->eps, step, step_dev, hp->zero_grad != 0, vec, s);
  }
  CK_LAUNCH();
  return SPLX_OK;
}
}  // namespace

int splx_step(splx_ctx_t ctx, const splx_params* p, const splx_params* g, const splx_params* m,
              const splx_params* v, const splx_adam* hp, int64_t step, splx_stream_t stream) {
  if (!ctx || step < 1) return SPLX_ERR_INVALID;
  CtxScope scope(ctx);
  return adam_all(ctx, p, g, m, v, hp, step, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

int splx_step_device(splx_ctx_t ctx, const splx_params* p, const splx_params* g,
                     const splx_params* m, const splx_params* v, const splx_adam* hp,
                     int64_t* step_dev, splx_stream_t stream) {
  if (!ctx || !step_dev) return SPLX_ERR_INVALID;
  CtxScope scope(ctx);
  return adam_all(ctx, p, g, m, v, hp, 0, step_dev, reinterpret_cast<cudaStream_t>(stream));
}

int splx_loss_l1(splx_ctx_t ctx, const float* img, const float* target, int64_t n,
                 float* loss_out, float* dL_dimg, splx_stream_t stream) {
  if (!ctx || !img || !target || !loss_out || n < 0) return SPLX_ERR_INVALID;
  CtxScope scope(ctx);
  launch_loss_l1(img, target, n, loss_out, dL_dimg, reinterpret_cast<cudaStream_t>(stream));
  CK_LAUNCH();
  return SPLX_OK;
}

int splx_loss_l1_dssim(splx_ctx_t ctx, const float* img, const float* target, int32_t width,
                       int32_t height, float lambda, float* loss_out, float* dL_dimg,
                       splx_stream_t stream) {
  if (!ctx || !img || !target || !loss_out || !dL_dimg || width < 1 || height < 1 ||
      !(lambda >= 0.0f) || !(lambda <= 1.0f))
    return SPLX_ERR_INVALID;
  CtxScope scope(ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const LossImgs L = make_loss_imgs(1, &width, &height);
  const size_t n = 3 * (size_t)width * height;
  float* maps = nullptr;
  double* sums = nullptr;
  int r;
  if ((r = ctx_alloc_t(ctx, &maps, 3 * n, s))) return r;
  if ((r = ctx_alloc_t(ctx, &sums, 2, s))) { ctx_free(ctx, maps, s); return r; }
  launch_loss_l1_dssim(L, img, target, lambda, maps, maps + n, maps + 2 * n, sums, loss_out,
                       dL_dimg, s);
  const cudaError_t e = cudaGetLastError();
  ctx_free(ctx, maps, s);
  ctx_free(ctx, sums, s);
  if (e != cudaSuccess) return cuda_fail(e, "loss_l1_dssim");
  return SPLX_OK;
}

// ---------------------------------------------------------------- batch
int splx_batch_create(splx_ctx_t ctx, const splx_gaussians* subsets, int32_t K,
                      const splx_camera* cams, int32_t V, const splx_opts* opts,
                      int64_t pair_capacity, splx_batch_t* out, splx_stream_t stream) {
  if (!ctx || !subsets || !cams || !out || K < 1 || K > kMaxK || V < 1 || V > kMaxViews ||
      pair_capacity < 0)
    return SPLX_ERR_INVALID;
  *out = nullptr;
  int r;
  if ((r = check_opts(opts))) return r;
  int64_t N = 0;
  for (int k = 0; k < K; ++k) {
    if ((r = check_gaussians(&subsets[k]))) return r;
    if (subsets[k].sh_degree != subsets[0].sh_degree) return SPLX_ERR_INVALID;
    N += subsets[k].n;
  }
  if (N >= (int64_t(1) << 32)) return SPLX_ERR_INVALID;
  for (int v = 0; v < V; ++v)
    if ((r = check_cam(&cams[v]))) return r;
  CtxScope scope(ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  splx_batch_s* bt = new (std::nothrow) splx_batch_s();
  if (!bt) return SPLX_ERR_BUDGET;
  Plan& P = bt->plan;
  P.ctx = ctx; P.V = V; P.K = K; P.deg = subsets[0].sh_degree; P.tile = opts->tile; P.N = N;
  P.opts = *opts;
  int64_t goff = 0;
  for (int k = 0; k < K; ++k) {
    P.subsets_h.push_back(make_subset(subsets[k], goff));
    goff += subsets[k].n;
  }
  for (int v = 0; v < V; ++v) P.views_h.push_back(make_view(cams[v], opts->tile));
  P.layout();
  const int64_t TP = P.total_pixels;
  auto fail = [&](int code) {
    P.release(s);
    ctx_free(ctx, bt->gCT, s);
    ctx_free(ctx, bt->partial, s);
    ctx_free(ctx, bt->last, s);
    if (bt->pinned_cams) cudaFreeHost(bt->pinned_cams);
    delete bt;
    return code;
  };
  if ((r = ctx_alloc_t(ctx, &bt->partial, (size_t)5 * K * TP, s))) return fail(r);
  if ((r = ctx_alloc_t(ctx, &bt->last, (size_t)K * TP, s))) return fail(r);
  if ((r = ctx_alloc_t(ctx, &bt->gCT, (size_t)K * TP, s))) return fail(r);
  // image (v, k): rgb planes at 3*(K*pix_off[v] + k*HW_v), T/D/last at K*pix_off[v] + k*HW_v
  float* rgb_base = bt->partial;
  float* T_base = bt->partial + (size_t)3 * K * TP;
  float* D_base = T_base + (size_t)K * TP;
  for (int v = 0; v < V; ++v) {
    const int64_t HW = (int64_t)P.views_h[v].W * P.views_h[v].H;
    for (int k = 0; k < K; ++k) {
      const int64_t o = (int64_t)K * P.pix_off[v] + (int64_t)k * HW;
      ImgDev im;
      im.rgb = rgb_base + 3 * o; im.T = T_base + o; im.D = D_base + o; im.last = bt->last + o;
      im.gCT = bt->gCT + o;
      P.imgs_h.push_back(im);
    }
  }
  if ((r = P.alloc_common(s))) return fail(r);
  if (V >= 2 && (r = P.alloc_split(s))) return fail(r);
  if ((r = P.alloc_select(s))) return fail(r);
  if ((r = ctx_alloc_t(ctx, &P.grad2d, (size_t)V * N * 3, s))) return fail(r);
  if ((r = ctx_alloc_t(ctx, &P.counters, kCounters, s))) return fail(r);
  if ((r = ctx_alloc_t(ctx, &P.work_ctr, 2, s))) return fail(r);
  if ((r = ctx_alloc_t(ctx, &P.omega, (size_t)4 * V * K, s))) return fail(r);
  P.visibility = true;
  cudaError_t e = cudaMemsetAsync(P.grad2d, 0, sizeof(float4) * 3 * (size_t)V * N, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.counters, 0, kCounters * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return fail(cuda_fail(e, "memset grad2d"));
  if (cudaMallocHost(&bt->pinned_cams, sizeof(splx_camera) * kMaxViews) != cudaSuccess)
    bt->pinned_cams = nullptr;
  int64_t cap = pair_capacity;
  if (cap == 0) {
    P.capacity = 0;
    if ((r = P.project_and_count(s))) return fail(r);
    uint64_t total = 0;
    if ((r = P.read_total(&total, s))) return fail(r);
    cap = (int64_t)(total + total / 4 + 1024);
  }
  if (cap >= (int64_t)UINT32_MAX) return fail(SPLX_ERR_CAPACITY);
  if ((r = P.alloc_pairs(cap, s))) return fail(r);
  *out = bt;
  return SPLX_OK;
}

int splx_batch_set_cameras(splx_batch_t bt, const splx_camera* cams, int32_t V, splx_stream_t stream) {
  if (!bt || !cams || V != bt->plan.V) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  for (int v = 0; v < V; ++v) {
    int r = check_cam(&cams[v]);
    if (r) return r;
    if (cams[v].width != P.views_h[v].W || cams[v].height != P.views_h[v].H) return SPLX_ERR_INVALID;
  }
  CtxScope scope(P.ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CK(cudaStreamSynchronize(s));
  for (int v = 0; v < V; ++v) P.views_h[v] = make_view(cams[v], P.tile);
  CK(cudaMemcpyAsync(P.views_d, P.views_h.data(), sizeof(ViewDev) * V, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return SPLX_OK;
}

int splx_batch_layout(splx_batch_t bt, int64_t* rgb_off, int64_t* pix_off) {
  if (!bt) return SPLX_ERR_INVALID;
  const Plan& P = bt->plan;
  for (int v = 0; v <= P.V; ++v) {
    if (rgb_off) rgb_off[v] = 3 * P.pix_off[v];
    if (pix_off) pix_off[v] = P.pix_off[v];
  }
  return SPLX_OK;
}

int splx_batch_forward(splx_batch_t bt, float* out_rgb, float* out_T, splx_stream_t stream) {
  if (!bt || !out_rgb) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int r;
  if ((r = P.bin(s))) return r;
  BatchDev b = P.dev();
  b.out_rgb = out_rgb;
  b.out_T = out_T;
  if (P.order_d && !P.stale()) {
    // saturation skipping: K waves, each sorting and rendering one subset of every view,
    // front to back
    if ((r = P.waves(b, s))) return r;
  } else {
    // (with a stale saturation state the rasteriser leaves the pruned pixels empty)
    launch_raster_fwd(b, s);
    launch_sort_retries(b, merge_rounds_bound(P.max_subset()), s);
    launch_raster_fwd_retry(b, s);
  }
  P.mark(5, s);
  launch_composite(b, P.total_pixels, s);
  if (P.stale()) launch_sat_update(b, P.order_d, P.total_pixels, s);
  P.mark(6, s);
  CK_LAUNCH();
  bt->forward_done = true;
  return SPLX_OK;
}

int splx_batch_backward(splx_batch_t bt, const float* dL_drgb, const float* dL_dT,
                        const splx_params* grads, splx_stream_t stream) {
  if (!bt || !dL_drgb || !grads) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  if (!bt->forward_done) return SPLX_ERR_STATE;
  GradTable gt;
  std::memset(&gt, 0, sizeof(gt));
  for (int k = 0; k < P.K; ++k) {
    if (P.subsets_h[k].n > 0 && (!grads[k].means || !grads[k].log_scales || !grads[k].quats ||
                                 !grads[k].opacity_logits || !grads[k].sh || !aligned16(grads[k].quats)))
      return SPLX_ERR_INVALID;
    gt.p[k][0] = grads[k].means; gt.p[k][1] = grads[k].log_scales; gt.p[k][2] = grads[k].quats;
    gt.p[k][3] = grads[k].opacity_logits; gt.p[k][4] = grads[k].sh;
  }
  CtxScope scope(P.ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  BatchDev b = P.dev();
  b.dL_drgb = dL_drgb;
  b.dL_dT = dL_dT;
  P.mark(7, s);
  launch_composite_bwd(b, P.total_pixels, s);
  P.mark(8, s);
  launch_raster_bwd(b, s);
  P.mark(9, s);
  launch_project_bwd(b, gt, s);
  P.mark(10, s);
  CK_LAUNCH();
  return SPLX_OK;
}

int splx_batch_backward_adam(splx_batch_t bt, const float* dL_drgb, const float* dL_dT,
                             const splx_params* params, const splx_params* m,
                             const splx_params* v, const splx_adam* hp, int64_t* step_dev,
                             splx_stream_t stream) {
  if (!bt || !dL_drgb || !params || !m || !v || !hp || !step_dev) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  if (!bt->forward_done) return SPLX_ERR_STATE;
  AdamTable at;
  std::memset(&at, 0, sizeof(at));
  for (int k = 0; k < P.K; ++k) {
    const SubsetDev& S = P.subsets_h[k];
    if (S.n == 0) continue;
    const splx_params* t[3] = {&params[k], &m[k], &v[k]};
    for (int j = 0; j < 3; ++j) {
      const splx_params& q = *t[j];
      if (q.n != S.n || q.sh_degree != P.deg || !q.means || !q.log_scales || !q.quats ||
          !q.opacity_logits || !q.sh)
        return SPLX_ERR_INVALID;
    }
    // the adjoint reads the batch's own parameter arrays, which this call then updates
    const splx_params& q = params[k];
    if (q.means != S.means || q.log_scales != S.log_scales || q.quats != S.quats ||
        q.opacity_logits != S.opacity_logits || q.sh != S.sh)
      return SPLX_ERR_INVALID;
    for (int j = 0; j < 3; ++j) {
      const splx_params& r = *t[j];
      float** dst = j == 0 ? at.p[k] : j == 1 ? at.m[k] : at.v[k];
      dst[0] = r.means; dst[1] = r.log_scales; dst[2] = r.quats;
      dst[3] = r.opacity_logits; dst[4] = r.sh;
    }
  }
  for (int j = 0; j < 6; ++j) at.lr[j] = hp->lr[j];
  at.b1 = hp->beta1;
  at.b2 = hp->beta2;
  at.eps = hp->eps;
  at.step_dev = step_dev;
  CtxScope scope(P.ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!P.defer) {
    int r = ctx_alloc_t(P.ctx, &P.defer, (size_t)std::max<int64_t>((P.N + 127) / 128, 1), s);
    if (r) return r;
  }
  at.defer = P.defer;
  BatchDev b = P.dev();
  b.dL_drgb = dL_drgb;
  b.dL_dT = dL_dT;
  P.mark(7, s);
  launch_composite_bwd(b, P.total_pixels, s);
  P.mark(8, s);
  launch_raster_bwd(b, s);
  P.mark(9, s);
  launch_project_bwd_adam(b, at, s);
  P.mark(10, s);
  CK_LAUNCH();
  return SPLX_OK;
}

int splx_batch_set_timing(splx_batch_t bt, int enable) {
  if (!bt) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  if (enable) {
    for (auto& e : P.ev)
      if (!e) CK(cudaEventCreate(&e));
    if (P.wev.empty()) {
      P.wev.assign(2 * P.K + 1, nullptr);
      for (auto& e : P.wev) CK(cudaEventCreate(&e));
    }
  }
  P.timing = enable != 0;
  return SPLX_OK;
}

int splx_batch_set_launch(splx_batch_t bt, int32_t raster_ctas_per_sm) {
  if (!bt || raster_ctas_per_sm < 0 || raster_ctas_per_sm > 64) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P.ctx->device));
  P.persist_grid = raster_ctas_per_sm * sms;
  return SPLX_OK;
}

int splx_batch_loss_l1_dssim(splx_batch_t bt, const float* rgb, const float* target, float lambda,
                             float* loss_out, float* dL_drgb, splx_stream_t stream) {
  if (!bt || !rgb || !target || !loss_out || !dL_drgb || !(lambda >= 0.0f) || !(lambda <= 1.0f))
    return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<int> W(P.V), H(P.V);
  for (int v = 0; v < P.V; ++v) { W[v] = P.views_h[v].W; H[v] = P.views_h[v].H; }
  const LossImgs L = make_loss_imgs(P.V, W.data(), H.data());
  const size_t n = 3 * (size_t)P.total_pixels;
  int r;
  if (!bt->ssim_maps) {
    if (stream_capturing(s)) return SPLX_ERR_STATE;  // allocate in an eager call first
    if ((r = ctx_alloc_t(P.ctx, &bt->ssim_maps, 3 * n, s))) return r;
    if ((r = ctx_alloc_t(P.ctx, &bt->ssim_sums, 2, s))) return r;
  }
  launch_loss_l1_dssim(L, rgb, target, lambda, bt->ssim_maps, bt->ssim_maps + n,
                       bt->ssim_maps + 2 * n, bt->ssim_sums, loss_out, dL_drgb, s);
  CK_LAUNCH();
  return SPLX_OK;
}

int splx_batch_set_visibility(splx_batch_t bt, int32_t enable) {
  if (!bt || !bt->plan.omega) return SPLX_ERR_INVALID;
  bt->plan.visibility = enable != 0;
  return SPLX_OK;
}

int splx_batch_set_prefix_sort(splx_batch_t bt, int32_t enable) {
  if (!bt || !bt->plan.sel) return SPLX_ERR_INVALID;
  bt->plan.select_prefix = enable != 0;
  return SPLX_OK;
}

int splx_batch_tune_prefix_sort(splx_batch_t bt, splx_stream_t stream) {
  if (!bt || !bt->plan.sel) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  if (!P.select_prefix || !P.counters) return SPLX_OK;
  CtxScope scope(P.ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long c[kCounters] = {};
  CK(cudaMemcpyAsync(c, P.counters, sizeof(c), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // counters[8]: items walked on a selected prefix, [9]: items handed to the whole sort
  if (c[8] > 0 && 4 * c[9] > c[8]) P.select_prefix = false;
  return SPLX_OK;
}

int splx_batch_set_order(splx_batch_t bt, const int32_t* order) {
  if (!bt) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  if (!order) {
    P.free_ptr((void*&)P.order_d, nullptr);
    P.free_ptr((void*&)P.rank_d, nullptr);
    P.free_ptr((void*&)P.sat_d, nullptr);
    P.free_ptr((void*&)P.tpre, nullptr);
    return SPLX_OK;
  }
  for (int v = 0; v < P.V; ++v) {
    std::vector<int> seen(P.K, 0);
    for (int r = 0; r < P.K; ++r) {
      const int k = order[v * P.K + r];
      if (k < 0 || k >= P.K || seen[k]++) return SPLX_ERR_INVALID;
    }
  }
  int r;
  if (!P.order_d && (r = ctx_alloc_t(P.ctx, &P.order_d, (size_t)P.V * P.K, nullptr))) return r;
  if (!P.rank_d && (r = ctx_alloc_t(P.ctx, &P.rank_d, (size_t)P.V * P.K, nullptr))) {
    P.free_ptr((void*&)P.order_d, nullptr);
    return r;
  }
  if (!P.tpre &&
      (r = ctx_alloc_t(P.ctx, &P.tpre, (size_t)std::max<int64_t>(P.total_pixels, 1), nullptr))) {
    P.free_ptr((void*&)P.order_d, nullptr);
    P.free_ptr((void*&)P.rank_d, nullptr);
    return r;
  }
  std::vector<int32_t> rank((size_t)P.V * P.K);
  for (int v = 0; v < P.V; ++v)
    for (int q = 0; q < P.K; ++q) rank[(size_t)v * P.K + order[v * P.K + q]] = q;
  CK(cudaMemcpy(P.order_d, order, sizeof(int32_t) * P.V * P.K, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P.rank_d, rank.data(), sizeof(int32_t) * P.V * P.K, cudaMemcpyHostToDevice));
  return SPLX_OK;
}

int splx_batch_set_stale(splx_batch_t bt, uint8_t* const* sat) {
  if (!bt) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  if (!sat) {
    P.free_ptr((void*&)P.sat_d, nullptr);
    return SPLX_OK;
  }
  if (!P.order_d) return SPLX_ERR_STATE;
  for (int v = 0; v < P.V; ++v)
    if (!sat[v]) return SPLX_ERR_INVALID;
  int r;
  if (!P.sat_d && (r = ctx_alloc_t(P.ctx, &P.sat_d, (size_t)P.V, nullptr))) return r;
  CK(cudaMemcpy(P.sat_d, sat, sizeof(uint8_t*) * P.V, cudaMemcpyHostToDevice));
  return SPLX_OK;
}

int splx_batch_set_cross_filter(splx_batch_t bt, const float* cells) {
  if (!bt) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  if (!cells) {
    P.cross_filter = false;
    return SPLX_OK;
  }
  for (int i = 0; i < 6 * P.K; ++i)
    if (std::isnan(cells[i])) return SPLX_ERR_INVALID;
  int r;
  if (!P.cells_d && (r = ctx_alloc_t(P.ctx, &P.cells_d, (size_t)6 * P.K, nullptr))) return r;
  if (!P.cross && (r = ctx_alloc_t(P.ctx, &P.cross, (size_t)std::max<int64_t>(P.N, 1), nullptr)))
    return r;
  if (!P.zr && (r = ctx_alloc_t(P.ctx, &P.zr, (size_t)2 * P.V * P.K, nullptr))) return r;
  if (!P.removed &&
      (r = ctx_alloc_t(P.ctx, &P.removed, (size_t)std::max<int64_t>(P.n_tiles, 1), nullptr)))
    return r;
  CK(cudaMemcpy(P.cells_d, cells, sizeof(float) * 6 * P.K, cudaMemcpyHostToDevice));
  P.cross_filter = true;
  P.visibility = true;
  return SPLX_OK;
}

int splx_batch_max_ctas_per_sm(splx_batch_t bt, int32_t* fwd, int32_t* bwd) {
  if (!bt || !fwd || !bwd) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  *fwd = raster_max_ctas_per_sm(P.tile, false);
  *bwd = raster_max_ctas_per_sm(P.tile, true);
  if (*fwd <= 0 || *bwd <= 0) return SPLX_ERR_CUDA;
  return SPLX_OK;
}

// Per-kernel times from the batch's timing events, each mapped through the graph's ring
// slot (no graph: the events themselves).
static int kernel_times_of(const Plan& P, const splx_graph_s* g, int slot, float* ms_out) {
  auto E = [&](cudaEvent_t e) { return g ? g->in_slot(e, slot) : e; };
  CK(cudaEventSynchronize(E(P.ev[10])));
  const int pairs[9][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}, {5, 6},
                           {7, 8}, {8, 9}, {9, 10}};
  for (int i = 0; i < 9; ++i) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, E(P.ev[pairs[i][0]]), E(P.ev[pairs[i][1]])));
    ms_out[i] = ms;
  }
  if (P.order_d && !P.stale() && (int)P.wev.size() == 2 * P.K + 1) {
    // waves interleave sort and rasteriser: sum each over the waves
    float sort = 0.0f, ras = 0.0f;
    for (int r = 0; r < P.K; ++r) {
      float a = 0.0f, c = 0.0f;
      CK(cudaEventElapsedTime(&a, E(P.wev[2 * r]), E(P.wev[2 * r + 1])));
      CK(cudaEventElapsedTime(&c, E(P.wev[2 * r + 1]), E(P.wev[2 * r + 2])));
      sort += a;
      ras += c;
    }
    ms_out[3] += sort;
    ms_out[4] = ras;
  }
  return SPLX_OK;
}

int splx_batch_kernel_times(splx_batch_t bt, float* ms_out) {
  if (!bt || !ms_out) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  if (!P.timing) return SPLX_ERR_STATE;
  CtxScope scope(P.ctx);
  return kernel_times_of(P, nullptr, -1, ms_out);
}

int splx_batch_kernel_times_slot(splx_batch_t bt, splx_graph_t g, int32_t slot, float* ms_out) {
  if (!bt || !g || !ms_out || slot < 0 || slot >= g->slots) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  if (!P.timing) return SPLX_ERR_STATE;
  CtxScope scope(P.ctx);
  return kernel_times_of(P, g, slot, ms_out);
}

int splx_batch_counters(splx_batch_t bt, int64_t* out, splx_stream_t stream) {
  if (!bt || !out) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long c[kCounters] = {};  // host copy of the device counters
  uint32_t total = 0;
  CK(cudaMemcpyAsync(c, P.counters, sizeof(c), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&total, P.tile_start + P.n_tiles, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  out[0] = (int64_t)total;
  for (int i = 0; i < kCounters; ++i) out[1 + i] = (int64_t)c[i];
  return SPLX_OK;
}

int splx_batch_visible(splx_batch_t bt, int64_t* visible_out, splx_stream_t stream) {
  if (!bt || !visible_out) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* d = nullptr;
  int r;
  if ((r = ctx_alloc_t(P.ctx, &d, 1, s))) return r;
  unsigned long long h = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(h), s);
  if (e == cudaSuccess) {
    count_nonzero_u32(P.counts, (int64_t)P.V * P.N, d, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  ctx_free(P.ctx, (void*)d, s);
  if (e != cudaSuccess) return cuda_fail(e, "splx_batch_visible");
  *visible_out = (int64_t)h;
  return SPLX_OK;
}

int splx_batch_status(splx_batch_t bt, int64_t* pairs_out, splx_stream_t stream) {
  if (!bt) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t total = 0;
  int st = 0;
  CK(cudaMemcpyAsync(&total, P.tile_start + P.n_tiles, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&st, P.ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (pairs_out) *pairs_out = (int64_t)total;
  if (st & ST_CAPACITY || total > (uint64_t)P.capacity) return SPLX_ERR_CAPACITY;
  if (st & ST_TIMEOUT) return SPLX_ERR_TIMEOUT;
  return SPLX_OK;
}

int splx_batch_destroy(splx_batch_t bt) {
  if (!bt) return SPLX_ERR_INVALID;
  Plan& P = bt->plan;
  CtxScope scope(P.ctx);
  cudaDeviceSynchronize();
  P.release(nullptr);
  ctx_free(P.ctx, bt->gCT, nullptr);
  ctx_free(P.ctx, bt->partial, nullptr);
  ctx_free(P.ctx, bt->last, nullptr);
  ctx_free(P.ctx, bt->ssim_maps, nullptr);
  ctx_free(P.ctx, bt->ssim_sums, nullptr);
  cudaDeviceSynchronize();
  if (bt->pinned_cams) cudaFreeHost(bt->pinned_cams);
  delete bt;
  return SPLX_OK;
}

// ---------------------------------------------------------------- serving
namespace {

struct SrvReq {
  int64_t id;
  splx_camera cam;
  float* out;  // device [3][H][W], caller-owned
  bool has_order = false;
  int32_t order[kMaxK];  // front-to-back subset order (saturation skipping)
};

// One launch of a server slot: the views of up to max_views requests x K subsets, on the
// slot's own stream.  Phase 1 = projected, waiting for the pair count (copied to pinned
// memory behind an event); phase 2 = binned, rendered, composited and copied out.
struct SrvLaunch {
  int phase = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  // device timeline of the launch: before its first kernel, after its projection and tile
  // counts (the pair count's copy), after its last copy-out
  cudaEvent_t t_begin = nullptr, t_counted = nullptr, t_end = nullptr;
  uint32_t* total_h = nullptr;
  Plan P;
  float* partial = nullptr;
  int32_t* last = nullptr;
  float* out_cat = nullptr;
  std::vector<SrvReq> reqs;
  size_t reserved = 0;
};

}  // namespace

struct splx_server_s {
  splx_ctx_t ctx = nullptr;
  std::vector<splx_gaussians> subsets;
  int64_t N = 0;
  splx_opts opts{};
  size_t budget = 0, reserved = 0;
  int max_views = 1;
  double pairs_per_px = 32.0;  // admission estimate; raised to the largest count seen
  int64_t next_id = 0;
  std::deque<SrvReq> pending;
  std::vector<SrvLaunch> slots;
  std::deque<std::pair<int64_t, int>> finished;  // (request id, status) not yet reported
  // per finished request: its launch's begin / counted / end times in ms after `epoch`
  // (the most recent kTimesKept requests)
  cudaEvent_t epoch = nullptr;
  std::unordered_map<int64_t, std::array<float, 3>> times;
  std::deque<int64_t> times_order;
};

namespace {

// Device bytes one launch holds: records and tile counts per (view, Gaussian), the K
// partial planes and the composited views, per-tile arrays, and the pair buffers.
size_t launch_bytes(const splx_server_s& S, const std::vector<SrvReq>& reqs, double pairs) {
  const int K = (int)S.subsets.size();
  int64_t px = 0, tiles = 0;
  for (const SrvReq& r : reqs) {
    px += (int64_t)r.cam.width * r.cam.height;
    tiles += (int64_t)K * ((r.cam.width + S.opts.tile - 1) / S.opts.tile) *
             ((r.cam.height + S.opts.tile - 1) / S.opts.tile);
  }
  const double b = (double)reqs.size() * S.N * (sizeof(Rec) + 4) + (double)px * K * 24.0 +
                   (double)px * 16.0 + (double)tiles * 48.0 + pairs * 16.0 +
                   (pairs / 2048.0 + 1.0) * 8.0 + 65536.0;
  return (size_t)b;
}

constexpr size_t kTimesKept = 1 << 16;

int64_t launch_pixels(const std::vector<SrvReq>& reqs) {
  int64_t px = 0;
  for (const SrvReq& r : reqs) px += (int64_t)r.cam.width * r.cam.height;
  return px;
}

void srv_free_launch(splx_server_s* S, SrvLaunch& L) {
  L.P.release(L.s);
  ctx_free(S->ctx, L.partial, L.s);
  ctx_free(S->ctx, L.last, L.s);
  ctx_free(S->ctx, L.out_cat, L.s);
  L.partial = nullptr; L.last = nullptr; L.out_cat = nullptr;
  S->reserved -= std::min(S->reserved, L.reserved);
  L.reserved = 0;
  L.phase = 0;
  L.reqs.clear();
  Plan fresh;
  L.P = fresh;
}

void srv_fail_launch(splx_server_s* S, SrvLaunch& L, int code) {
  for (const SrvReq& r : L.reqs) S->finished.emplace_back(r.id, code);
  srv_free_launch(S, L);
}

// Plans the launch and enqueues projection + tile counting + scan and the copy of the
// pair count; returns an error code (the caller fails the launch's requests).
int srv_start(splx_server_s* S, SrvLaunch& L) {
  Plan& P = L.P;
  const int K = (int)S->subsets.size();
  const int V = (int)L.reqs.size();
  CK(cudaEventRecord(L.t_begin, L.s));
  P.ctx = S->ctx; P.V = V; P.K = K; P.deg = S->subsets[0].sh_degree; P.tile = S->opts.tile;
  P.N = S->N; P.opts = S->opts;
  int64_t goff = 0;
  for (int k = 0; k < K; ++k) {
    P.subsets_h.push_back(make_subset(S->subsets[k], goff));
    goff += S->subsets[k].n;
  }
  for (int v = 0; v < V; ++v) P.views_h.push_back(make_view(L.reqs[v].cam, S->opts.tile));
  P.layout();
  const int64_t TP = P.total_pixels;
  int r;
  if ((r = ctx_alloc_t(S->ctx, &L.partial, (size_t)5 * K * TP, L.s))) return r;
  if ((r = ctx_alloc_t(S->ctx, &L.last, (size_t)K * TP, L.s))) return r;
  if ((r = ctx_alloc_t(S->ctx, &L.out_cat, (size_t)3 * TP, L.s))) return r;
  float* rgb_base = L.partial;
  float* T_base = L.partial + (size_t)3 * K * TP;
  float* D_base = T_base + (size_t)K * TP;
  for (int v = 0; v < V; ++v) {
    const int64_t HW = (int64_t)P.views_h[v].W * P.views_h[v].H;
    for (int k = 0; k < K; ++k) {
      const int64_t o = (int64_t)K * P.pix_off[v] + (int64_t)k * HW;
      ImgDev im;
      im.rgb = rgb_base + 3 * o; im.T = T_base + o; im.D = D_base + o; im.last = L.last + o;
      im.gCT = nullptr;
      P.imgs_h.push_back(im);
    }
  }
  if ((r = P.alloc_common(L.s))) return r;
  if ((r = ctx_alloc_t(S->ctx, &P.omega, (size_t)4 * V * K, L.s))) return r;
  P.visibility = true;
  bool ordered = true;
  for (const SrvReq& q : L.reqs) ordered = ordered && q.has_order;
  if (ordered) {  // saturation skipping for the launch: per-view orders, prefix buffer
    std::vector<int32_t> ord((size_t)V * K);
    for (int v = 0; v < V; ++v)
      for (int k = 0; k < K; ++k) ord[(size_t)v * K + k] = L.reqs[v].order[k];
    if ((r = ctx_alloc_t(S->ctx, &P.order_d, ord.size(), L.s))) return r;
    if ((r = ctx_alloc_t(S->ctx, &P.tpre, (size_t)std::max<int64_t>(TP, 1), L.s))) return r;
    CK(cudaMemcpyAsync(P.order_d, ord.data(), sizeof(int32_t) * ord.size(),
                       cudaMemcpyHostToDevice, L.s));
  }
  if ((r = P.project_and_count(L.s))) return r;
  CK(cudaMemcpyAsync(L.total_h, P.tile_start + P.n_tiles, sizeof(uint32_t),
                     cudaMemcpyDeviceToHost, L.s));
  CK(cudaEventRecord(L.t_counted, L.s));
  CK(cudaEventRecord(L.ev, L.s));
  L.phase = 1;
  return SPLX_OK;
}

// Binning, local render, composition and the copies into the requests' buffers.
int srv_render(splx_server_s* S, SrvLaunch& L, uint64_t total) {
  Plan& P = L.P;
  int r;
  if (total >= (uint64_t)UINT32_MAX) return SPLX_ERR_CAPACITY;
  if ((r = P.alloc_pairs((int64_t)total, L.s))) return r;
  if ((r = P.fill_and_sort(L.s))) return r;
  BatchDev b = P.dev();
  b.out_rgb = L.out_cat;
  b.out_T = nullptr;
  if (P.order_d) {
    if ((r = P.waves(b, L.s))) return r;
  } else {
    launch_raster_fwd(b, L.s);
  }
  launch_composite(b, P.total_pixels, L.s);
  CK_LAUNCH();
  for (int v = 0; v < P.V; ++v) {
    const size_t bytes = sizeof(float) * 3 * (size_t)P.views_h[v].W * P.views_h[v].H;
    CK(cudaMemcpyAsync(L.reqs[v].out, L.out_cat + 3 * P.pix_off[v], bytes,
                       cudaMemcpyDeviceToDevice, L.s));
  }
  CK(cudaEventRecord(L.t_end, L.s));
  CK(cudaEventRecord(L.ev, L.s));
  L.phase = 2;
  return SPLX_OK;
}

bool srv_any_inflight(const splx_server_s* S) {
  for (const SrvLaunch& L : S->slots)
    if (L.phase != 0) return true;
  return false;
}

// One scheduling pass: retire finished launches, move counted launches on to rendering
// once their pair buffers fit the budget, then admit pending requests into idle slots.
int srv_advance(splx_server_s* S) {
  for (SrvLaunch& L : S->slots) {
    if (L.phase == 0) continue;
    const cudaError_t q = cudaEventQuery(L.ev);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) {
      srv_fail_launch(S, L, cuda_fail(q, "server launch"));
      continue;
    }
    if (L.phase == 2) {
      std::array<float, 3> t = {0.0f, 0.0f, 0.0f};
      cudaEvent_t marks[3] = {L.t_begin, L.t_counted, L.t_end};
      for (int i = 0; i < 3; ++i)
        if (cudaEventElapsedTime(&t[i], S->epoch, marks[i]) != cudaSuccess) t[i] = -1.0f;
      for (const SrvReq& r : L.reqs) {
        S->finished.emplace_back(r.id, SPLX_OK);
        S->times[r.id] = t;
        S->times_order.push_back(r.id);
        if (S->times_order.size() > kTimesKept) {
          S->times.erase(S->times_order.front());
          S->times_order.pop_front();
        }
      }
      srv_free_launch(S, L);
      continue;
    }
    // phase 1: the pair count is known; re-reserve with it and render if it fits.  If it
    // does not: wait while a rendering launch will free memory; fail if this launch is
    // alone; otherwise (only other counted launches hold memory) give its requests back
    // to the head of the queue, so no two launches wait on each other.
    const uint64_t total = *L.total_h;
    const int64_t px = launch_pixels(L.reqs);
    if (px > 0) S->pairs_per_px = std::max(S->pairs_per_px, (double)total / (double)px);
    const size_t need = launch_bytes(*S, L.reqs, (double)total);
    const size_t others = S->reserved - std::min(S->reserved, L.reserved);
    if (others + need > S->budget) {
      bool rendering = false, alone = true;
      for (const SrvLaunch& o : S->slots) {
        if (&o == &L || o.phase == 0) continue;
        alone = false;
        if (o.phase == 2) rendering = true;
      }
      if (rendering) continue;
      if (alone) {
        srv_fail_launch(S, L, SPLX_ERR_BUDGET);
      } else {
        for (auto it = L.reqs.rbegin(); it != L.reqs.rend(); ++it) S->pending.push_front(*it);
        L.reqs.clear();
        srv_free_launch(S, L);
      }
      continue;
    }
    S->reserved = others + need;
    L.reserved = need;
    const int r = srv_render(S, L, total);
    if (r) srv_fail_launch(S, L, r);
  }
  for (SrvLaunch& L : S->slots) {
    if (L.phase != 0 || S->pending.empty()) continue;
    std::vector<SrvReq> take;
    size_t bytes = 0;
    while (!S->pending.empty() && (int)take.size() < S->max_views) {
      take.push_back(S->pending.front());
      const size_t b = launch_bytes(*S, take, S->pairs_per_px * launch_pixels(take));
      if (S->reserved + b > S->budget) {
        take.pop_back();
        break;
      }
      bytes = b;
      S->pending.pop_front();
    }
    if (take.empty()) {
      if (srv_any_inflight(S)) break;  // wait for memory to free up
      // nothing in flight: the estimate alone never rejects a request.  Admit the oldest
      // if its footprint without pair buffers fits; its exact pair count decides later.
      take.push_back(S->pending.front());
      S->pending.pop_front();
      bytes = launch_bytes(*S, take, 0.0);
      if (S->reserved + bytes > S->budget) {
        S->finished.emplace_back(take[0].id, SPLX_ERR_BUDGET);
        continue;
      }
    }
    L.reqs = std::move(take);
    L.reserved = bytes;
    S->reserved += bytes;
    const int r = srv_start(S, L);
    if (r) srv_fail_launch(S, L, r);
  }
  return SPLX_OK;
}

}  // namespace

int splx_server_create(splx_ctx_t ctx, const splx_gaussians* subsets, int32_t K,
                       const splx_opts* opts, size_t hbm_budget_bytes, int32_t slots,
                       int32_t max_views, splx_server_t* out) {
  if (!ctx || !subsets || !out || K < 1 || K > kMaxK || slots < 1 || slots > 16 ||
      max_views < 1 || max_views > kMaxViews || hbm_budget_bytes == 0)
    return SPLX_ERR_INVALID;
  *out = nullptr;
  int r;
  if ((r = check_opts(opts))) return r;
  int64_t N = 0;
  for (int k = 0; k < K; ++k) {
    if ((r = check_gaussians(&subsets[k]))) return r;
    if (subsets[k].sh_degree != subsets[0].sh_degree) return SPLX_ERR_INVALID;
    N += subsets[k].n;
  }
  if (N >= (int64_t(1) << 32)) return SPLX_ERR_INVALID;
  CtxScope scope(ctx);
  splx_server_s* S = new (std::nothrow) splx_server_s();
  if (!S) return SPLX_ERR_BUDGET;
  S->ctx = ctx;
  S->subsets.assign(subsets, subsets + K);
  S->N = N;
  S->opts = *opts;
  S->budget = hbm_budget_bytes;
  S->max_views = max_views;
  S->slots.resize((size_t)slots);
  cudaError_t e = cudaSuccess;
  for (SrvLaunch& L : S->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&L.t_begin);
    if (e == cudaSuccess) e = cudaEventCreate(&L.t_counted);
    if (e == cudaSuccess) e = cudaEventCreate(&L.t_end);
    if (e == cudaSuccess) e = cudaMallocHost(&L.total_h, sizeof(uint32_t));
  }
  if (e == cudaSuccess) e = cudaEventCreate(&S->epoch);
  if (e == cudaSuccess) e = cudaEventRecord(S->epoch, S->slots[0].s);
  if (e != cudaSuccess) {
    splx_server_destroy(S);
    return cuda_fail(e, "splx_server_create");
  }
  *out = S;
  return SPLX_OK;
}

int splx_server_submit(splx_server_t S, const splx_camera* cam, const int32_t* order,
                       float* out_rgb, int64_t* id_out) {
  if (!S || !out_rgb || !id_out) return SPLX_ERR_INVALID;
  int r;
  if ((r = check_cam(cam))) return r;
  SrvReq q;
  const int K = (int)S->subsets.size();
  if (order) {
    std::vector<int> seen(K, 0);
    for (int k = 0; k < K; ++k)
      if (order[k] < 0 || order[k] >= K || seen[order[k]]++) return SPLX_ERR_INVALID;
    std::memcpy(q.order, order, sizeof(int32_t) * K);
    q.has_order = true;
  }
  q.id = S->next_id++;
  q.cam = *cam;
  q.out = out_rgb;
  S->pending.push_back(q);
  *id_out = q.id;
  CtxScope scope(S->ctx);
  return srv_advance(S);
}

int splx_server_poll(splx_server_t S, int64_t* ids, int32_t* status, int32_t cap, int32_t* n_out) {
  if (!S || !n_out || cap < 0 || (cap > 0 && (!ids || !status))) return SPLX_ERR_INVALID;
  CtxScope scope(S->ctx);
  int r = srv_advance(S);
  int n = 0;
  while (n < cap && !S->finished.empty()) {
    ids[n] = S->finished.front().first;
    status[n] = S->finished.front().second;
    S->finished.pop_front();
    ++n;
  }
  *n_out = n;
  return r;
}

int splx_server_stats(splx_server_t S, int32_t* queued, int32_t* inflight, size_t* reserved) {
  if (!S) return SPLX_ERR_INVALID;
  int n = 0;
  for (const SrvLaunch& L : S->slots)
    if (L.phase != 0) n += (int)L.reqs.size();
  if (queued) *queued = (int32_t)S->pending.size();
  if (inflight) *inflight = n;
  if (reserved) *reserved = S->reserved;
  return SPLX_OK;
}

int splx_server_destroy(splx_server_t S) {
  if (!S) return SPLX_ERR_INVALID;
  CtxScope scope(S->ctx);
  for (SrvLaunch& L : S->slots) {
    if (L.s) cudaStreamSynchronize(L.s);
    if (L.phase != 0) srv_free_launch(S, L);
    if (L.s) cudaStreamSynchronize(L.s);
    if (L.s) cudaStreamDestroy(L.s);
    if (L.ev) cudaEventDestroy(L.ev);
    for (cudaEvent_t t : {L.t_begin, L.t_counted, L.t_end})
      if (t) cudaEventDestroy(t);
    if (L.total_h) cudaFreeHost(L.total_h);
  }
  if (S->epoch) cudaEventDestroy(S->epoch);
  delete S;
  return SPLX_OK;
}

int splx_server_request_times(splx_server_t S, int64_t id, float* times_ms) {
  if (!S || !times_ms) return SPLX_ERR_INVALID;
  auto it = S->times.find(id);
  if (it == S->times.end()) return SPLX_ERR_INVALID;
  for (int i = 0; i < 3; ++i) times_ms[i] = it->second[i];
  return SPLX_OK;
}

// ---------------------------------------------------------------- graphs
int splx_graph_begin(splx_ctx_t ctx, splx_stream_t stream) {
  if (!ctx || !stream) return SPLX_ERR_INVALID;
  CtxScope scope(ctx);
  CK(cudaStreamBeginCapture(reinterpret_cast<cudaStream_t>(stream), cudaStreamCaptureModeThreadLocal));
  return SPLX_OK;
}

int splx_graph_end(splx_ctx_t ctx, splx_stream_t stream, splx_graph_t* out) {
  if (!ctx || !stream || !out) return SPLX_ERR_INVALID;
  CtxScope scope(ctx);
  splx_graph_s* g = new (std::nothrow) splx_graph_s();
  if (!g) return SPLX_ERR_BUDGET;
  cudaError_t e = cudaStreamEndCapture(reinterpret_cast<cudaStream_t>(stream), &g->graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) {
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return cuda_fail(e, "graph capture");
  }
  *out = g;
  return SPLX_OK;
}

int splx_graph_launch(splx_graph_t g, splx_stream_t stream) {
  if (!g) return SPLX_ERR_INVALID;
  if (g->slots > 0) {
    // this launch records its timing events into the next ring slot
    const int slot = g->next;
    g->next = (g->next + 1) % g->slots;
    const size_t n = g->ev_nodes.size();
    for (size_t k = 0; k < n; ++k)
      CK(cudaGraphExecEventRecordNodeSetEvent(g->exec, g->ev_nodes[k], g->ring[(size_t)slot * n + k]));
  }
  CK(cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)));
  return SPLX_OK;
}

int splx_graph_set_timing_ring(splx_graph_t g, int32_t slots) {
  if (!g || slots < 0 || slots > 4096) return SPLX_ERR_INVALID;
  // the executable graph's event nodes go back to their captured events before the ring's
  // events are destroyed (a later launch must not record into a destroyed event)
  // (an event still pending in a launch in flight is released once it completes)
  if (!g->ring.empty()) {
    for (size_t k = 0; k < g->ev_nodes.size(); ++k)
      CK(cudaGraphExecEventRecordNodeSetEvent(g->exec, g->ev_nodes[k], g->ev_orig[k]));
  }
  for (cudaEvent_t e : g->ring) cudaEventDestroy(e);
  g->ring.clear();
  g->ev_nodes.clear();
  g->ev_orig.clear();
  g->slots = 0;
  g->next = 0;
  if (slots == 0) return SPLX_OK;
  size_t n = 0;
  CK(cudaGraphGetNodes(g->graph, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) CK(cudaGraphGetNodes(g->graph, nodes.data(), &n));
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nd, &t));
    if (t != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t e = nullptr;
    CK(cudaGraphEventRecordNodeGetEvent(nd, &e));
    g->ev_nodes.push_back(nd);
    g->ev_orig.push_back(e);
  }
  g->ring.assign((size_t)slots * g->ev_nodes.size(), nullptr);
  for (auto& e : g->ring) CK(cudaEventCreate(&e));
  g->slots = slots;
  return SPLX_OK;
}

int splx_graph_destroy(splx_graph_t g) {
  if (!g) return SPLX_ERR_INVALID;
  for (cudaEvent_t e : g->ring) cudaEventDestroy(e);
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
  return SPLX_OK;
}

// ---------------------------------------------------------------- diagnostics
int splx_device_status(splx_ctx_t ctx, splx_stream_t stream) {
  if (!ctx) return SPLX_ERR_INVALID;
  CtxScope scope(ctx);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int st = 0;
  CK(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s));
  CK(cudaStreamSynchronize(s));
  if (st & ST_CAPACITY) return SPLX_ERR_CAPACITY;
  if (st & ST_TIMEOUT) return SPLX_ERR_TIMEOUT;
  if (st & ST_BOUNDS) return SPLX_ERR_STATE;
  return SPLX_OK;
}

const char* splx_strerror(int st) {
  switch (st) {
    case SPLX_OK: return "ok";
    case SPLX_ERR_INVALID: return "invalid argument";
    case SPLX_ERR_BUDGET: return "HBM budget exceeded";
    case SPLX_ERR_CAPACITY: return "pair capacity exceeded";
    case SPLX_ERR_CUDA: return "CUDA error";
    case SPLX_ERR_TIMEOUT: return "bounded device wait timed out";
    case SPLX_ERR_STATE: return "object in wrong state";
    default: return "unknown status";
  }
}

const char* splx_last_cuda_error(void) { return g_cuda_err; }

int64_t splx_launch_count(splx_ctx_t ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
