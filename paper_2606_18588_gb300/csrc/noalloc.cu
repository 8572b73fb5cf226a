// Allocation-free variant of splx_render_partial (declared in include/splx.h).
//
// Some callers cannot allocate device memory: a process whose HBM is reserved up front
// by another allocator (an inference server's arena, a framework's caching allocator
// that already holds the device), or a latency-critical loop where the implicit device
// synchronisation of cudaMalloc/cudaFree is not acceptable.  For them this entry point
// renders one subset for one view using only a fixed scratch array that lives in this
// file: every GPU that loads libsplx holds those kNoAllocScratchBytes until the process
// exits.  It runs the same kernels as splx_render_partial (project, scan, fill, segment
// sort, raster forward) on sub-ranges of that array.
//
// Rules a caller must know:
//   * The first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it; make that first call
//     before any stream capture.
//   * All calls share the one array and leave their contents in it.  Calls that overlap
//     on the GPU (two streams, or two host threads) race on it: serialise them.
//   * Limits: n <= kNoAllocMaxGaussians, at most kNoAllocMaxPairs (Gaussian, tile) pairs,
//     at most kNoAllocMaxTiles tiles.  Larger requests are rejected with
//     SPLX_ERR_INVALID before any work; a pair overflow found on the device returns
//     SPLX_ERR_CAPACITY (the output is then not valid).
//   * The call synchronises `stream` once at the end to read the device status.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace splx {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int64_t kNoAllocMaxGaussians = 65536;
constexpr int64_t kNoAllocMaxPairs = int64_t(1) << 20;
constexpr int64_t kNoAllocMaxTiles = 65536;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t noalloc_scratch(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[device]);
  return cudaSuccess;
}

// Bump carving of the scratch array into 256-byte aligned regions.
struct Carver {
  unsigned char* base;
  size_t used = 0;
  bool ok = true;
  template <typename T>
  T* take(size_t count) {
    const size_t bytes = ((count * sizeof(T)) + 255) & ~size_t(255);
    if (used + bytes > kNoAllocScratchBytes) {
      ok = false;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

}  // namespace
}  // namespace splx

using namespace splx;

extern "C" int splx_render_partial_noalloc(const splx_gaussians* g, const splx_camera* c,
                                           const splx_opts* o, const splx_partial* out,
                                           splx_stream_t stream) {
  if (!g || !c || !o || !out || !out->rgb || !out->T || !out->depth || !out->last)
    return SPLX_ERR_INVALID;
  if (g->n < 0 || g->n > kNoAllocMaxGaussians || g->sh_degree < 0 || g->sh_degree > 3)
    return SPLX_ERR_INVALID;
  if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh ||
                   ((uintptr_t)g->quats & 15u)))
    return SPLX_ERR_INVALID;
  if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384 ||
      !(c->fx > 0.0f) || !(c->fy > 0.0f))
    return SPLX_ERR_INVALID;
  if (o->tile != 8 && o->tile != 16 && o->tile != 32) return SPLX_ERR_INVALID;
  if (!(o->alpha_min >= 0.0f) || !(o->alpha_max > 0.0f) || !(o->alpha_max < 1.0f) ||
      !(o->eps_T >= 0.0f) || !(o->eps_comp >= 0.0f))
    return SPLX_ERR_INVALID;
  const int tile = o->tile;
  const int tiles_x = (c->width + tile - 1) / tile, tiles_y = (c->height + tile - 1) / tile;
  const int64_t n_tiles = (int64_t)tiles_x * tiles_y;
  if (n_tiles > kNoAllocMaxTiles) return SPLX_ERR_INVALID;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
    return SPLX_ERR_CUDA;
  unsigned char* base = nullptr;
  if (noalloc_scratch(device, &base) != cudaSuccess) return SPLX_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t N = g->n;

  Carver cv{base};
  int* status = cv.take<int>(1);
  SubsetDev* sub_d = cv.take<SubsetDev>(1);
  ViewDev* view_d = cv.take<ViewDev>(1);
  ImgDev* img_d = cv.take<ImgDev>(1);
  Rec* rec = cv.take<Rec>((size_t)(N > 0 ? N : 1));
  uint32_t* counts = cv.take<uint32_t>((size_t)(N > 0 ? N : 1));
  uint32_t* tile_cnt = cv.take<uint32_t>((size_t)n_tiles);
  uint32_t* tile_start = cv.take<uint32_t>((size_t)n_tiles + 1);
  uint32_t* big_list = cv.take<uint32_t>((size_t)n_tiles);
  unsigned* big_count = cv.take<unsigned>(2);  // count, most chunks of one segment
  uint2* chunks = cv.take<uint2>((size_t)chunk_list_capacity(n_tiles, kNoAllocMaxPairs));
  unsigned* chunk_count = cv.take<unsigned>(1);
  void* scan_temp = cv.take<unsigned char>(scan_u32_temp_bytes(n_tiles));
  uint64_t* keys = cv.take<uint64_t>(kNoAllocMaxPairs);
  uint64_t* keys_alt = cv.take<uint64_t>(kNoAllocMaxPairs);
  uint2* ranges = cv.take<uint2>((size_t)n_tiles);
  if (!cv.ok) return SPLX_ERR_INVALID;

  // descriptors (same conversions as the allocating entry point)
  SubsetDev sd;
  std::memset(&sd, 0, sizeof(sd));
  sd.means = g->means; sd.log_scales = g->log_scales; sd.quats = g->quats;
  sd.opacity_logits = g->opacity_logits; sd.sh = g->sh; sd.n = N; sd.goff = 0;
  ViewDev vd;
  std::memcpy(vd.R, c->R, sizeof(vd.R));
  std::memcpy(vd.t, c->t, sizeof(vd.t));
  vd.fx = c->fx; vd.fy = c->fy; vd.cx = c->cx; vd.cy = c->cy; vd.near_plane = c->near_plane;
  for (int k = 0; k < 3; ++k)
    vd.eye[k] = (float)(-((double)c->R[k] * c->t[0] + (double)c->R[3 + k] * c->t[1] +
                          (double)c->R[6 + k] * c->t[2]));
  vd.W = c->width; vd.H = c->height; vd.tiles_x = tiles_x; vd.tiles_y = tiles_y;
  ImgDev im;
  im.rgb = out->rgb; im.T = out->T; im.D = out->depth; im.last = out->last; im.gCT = nullptr;

  BatchDev b;
  std::memset(&b, 0, sizeof(b));
  b.V = 1; b.K = 1; b.sh_degree = g->sh_degree; b.nc = n_sh(g->sh_degree); b.N = N;
  b.tile = tile;
  b.n_tiles = n_tiles;
  int tb = 1;
  while (tb < 62 && (int64_t(1) << tb) < n_tiles + 1) ++tb;
  b.tile_bits = tb;
  b.capacity = kNoAllocMaxPairs;
  b.eps_T = o->eps_T; b.eps_comp = o->eps_comp; b.alpha_min = o->alpha_min;
  b.alpha_max = o->alpha_max;
  for (int k = 0; k < 3; ++k) b.bg[k] = o->bg[k];
  b.subsets = sub_d; b.views = view_d; b.imgs = img_d;
  b.rec = rec; b.counts = counts; b.tile_cnt = tile_cnt; b.tile_start = tile_start;
  b.keys = keys; b.keys_alt = keys_alt; b.big_list = big_list; b.big_count = big_count;
  b.chunks = chunks; b.chunk_count = chunk_count;
  b.ranges = ranges; b.grad2d = nullptr; b.status = status; b.counters = nullptr;
  b.goff[0] = 0; b.goff[1] = N;
  b.tile_base[0] = 0; b.tile_base[1] = n_tiles;
  b.pix_off[0] = 0; b.pix_off[1] = (int64_t)c->width * c->height;

  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sub_d, &sd, sizeof(sd), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(view_d, &vd, sizeof(vd), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(img_d, &im, sizeof(im), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tile_cnt, 0, sizeof(uint32_t) * (size_t)n_tiles, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(big_count, 0, 2 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(chunk_count, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return SPLX_ERR_CUDA;

  launch_project(b, s);
  scan_u32(tile_cnt, tile_start, n_tiles, scan_temp, s);
  launch_fill(b, s);
  launch_seg_sort(b, merge_rounds_bound(N), s);
  launch_raster_fwd(b, s);
  if (cudaGetLastError() != cudaSuccess) return SPLX_ERR_CUDA;

  int st = 0;
  uint32_t total = 0;
  e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&total, tile_start + n_tiles, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return SPLX_ERR_CUDA;
  if ((st & ST_CAPACITY) || total > (uint64_t)kNoAllocMaxPairs) return SPLX_ERR_CAPACITY;
  if (st & ST_BOUNDS) return SPLX_ERR_STATE;
  return SPLX_OK;
}
