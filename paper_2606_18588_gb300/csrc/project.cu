// Projection (Sec. 2 step 1).
//
// One thread per Gaussian loops over every view of the batch, so the 59 parameters of
// a degree-3 Gaussian are read from HBM once per batch, not once per view.  Per (view,
// Gaussian) it writes one 64-byte record (2-D mean, scaled conic, opacity, depth, SH
// colour, packed pixel rectangle) and the number of tiles touched, and adds one to the
// pair count of each of those tiles (the segment sizes of the binning in bin.cu).
#include "common.cuh"
#include "spec.cuh"
#include "walk.cuh"

namespace splx {

// Real SH basis with the Condon-Shortley phase, degrees 0-3, ordered m = -l..l.
// Constants: sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the polynomial prefactors:
//   Y00 = 1/(2 sqrt(pi)); k1 = sqrt(3/(4pi)); k2a = sqrt(15/(4pi)); k2b = sqrt(5/(16pi));
//   k2c = sqrt(15/(16pi)); k3a = sqrt(35/(32pi)); k3b = sqrt(105/(4pi));
//   k3c = sqrt(21/(32pi)); k3d = sqrt(7/(16pi)); k3e = sqrt(105/(16pi)).
struct ShK {
  static constexpr float Y00 = 0.28209479177387814f;
  static constexpr float k1 = 0.48860251190291992f;
  static constexpr float k2a = 1.09254843059207907f;
  static constexpr float k2b = 0.31539156525252005f;
  static constexpr float k2c = 0.54627421529603953f;
  static constexpr float k3a = 0.59004358992664352f;
  static constexpr float k3b = 2.89061144264055405f;
  static constexpr float k3c = 0.45704579946446572f;
  static constexpr float k3d = 0.37317633259011540f;
  static constexpr float k3e = 1.44530572132027702f;
};

template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float* Y) {
  Y[0] = ShK::Y00;
  if (DEG >= 1) {
    Y[1] = -ShK::k1 * y;
    Y[2] = ShK::k1 * z;
    Y[3] = -ShK::k1 * x;
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = ShK::k2a * x * y;
    Y[5] = -ShK::k2a * y * z;
    Y[6] = ShK::k2b * (2.0f * zz - xx - yy);
    Y[7] = -ShK::k2a * x * z;
    Y[8] = ShK::k2c * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -ShK::k3a * y * (3.0f * xx - yy);
      Y[10] = ShK::k3b * x * y * z;
      Y[11] = -ShK::k3c * y * (4.0f * zz - xx - yy);
      Y[12] = ShK::k3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
      Y[13] = -ShK::k3c * x * (4.0f * zz - xx - yy);
      Y[14] = ShK::k3e * z * (xx - yy);
      Y[15] = -ShK::k3a * x * (xx - 3.0f * yy);
    }
  }
}

constexpr int kProjThreads = 256;
constexpr int kWalkFields = 13;  // per lane: tile test (8), rect x, rect y, tile base, width, 1/width

template <int DEG>
__global__ void __launch_bounds__(kProjThreads, 4) k_project(const BatchDev b) {
  // the warp's tile walk: each lane's tile-test inputs, [field][lane], and its outcome
  __shared__ float s_walk[kProjThreads / 32][kWalkFields][32];
  __shared__ int s_own[kProjThreads / 32][32];
  __shared__ uint32_t s_hits[kProjThreads / 32][32], s_any[kProjThreads / 32][32];
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lanes = __ballot_sync(0xffffffffu, g < b.N);  // lanes in the warp collectives
  if (g >= b.N) return;
  const int k = subset_of(b, g);
  const SubsetDev S = b.subsets[k];
  const int64_t i = g - S.goff;
  float m[3], ls[3], q[4];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    m[e] = __ldg(S.means + 3 * i + e);
    ls[e] = __ldg(S.log_scales + 3 * i + e);
  }
  const float4 qv = __ldg(reinterpret_cast<const float4*>(S.quats) + i);
  q[0] = qv.x; q[1] = qv.y; q[2] = qv.z; q[3] = qv.w;
  const float logit = __ldg(S.opacity_logits + i);
  const float opac = 1.0f / (1.0f + __expf(-logit));
  // the tile test's threshold on the conic's quadratic form (view independent)
  const float qmax = tile_cull_qmax(spec_opacity(logit), b.alpha_min);
  constexpr int NC = (DEG + 1) * (DEG + 1);
  // SH coefficients are read per visible view (L1/L2-resident across the view loop)
  // rather than held in registers, which keeps the kernel's occupancy up
  const float* shp = S.sh + i * (NC * 3);
  const bool sh_vec = (NC * 3) % 4 == 0 && (reinterpret_cast<uintptr_t>(shp) & 15) == 0;

  const SpecG G = spec_gaussian(ls, q);  // view-independent part of the specification
  if (b.cross) {
    // cross-boundary filtering: the other cells that the support box mu +- 3 s_max meets
    // (FP32 basic operations on the specification's activated scales)
    float smax = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) smax = fmaxf(smax, exp_spec(ls[a]));
    const float r3 = fm(3.0f, smax);
    const float lo[3] = {fs(m[0], r3), fs(m[1], r3), fs(m[2], r3)};
    const float hi[3] = {fa(m[0], r3), fa(m[1], r3), fa(m[2], r3)};
    unsigned long long mask = 0ull;
    const int own = b.cell_self >= 0 ? b.cell_self : k;
    for (int c = 0; c < b.ncells; ++c) {
      if (c == own) continue;
      const float* cb = b.cells + 6 * c;
      if (lo[0] <= cb[3] && hi[0] >= cb[0] && lo[1] <= cb[4] && hi[1] >= cb[1] &&
          lo[2] <= cb[5] && hi[2] >= cb[2])
        mask |= 1ull << c;
    }
    b.cross[g] = mask;
  }
  for (int v = 0; v < b.V; ++v) {
    const ViewDev& cam = b.views[v];
    const SpecOut so = bin_spec(m, G, cam.R, cam.t, cam.fx, cam.fy, cam.cx, cam.cy, cam.W,
                                cam.H, cam.near_plane);
    Rec r;
    uint32_t tiles = 0;
    float sA = 0.f, sB = 0.f, sC = 0.f;
    if (so.visible) {
      float bu, bv;
      blend_center(so, cam.fx, cam.fy, cam.cx, cam.cy, bu, bv);
      spec_conic(so, sA, sB, sC);
      const float inv = 1.0f / so.det;
      const float A = so.c * inv, B = -so.b * inv, Cc = so.a * inv;
      // p2 = power * log2(e) = qa dx^2 + qb dx dy + qc dy^2, about the blend's 2-D mean
      r.a = make_float4(bu, bv, -0.5f * kLog2e * A, -kLog2e * B);
      float dx = m[0] - cam.eye[0], dy = m[1] - cam.eye[1], dz = m[2] - cam.eye[2];
      const float rn = rsqrtf(dx * dx + dy * dy + dz * dz);
      dx *= rn; dy *= rn; dz *= rn;
      float Y[NC];
      sh_eval<DEG>(dx, dy, dz, Y);
      // colour = SH(direction) + 0.5 per channel, coefficients summed in degree order
      float acc[3] = {0.5f, 0.5f, 0.5f};
      if (sh_vec) {
        const float4* s4 = reinterpret_cast<const float4*>(shp);
#pragma unroll
        for (int q4 = 0; q4 < (NC * 3) / 4; ++q4) {
          const float4 sv = __ldg(s4 + q4);
          const float vals[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int e = 4 * q4 + c;
            acc[e % 3] = fmaf(Y[e / 3], vals[c], acc[e % 3]);
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < NC * 3; ++e) acc[e % 3] = fmaf(Y[e / 3], __ldg(shp + e), acc[e % 3]);
      }
      const float col[3] = {fmaxf(acc[0], 0.0f), fmaxf(acc[1], 0.0f), fmaxf(acc[2], 0.0f)};
      const uint32_t rx = (uint32_t)so.x0 | ((uint32_t)so.x1 << 16);
      const uint32_t ry = (uint32_t)so.y0 | ((uint32_t)so.y1 << 16);
      r.b = make_float4(-0.5f * kLog2e * Cc, opac, so.tz, __uint_as_float(rx));
      r.c = make_float4(col[0], col[1], col[2], __uint_as_float(ry));
      const int B_ = b.tile;
      const int tx0 = so.x0 / B_, tx1 = so.x1 / B_, ty0 = so.y0 / B_, ty1 = so.y1 / B_;
      tiles = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
    }
    // a culled Gaussian's record is never read (its count is 0; nothing lists it), so it
    // is not written: for views that see a small part of the scene that is most records
    Rec* dst = b.rec + (int64_t)v * b.N + g;
    if (so.visible) { dst->a = r.a; dst->b = r.b; dst->c = r.c; }
    b.counts[(int64_t)v * b.N + g] = tiles;
    // count this Gaussian in every tile of its rectangle that passes the tile test (the
    // segment sizes of the binning); lanes that hit the same tile add together
    // (neighbouring Gaussians are neighbours in memory), so most tiles see one atomic
    // per warp
    const int tw = so.visible ? so.x1 / b.tile - so.x0 / b.tile + 1 : 1;
    const int64_t tbase = b.tile_base[v] + (int64_t)k * cam.tiles_x * cam.tiles_y +
                          (int64_t)(so.visible ? so.y0 / b.tile : 0) * cam.tiles_x +
                          (so.visible ? so.x0 / b.tile : 0);
    const int tx0 = so.visible ? so.x0 / b.tile : 0, ty0 = so.visible ? so.y0 / b.tile : 0;
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    const TileCull tc = tile_cull_prep(so.u, so.v, sA, sB, sC, so.visible ? qmax : -1.0f);
    uint32_t hits = 0;  // bit j: the j-th tile of the rectangle passes the tile test
    bool any_pair = false;
    // head: every lane tests its own first H tiles, H = the warp's mean count rounded up
    const int nact = __popc(lanes);
    const int H = ((int)__reduce_add_sync(lanes, tiles) + nact - 1) / nact;
    int jx = 0, jy = 0;  // column / row of the j-th tile inside the rectangle
    for (int j = 0; j < H; ++j) {
      unsigned t = 0xFFFFFFFFu;
      if (j < (int)tiles &&
          tile_hits_spec(tc, so.x0, so.x1, so.y0, so.y1, tx0 + jx, ty0 + jy, b.tile)) {
        t = (unsigned)(tbase + jy * cam.tiles_x + jx);
        any_pair = true;
        if (j < 32) hits |= 1u << j;
      }
      if (++jx == tw) { jx = 0; ++jy; }
      const unsigned peers = __match_any_sync(lanes, t);
      if (t != 0xFFFFFFFFu && lane == __ffs(peers) - 1)
        atomicAdd(&b.tile_cnt[t], (unsigned)__popc(peers));
    }
    // tail: the tiles beyond H of the lanes that have more, spread evenly over the warp
    const int rest = (int)tiles > H ? (int)tiles - H : 0;
    if (__any_sync(lanes, rest > 0)) {
      float(*f)[32] = s_walk[warp];
      f[0][lane] = tc.u; f[1][lane] = tc.v; f[2][lane] = tc.A; f[3][lane] = tc.B;
      f[4][lane] = tc.C; f[5][lane] = tc.qmax; f[6][lane] = tc.rBC; f[7][lane] = tc.rBA;
      f[8][lane] = __uint_as_float((uint32_t)so.x0 | ((uint32_t)so.x1 << 16));
      f[9][lane] = __uint_as_float((uint32_t)so.y0 | ((uint32_t)so.y1 << 16));
      f[10][lane] = __uint_as_float((uint32_t)tbase);
      f[11][lane] = __int_as_float(tw);
      f[12][lane] = 1.0f / (float)tw;
      s_hits[warp][lane] = 0u;
      s_any[warp][lane] = 0u;
      const WarpWalk walk = warp_walk_begin(lanes, rest);
      for (int base = 0; base < walk.total; base += walk.nact) {
        int jr;
        const int o = warp_walk_owner(walk, base, s_own[warp], jr);
        unsigned t = 0xFFFFFFFFu;
        if (o >= 0) {
          const int j = H + jr;
          TileCull oc;
          oc.u = f[0][o]; oc.v = f[1][o]; oc.A = f[2][o]; oc.B = f[3][o];
          oc.C = f[4][o]; oc.qmax = f[5][o]; oc.rBC = f[6][o]; oc.rBA = f[7][o];
          const uint32_t rx = __float_as_uint(f[8][o]), ry = __float_as_uint(f[9][o]);
          const int x0 = (int)(rx & 0xFFFFu), x1 = (int)(rx >> 16);
          const int y0 = (int)(ry & 0xFFFFu), y1 = (int)(ry >> 16);
          int ox, oy;
          walk_tile(j, __float_as_int(f[11][o]), f[12][o], ox, oy);
          if (tile_hits_spec(oc, x0, x1, y0, y1, x0 / b.tile + ox, y0 / b.tile + oy, b.tile)) {
            t = __float_as_uint(f[10][o]) + (unsigned)(oy * cam.tiles_x + ox);
            if (j < 32) atomicOr(&s_hits[warp][o], 1u << j);
            s_any[warp][o] = 1u;
          }
        }
        const unsigned peers = __match_any_sync(lanes, t);
        if (t != 0xFFFFFFFFu && lane == __ffs(peers) - 1)
          atomicAdd(&b.tile_cnt[t], (unsigned)__popc(peers));
      }
      __syncwarp(lanes);
      hits |= s_hits[warp][lane];
      any_pair = any_pair || s_any[warp][lane] != 0u;
    }
    // cross-boundary filtering: the depth range of the subset's kept Gaussians in this view
    if (b.zr) {
      const unsigned peers = __match_any_sync(lanes, so.visible ? k : -1);
      if (so.visible) {
        const uint32_t d = __float_as_uint(so.tz);
        const uint32_t dmin = __reduce_min_sync(peers, d), ndmax = __reduce_min_sync(peers, ~d);
        if (lane == __ffs(peers) - 1) {
          uint32_t* z = b.zr + 2 * ((int64_t)v * b.K + k);
          atomicMin(z, dmin);
          atomicMin(z + 1, ndmax);
        }
      }
    }
    // spatial visibility: grow the subset's bounding tile rectangle in this view by this
    // Gaussian's tile rectangle (lanes of one subset reduce first, one atomic each)
    if (b.omega) {
      const unsigned peers = __match_any_sync(lanes, any_pair ? k : -1);
      if (any_pair) {
        uint32_t e[4] = {(uint32_t)tx0, (uint32_t)ty0, ~(uint32_t)(so.x1 / b.tile),
                         ~(uint32_t)(so.y1 / b.tile)};
#pragma unroll
        for (int q = 0; q < 4; ++q) e[q] = __reduce_min_sync(peers, e[q]);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) {
          uint32_t* om = b.omega + ((int64_t)v * b.K + k) * 4;
#pragma unroll
          for (int q = 0; q < 4; ++q) atomicMin(om + q, e[q]);
        }
      }
    }
    // what fill needs to repeat exactly these decisions: the pass bits of the rectangle's
    // tiles when there are at most 32 of them, else the test's inputs
    if (so.visible)
      dst->d = make_float4(sA, sB, sC, tiles <= 32u ? __uint_as_float(hits) : qmax);
  }
}

void launch_project(const BatchDev& b, cudaStream_t s) {
  const BatchDev& P = b;
  const int threads = kProjThreads;
  const int64_t blocks = (b.N + threads - 1) / threads;
  if (blocks == 0) return;
  switch (b.sh_degree) {
    case 0: k_project<0><<<(unsigned)blocks, threads, 0, s>>>(P); break;
    case 1: k_project<1><<<(unsigned)blocks, threads, 0, s>>>(P); break;
    case 2: k_project<2><<<(unsigned)blocks, threads, 0, s>>>(P); break;
    default: k_project<3><<<(unsigned)blocks, threads, 0, s>>>(P); break;
  }
  count_launch();
}

}  // namespace splx
