// Local rendering of every (view, subset) tile: forward (Eq. 1-4) and backward.
//
// One CTA per image tile of TS x TS pixels; each thread owns PPT pixels, one in each of
// PPT blocks of 8 x 4 pixels (TS x TS/PPT threads; layout below), so the shared-memory
// loads, the rectangle test and the dx-dependent terms of an entry are shared by PPT
// pixels, and in the backward the per-entry warp reduction and atomics are amortised over
// PPT pixels.
// The tile's sorted list is walked in batches of NB entries staged in shared memory.
// A pixel takes a Gaussian only inside its integer 3-sigma rectangle (so the result does
// not depend on TS), with alpha = min(alpha_max, o 2^(p2)) >= alpha_min, and stops before
// the Gaussian that would take its transmittance below eps_T.  The CTA leaves the list
// once every pixel has stopped (__syncthreads_count).
//
// The backward walks the same list back to front from each pixel's last blended entry,
// recovering T_i = T_{i+1} / (1 - alpha_i) from the stored final T^m, and applies the
// adjoint of Eq. 3-4 with the composite adjoint (dL/dC^m, dL/dT^m of Eq. 6-7) as input:
//   dC^m/dc_i = alpha_i T_i,  dC^m/dalpha_i = c_i T_i - B_i / (1 - alpha_i),
//   dT^m/dalpha_i = -T^m / (1 - alpha_i),  B_i = sum_{j>i} c_j alpha_j T_j.
// Per-Gaussian sums over the tile's pixels are reduced with warp shuffles and added to
// the per-(view, Gaussian) 2-D gradient with float4 atomics.  With gp = dL/dpower at a
// pixel, power = -(A dx^2 + 2 B dx dy + C dy^2) / 2 and (dx, dy) = pixel centre - (u, v),
// the record holds the conic-free moments of ge = gp / o = dL/dalpha e^power (0 where
// alpha is clamped), sum ge dx, ge dy, ge dx^2, ge dx dy, ge dy^2, and dL/do = sum ge;
// dL/du = o (A sum ge dx + B sum ge dy), dL/dA = -o sum ge dx^2 / 2 and the rest follow
// linearly in the projection adjoint, which knows the conic and the opacity.
#include "common.cuh"

namespace splx {

namespace {

// Per-entry terms shared by the pixels of one column: dx, qa dx^2 and qb dx.
struct ColTerms {
  float dx, hx, bx;
};

__device__ __forceinline__ ColTerms col_terms(const float4 a, float pcx) {
  ColTerms c;
  c.dx = __fsub_rn(pcx, a.x);
  c.hx = __fmul_rn(__fmul_rn(a.z, c.dx), c.dx);
  c.bx = __fmul_rn(a.w, c.dx);
  return c;
}

// 2^x and 1/x as single special-function-unit instructions (relative error about 2^-22;
// subnormal results flush to zero, which the alpha threshold rejects anyway).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// alpha of an entry at one pixel of the column; the same code runs in the forward and
// the backward so both take bit-identical decisions.  Returns false if skipped.
__device__ __forceinline__ bool pixel_alpha(const ColTerms& c, float ay, float qc, float o,
                                            float pcy, float amin, float amax, float& alpha,
                                            float& ex, float& dy, bool& clamped) {
  dy = __fsub_rn(pcy, ay);
  const float p2 = __fmaf_rn(__fmaf_rn(qc, dy, c.bx), dy, c.hx);
  ex = ex2_approx(p2);  // finite for the rounding-sized p2 > 0 that the test below rejects
  const float raw = __fmul_rn(o, ex);
  clamped = raw > amax;
  alpha = clamped ? amax : raw;
  return p2 <= 0.0f && alpha >= amin;
}

// Adds per-thread counts into counters[slot] with one atomic per warp.
__device__ __forceinline__ void flush_counter(unsigned long long* counters, int slot, unsigned v) {
  if (!counters) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(counters + slot, (unsigned long long)v);
}

// Sum of v[0..8] over the warp by reduce-scatter: each exchange sends half of the
// values a lane still holds, so 8 values take 4 + 2 + 1 + 1 + 1 shuffles instead of
// 8 x 5.  Afterwards lane l holds the full sum of value (l >> 2) & 7 in `mine`, and
// every lane holds the sum of value 8 in `v8`.
__device__ __forceinline__ void warp_reduce9(const float (&v)[9], int lane, float& mine,
                                             float& v8) {
  const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0, h2 = (lane & 4) != 0;
  float a[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float send = h4 ? v[k] : v[k + 4];
    const float keep = h4 ? v[k + 4] : v[k];
    a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float c[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = h3 ? a[k] : a[k + 2];
    const float keep = h3 ? a[k + 2] : a[k];
    c[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float d = (h2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h2 ? c[0] : c[1], 4);
  d += __shfl_xor_sync(0xffffffffu, d, 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  mine = d;
  float e = v[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  v8 = e;
}

// Pixels of a thread: slot i of PPT is an 8 x 4 block of the tile, lanes laid out as
// 8 columns x 4 rows inside it; a warp's PPT blocks tile a 16 x 16 region (PPT = 8), a
// 16 x 8 region (PPT = 4) or an 8 x 8 region (PPT = 2).  A Gaussian's footprint then meets
// few blocks, and a block it meets keeps many lanes busy.  (x, y) is the thread's pixel in
// slot 0; slot i adds (8 (i & 1), 4 (i >> 1)) for PPT = 4 and 8, and (0, 4 i) for PPT = 2.
struct TileInfo {
  int v, k, x, y, W, H, tx, ty;
};

// Compacts the staged entries [0, cnt) whose rectangle meets the warp's region (origin RX,
// RY; 8 x 8 pixels for PPT = 2, 16 x 8 for PPT = 4) into list[], in entry order, as
// entry | (region columns the rectangle spans) << 8 | (region rows it spans) << 24: bit c
// of the column mask for column RX + c, bit r of the row mask for row RY + r.  A lane's
// slot test is then two bit extractions (slot_mask).  One lane tests one entry, 32 at a
// time; returns the number listed.
template <int PPT>
__device__ __forceinline__ int compact_entries(const float4* sB, const float4* sC, int cnt,
                                               int RX, int RY, int lane, uint32_t* list) {
  constexpr int RW = PPT == 4 ? 16 : 8;  // region width
  int nl = 0;
  for (int g0 = 0; g0 < cnt; g0 += 32) {
    const int e = g0 + lane;
    uint32_t item = 0;
    if (e < cnt) {
      const uint32_t rx = __float_as_uint(sB[e].w), ry = __float_as_uint(sC[e].w);
      const int c0 = max((int)(rx & 0xFFFFu) - RX, 0), c1 = min((int)(rx >> 16) - RX, RW - 1);
      const int r0 = max((int)(ry & 0xFFFFu) - RY, 0), r1 = min((int)(ry >> 16) - RY, 7);
      if (c0 <= c1 && r0 <= r1) {
        const uint32_t cm = ((2u << (c1 - c0)) - 1u) << c0;
        const uint32_t rm = ((2u << (r1 - r0)) - 1u) << r0;
        item = (uint32_t)e | (cm << 8) | (rm << 24);
      }
    }
    const unsigned hit = __ballot_sync(0xffffffffu, item != 0u);
    if (item) list[nl + __popc(hit & ((1u << lane) - 1u))] = item;
    nl += __popc(hit);
  }
  __syncwarp();
  return nl;
}

// Slots of the lane at column lx, row ly of its 8 x 4 blocks whose pixel lies in the
// rectangle of a compacted list item: bit i for slot i (pixel column lx + 8 col(i), row
// ly + 4 row(i) of the region).
template <int PPT>
__device__ __forceinline__ unsigned slot_mask(uint32_t item, int lx, int ly) {
  const uint32_t cs = item >> (8 + lx), rs = item >> (24 + ly);
  const uint32_t c0 = cs & 1u, r0 = rs & 1u, r1 = (rs >> 4) & 1u;
  if (PPT == 4) {
    const uint32_t c1 = (cs >> 8) & 1u;
    return (c0 & r0) | ((c1 & r0) << 1) | ((c0 & r1) << 2) | ((c1 & r1) << 3);
  }
  return (c0 & r0) | ((c0 & r1) << 1);
}

template <int PPT>
__device__ __forceinline__ int slot_col(int i) { return PPT >= 4 ? (i & 1) : 0; }
template <int PPT>
__device__ __forceinline__ int slot_row(int i) { return PPT >= 4 ? (i >> 1) : i; }
// block columns (x offsets 0, 8) and rows (y offsets 0, 4, ...) of a thread's slots
template <int PPT>
constexpr int kSlotCols = PPT >= 4 ? 2 : 1;
template <int PPT>
constexpr int kSlotRows = PPT / kSlotCols<PPT>;

template <int TS, int PPT>
__device__ __forceinline__ TileInfo decode_tile(const BatchDev& b, int64_t id) {
  TileInfo ti;
  ti.v = view_of(b.tile_base, b.V, id);
  const ViewDev& cam = b.views[ti.v];
  const int64_t nt = (int64_t)cam.tiles_x * cam.tiles_y;
  const int64_t rem = id - b.tile_base[ti.v];
  ti.k = (int)(rem / nt);
  const int64_t t = rem - (int64_t)ti.k * nt;
  const int tx = (int)(t % cam.tiles_x), ty = (int)(t / cam.tiles_x);
  ti.tx = tx;
  ti.ty = ty;
  const int w = (int)(threadIdx.x >> 5), l = (int)(threadIdx.x & 31);
  int rx0 = 0, ry0 = 0;
  if (PPT == 8) {  // 16 x 16 regions
    rx0 = 16 * (w % (TS / 16));
    ry0 = 16 * (w / (TS / 16));
  } else if (PPT == 4) {  // 16 x 8 regions
    constexpr int kRegionsPerRow = TS >= 16 ? TS / 16 : 1;
    rx0 = 16 * (w % kRegionsPerRow);
    ry0 = 8 * (w / kRegionsPerRow);
  } else {  // 8 x 8 regions
    rx0 = 8 * (w % (TS / 8));
    ry0 = 8 * (w / (TS / 8));
  }
  ti.x = tx * TS + rx0 + (l & 7);
  ti.y = ty * TS + ry0 + (l >> 3);
  ti.W = cam.W;
  ti.H = cam.H;
  return ti;
}

}  // namespace

// kCount variants (eager runs only) also count the work for the roofline: thread-entries
// examined, (pixel, entry) alpha evaluations and blends / contributions.
constexpr int kNB = 256;  // list entries staged in shared memory per batch
static_assert(kNB <= 256, "a compacted list item holds the entry in 8 bits");
// the backward stages fewer at a time where its threads allow (one entry per thread at
// least); one-warp CTAs stage 64, which keeps their shared memory at 7.4 KB
template <int TS, int PPT>
constexpr int kNBBwd = TS * TS / PPT > 128 ? TS * TS / PPT : (TS * TS / PPT == 32 ? 64 : 128);
// resident CTAs the backward's register limit is set for
template <int TS, int PPT>
constexpr int kMinBlocksBwd = TS == 16 ? (PPT == 8 ? 28 : 16) : 1;
// backward: up to this many lanes with a contribution add their gradients with their own
// atomics (three per lane) instead of the warp reduction (about 45 instructions and nine
// atomics); measured on the 10M step: 3 -> 18.58 ms, 12 -> 17.95, 20 -> 17.55, 32 -> 19.19
constexpr int kDirectLanes = 20;

template <int TS, int PPT, bool kCount>
__device__ __forceinline__ void fwd_item(const BatchDev& b, const int64_t id, float4* sA,
                                         float4* sB, float4* sC, uint32_t* sL) {
  constexpr int NTH = TS * TS / PPT;
  constexpr int NB = kNB;
  const TileInfo ti = decode_tile<TS, PPT>(b, id);
  if (!in_omega(b, ti.v, ti.k, ti.tx, ti.ty)) {
    // outside the subset's visible region: no pairs; the composite never reads this tile.
    // Its transmittance is 1, which the first saturation-skipping wave must still record.
    if (kCount && threadIdx.x == 0 && b.counters) atomicAdd(b.counters + 7, 1ull);
    if (b.order && b.wave == 0) {
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        const int px = ti.x + 8 * slot_col<PPT>(i), py = ti.y + 4 * slot_row<PPT>(i);
        if (px < ti.W && py < ti.H) b.tpre[b.pix_off[ti.v] + (int64_t)py * ti.W + px] = 1.0f;
      }
    }
    return;
  }
  const uint2 rg = b.ranges[id];
  const int64_t start = rg.x, end = rg.y > rg.x ? rg.y : rg.x;
  const Rec* rec = b.rec + (int64_t)ti.v * b.N;
  const float pcx0 = (float)ti.x + 0.5f, pcx1 = (float)(ti.x + 8) + 0.5f;
  const float amin = b.alpha_min, amax = b.alpha_max, epsT = b.eps_T;
  float T[PPT], c0[PPT], c1[PPT], c2[PPT], D[PPT];
  int last[PPT];
  unsigned live = 0;  // bit i: pixel i still blending
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    T[i] = 1.0f; c0[i] = c1[i] = c2[i] = D[i] = 0.0f; last[i] = -1;
    if (ti.x + 8 * slot_col<PPT>(i) < ti.W && ti.y + 4 * slot_row<PPT>(i) < ti.H) live |= 1u << i;
  }
  const ImgDev im = b.imgs[ti.v * b.K + ti.k];
  const int64_t HW = (int64_t)ti.W * ti.H;
  if ((b.order && b.wave > 0) || b.sat) {
    const unsigned inb = live;  // slots inside the image
    // saturation skipping: a pixel where the subsets rendered before this one took the
    // transmittance below eps_comp leaves this subset's pixel set (the composite would
    // skip this subset there anyway): it stays empty (T = 1, no contributor); a tile with
    // no open pixel is left empty as a whole.  With a stale saturation state the pixel
    // set is the one the state names (ranks below the pixel's state)
    if (b.sat) {
      const uint8_t* sp = b.sat[ti.v];
      const int rk = b.rank[ti.v * b.K + ti.k];
#pragma unroll
      for (int i = 0; i < PPT; ++i)
        if ((live >> i) & 1u &&
            !((int)sp[(int64_t)(ti.y + 4 * slot_row<PPT>(i)) * ti.W + ti.x + 8 * slot_col<PPT>(i)] >
              rk))
          live &= ~(1u << i);
    } else {
      const float* tp = b.tpre + b.pix_off[ti.v];
#pragma unroll
      for (int i = 0; i < PPT; ++i)
        if ((live >> i) & 1u &&
            !(tp[(int64_t)(ti.y + 4 * slot_row<PPT>(i)) * ti.W + ti.x + 8 * slot_col<PPT>(i)] >=
              b.eps_comp))
          live &= ~(1u << i);
    }
    if (!__syncthreads_or(live != 0)) {
      if (kCount && threadIdx.x == 0 && b.counters) atomicAdd(b.counters + 6, 1ull);
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        if (!((inb >> i) & 1u)) continue;
        const int64_t p = (int64_t)(ti.y + 4 * slot_row<PPT>(i)) * ti.W + ti.x + 8 * slot_col<PPT>(i);
        im.rgb[p] = 0.0f;
        im.rgb[HW + p] = 0.0f;
        im.rgb[2 * HW + p] = 0.0f;
        im.T[p] = 1.0f;
        im.D[p] = 0.0f;
        im.last[p] = -1;
      }
      return;
    }
  }
  // with no selected prefix (kSelNone) the item goes straight to the full sort and its
  // second forward (a selected prefix needs nothing here: its range points into keys_alt)
  // The item's id, if its list is a selected prefix, waits in shared memory for the end of
  // the walk (no register held across it).  A second forward after a prefix (kSelResume)
  // takes the pixels' state from the planes the first one wrote and walks the whole
  // sorted list from the prefix's end: its first entries are the prefix's, in its order.
  __shared__ uint32_t s_prefix_item;
  int64_t walk0 = start;
  if (b.sel) {
    const uint32_t sv = b.sel[id];
    if (sv == kSelNone) {
      if (threadIdx.x == 0) {
        b.retry[atomicAdd(b.retry_count, 1u)] = (uint32_t)id;
        if (kCount && b.counters) atomicAdd(b.counters + 9, 1ull);
      }
      return;
    }
    if (sv & kSelResume) {
      walk0 = start + (sv & ~kSelResume);
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        const int px = ti.x + 8 * slot_col<PPT>(i), py = ti.y + 4 * slot_row<PPT>(i);
        if (px >= ti.W || py >= ti.H) continue;
        const int64_t p = (int64_t)py * ti.W + px;
        c0[i] = im.rgb[p];
        c1[i] = im.rgb[HW + p];
        c2[i] = im.rgb[2 * HW + p];
        T[i] = im.T[p];
        D[i] = im.D[p];
        const int l = im.last[p];
        last[i] = l <= -2 ? -3 - l : l;
        if (l <= -2) live &= ~(1u << i);  // it had stopped inside the prefix
      }
    }
    if (threadIdx.x == 0) s_prefix_item = sv && !(sv & kSelResume) ? (uint32_t)id : kSelNone;
  }
  unsigned n_eval = 0, n_pix = 0, n_blend = 0;
  for (int64_t base = walk0; base < end; base += NB) {
    if (__syncthreads_count(live == 0) == NTH) break;
#pragma unroll
    for (int r = 0; r < NB / NTH; ++r) {
      const int slot = r * NTH + (int)threadIdx.x;
      const int64_t j = base + slot;
      if (j < end) {
        uint32_t g = (uint32_t)b.keys[j];  // low half of the sorted key
        if (g >= (uint32_t)b.N) { atomicOr(b.status, ST_BOUNDS); g = 0; }
        const Rec* rp = rec + g;
        sA[slot] = rp->a;
        sB[slot] = rp->b;
        sC[slot] = rp->c;
      }
    }
    __syncthreads();
    if (__any_sync(0xffffffffu, live != 0)) {
      const int cnt = (int)((end - base) < NB ? (end - base) : NB);
      const int lane = (int)(threadIdx.x & 31);
      uint32_t* list = sL + (threadIdx.x >> 5) * NB;
      const int nl = compact_entries<PPT>(sB, sC, cnt, ti.x - (lane & 7), ti.y - (lane >> 3),
                                          lane, list);
      auto entry = [&](const uint32_t item) {
        const int jj = (int)(item & 0xFFu);
        const float4 Bv = sB[jj];
        const float4 Cv = sC[jj];
        // slots to evaluate: in the rectangle, still blending
        const unsigned todo = live & slot_mask<PPT>(item, lane & 7, lane >> 3);
        const float4 Av = sA[jj];
        const ColTerms ct0 = col_terms(Av, pcx0), ct1 = col_terms(Av, pcx1);
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          if (!((todo >> i) & 1u)) continue;
          const int ci = slot_col<PPT>(i), ri = slot_row<PPT>(i);
          if (kCount) ++n_pix;
          float alpha, ex, dy;
          bool cl;
          if (!pixel_alpha(ci ? ct1 : ct0, Av.y, Bv.x, Bv.y, (float)(ti.y + 4 * ri) + 0.5f, amin,
                           amax, alpha, ex, dy, cl))
            continue;
          const float Tn = T[i] * (1.0f - alpha);
          if (Tn < epsT) { live &= ~(1u << i); continue; }
          const float w = alpha * T[i];
          c0[i] = fmaf(Cv.x, w, c0[i]);
          c1[i] = fmaf(Cv.y, w, c1[i]);
          c2[i] = fmaf(Cv.z, w, c2[i]);
          D[i] = fmaf(Bv.z, w, D[i]);
          T[i] = Tn;
          last[i] = (int)(base - start) + jj;
          if (kCount) ++n_blend;
        }
      };
      // four entries per warp-wide test of whether any pixel still blends (entries after
      // the warp's last pixel has stopped find no slot to evaluate)
      int q = 0;
      for (; q < nl; q += 4) {
        if (!__any_sync(0xffffffffu, live != 0)) break;
        entry(list[q]);
        if (q + 1 < nl) entry(list[q + 1]);
        if (q + 2 < nl) entry(list[q + 2]);
        if (q + 3 < nl) entry(list[q + 3]);
      }
      q = q < nl ? q : nl;
      if (kCount && lane == 0) n_eval += (unsigned)q;
    }
  }
  if (kCount) {
    flush_counter(b.counters, 0, n_eval);
    flush_counter(b.counters, 1, n_pix);
    flush_counter(b.counters, 2, n_blend);
  }
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int px = ti.x + 8 * slot_col<PPT>(i), py = ti.y + 4 * slot_row<PPT>(i);
    if (px >= ti.W || py >= ti.H) continue;
    const int64_t p = (int64_t)py * ti.W + px;
    im.rgb[p] = c0[i];
    im.rgb[HW + p] = c1[i];
    im.rgb[2 * HW + p] = c2[i];
    im.T[p] = T[i];
    im.D[p] = D[i];
    im.last[p] = last[i];
  }
  if (b.sel) {
    // a walk that ended inside a sorted prefix is exact unless a pixel is still blending, in
    // which case the entries after the prefix matter in their sorted order (the barrier
    // also publishes s_prefix_item)
    const bool more = __syncthreads_or(live != 0);
    const uint32_t pid = s_prefix_item;
    if (pid != kSelNone) {
      if (threadIdx.x == 0 && kCount && b.counters) atomicAdd(b.counters + 8, 1ull);
      if (more) {
        if (threadIdx.x == 0) {
          b.retry[atomicAdd(b.retry_count, 1u)] = pid;
          if (kCount && b.counters) atomicAdd(b.counters + 9, 1ull);
        }
        // the planes hold the state at the prefix's end for the second forward: a pixel
        // that has stopped keeps its last index as -3 - last
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          const int px = ti.x + 8 * slot_col<PPT>(i), py = ti.y + 4 * slot_row<PPT>(i);
          if (px < ti.W && py < ti.H && !((live >> i) & 1u))
            im.last[(int64_t)py * ti.W + px] = -3 - last[i];
        }
        return;  // the second forward writes the prefix transmittance and the planes
      }
    }
  }
  if (b.order) {
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int px = ti.x + 8 * slot_col<PPT>(i), py = ti.y + 4 * slot_row<PPT>(i);
      if (px >= ti.W || py >= ti.H) continue;
      float* tp = b.tpre + b.pix_off[ti.v] + (int64_t)py * ti.W + px;
      *tp = b.wave == 0 ? T[i] : *tp * T[i];
    }
  }
}

template <int TS, int PPT, bool kCount>
__device__ __forceinline__ void bwd_item(const BatchDev& b, const int64_t id, float4* sA,
                                         float4* sB, float4* sC, uint32_t* sG, int& s_maxlast,
                                         float4* sQ) {
  constexpr int NTH = TS * TS / PPT;
  constexpr int NB = kNBBwd<TS, PPT>;
  const TileInfo ti = decode_tile<TS, PPT>(b, id);
  if (!in_omega(b, ti.v, ti.k, ti.tx, ti.ty)) return;  // nothing written there, nothing to do
  const uint2 rg = b.ranges[id];
  const int64_t start = rg.x;  // (a selected prefix's range points into keys_alt)
  const ImgDev im = b.imgs[ti.v * b.K + ti.k];
  // composite adjoint of the thread's pixels: (dL/dC^m rgb, -T^m dL/dT^m) per slot, in
  // shared memory (read only where a pixel takes an entry), which keeps registers down
  float4* gq = sQ + threadIdx.x;  // slot i at gq[i * NTH]
  // W = -T^m dL/dT^m - sum_ch dL/dC^m_ch B_ch: the colour suffix sums B enter the alpha
  // adjoint only through this dot product, so one scalar per pixel carries them
  float T[PPT], W[PPT];
  int mylast[PPT];
  int tlast = -1;  // largest last over this thread's pixels
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    float4 gct = make_float4(0.f, 0.f, 0.f, 0.f);
    T[i] = 1.0f;
    mylast[i] = -1;
    const int px = ti.x + 8 * slot_col<PPT>(i), py = ti.y + 4 * slot_row<PPT>(i);
    if (px < ti.W && py < ti.H) {
      const int64_t p = (int64_t)py * ti.W + px;
      gct = im.gCT[p];
      T[i] = im.T[p];
      mylast[i] = im.last[p];
      if (gct.x == 0.0f && gct.y == 0.0f && gct.z == 0.0f && gct.w == 0.0f)
        mylast[i] = -1;
    }
    W[i] = -T[i] * gct.w;
    gq[i * NTH] = make_float4(gct.x, gct.y, gct.z, 0.0f);
    tlast = mylast[i] > tlast ? mylast[i] : tlast;
  }
  if (threadIdx.x == 0) s_maxlast = -1;
  __syncthreads();
  if (tlast >= 0) atomicMax(&s_maxlast, tlast);
  __syncthreads();
  const int maxlast = s_maxlast;
  if (maxlast < 0) return;

  const Rec* rec = b.rec + (int64_t)ti.v * b.N;
  float4* g2 = b.grad2d + (int64_t)ti.v * b.N * 3;
  const float pcx0 = (float)ti.x + 0.5f, pcx1 = (float)(ti.x + 8) + 0.5f;
  const float amin = b.alpha_min, amax = b.alpha_max;
  const int lane = threadIdx.x & 31;
  unsigned n_evalb = 0, n_pixb = 0, n_actb = 0;

  // the thread's keys of the next batch (low halves: the Gaussian indices), loaded one
  // batch ahead so that staging waits for the records only
  uint32_t nk[NB / NTH];
  auto load_keys = [&](int top) {
#pragma unroll
    for (int r = 0; r < NB / NTH; ++r) {
      const int j = top - (r * NTH + (int)threadIdx.x);
      nk[r] = j >= 0 ? (uint32_t)b.keys[start + j] : 0u;
    }
  };
  load_keys(maxlast);
  for (int top = maxlast; top >= 0; top -= NB) {
    const int lo = top - NB + 1 > 0 ? top - NB + 1 : 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NB / NTH; ++r) {
      const int slot = r * NTH + (int)threadIdx.x;  // slot s holds entry top - s
      const int j = top - slot;
      if (j >= lo) {
        uint32_t g = nk[r];
        if (g >= (uint32_t)b.N) { atomicOr(b.status, ST_BOUNDS); g = 0; }
        const Rec* rp = rec + g;
        sA[slot] = rp->a;
        sB[slot] = rp->b;
        sC[slot] = rp->c;
        sG[slot] = g;
      }
    }
    load_keys(top - NB);
    __syncthreads();
    const int cnt = top - lo + 1;
    if (kCount && tlast >= lo) n_evalb += (unsigned)((tlast < top ? tlast : top) - lo + 1);
    for (int jj = 0; jj < cnt; ++jj) {
      const int j = top - jj;
      // the entry's sums over the warp's pixels: ge dx, ge dy, ge dx^2, ge dx dy, ge dy^2
      // (ge = dL/dpower / o), dL/do and dL/dcolour; the projection adjoint applies the conic
      // and the opacity
      float sx = 0.f, sy = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f, go = 0.f, gr = 0.f, gg = 0.f,
            gb = 0.f;
      bool act = false;
      if (j <= tlast) {
        const float4 Bv = sB[jj];
        const float4 Cv = sC[jj];
        const uint32_t rx = __float_as_uint(Bv.w), ry = __float_as_uint(Cv.w);
        const int x0 = (int)(rx & 0xFFFFu), x1 = (int)(rx >> 16);
        const int y0 = (int)(ry & 0xFFFFu), y1 = (int)(ry >> 16);
        // inside [x0, x1] as one unsigned compare (a pixel left of x0 wraps to a large value)
        const unsigned rw = (unsigned)(x1 - x0), rh = (unsigned)(y1 - y0);
        bool cin[kSlotCols<PPT>], rin[kSlotRows<PPT>], anyc = false, anyr = false;
#pragma unroll
        for (int c = 0; c < kSlotCols<PPT>; ++c) {
          cin[c] = (unsigned)(ti.x + 8 * c - x0) <= rw;
          anyc |= cin[c];
        }
#pragma unroll
        for (int r = 0; r < kSlotRows<PPT>; ++r) {
          rin[r] = (unsigned)(ti.y + 4 * r - y0) <= rh;
          anyr |= rin[r];
        }
        if (anyc && anyr) {
          const float4 Av = sA[jj];
          const ColTerms ct0 = col_terms(Av, pcx0), ct1 = col_terms(Av, pcx1);
#pragma unroll
          for (int i = 0; i < PPT; ++i) {
            const int ci = slot_col<PPT>(i), ri = slot_row<PPT>(i);
            if (j > mylast[i] || !cin[ci] || !rin[ri]) continue;
            if (kCount) ++n_pixb;
            const ColTerms& ct = ci ? ct1 : ct0;
            float alpha, ex, dy;
            bool cl;
            if (!pixel_alpha(ct, Av.y, Bv.x, Bv.y, (float)(ti.y + 4 * ri) + 0.5f, amin, amax, alpha,
                             ex, dy, cl))
              continue;
            if (kCount) ++n_actb;
            act = true;
            const float rinv = rcp_approx(1.0f - alpha);
            const float Ti = T[i] * rinv;
            const float aT = alpha * Ti;
            const float4 q = gq[i * NTH];
            gr = fmaf(q.x, aT, gr);
            gg = fmaf(q.y, aT, gg);
            gb = fmaf(q.z, aT, gb);
            const float qc = fmaf(q.z, Cv.z, fmaf(q.y, Cv.y, q.x * Cv.x));  // dL/dC^m . c_i
            const float ga = fmaf(Ti, qc, W[i] * rinv);                      // dL/dalpha_i
            // dL/do = ga e^power and dL/dpower = o ga e^power where alpha is not clamped,
            // 0 where it is; the moments are of ga e^power (the projection adjoint applies o)
            const float ge = cl ? 0.0f : ga * ex;
            go += ge;
            const float px = ge * ct.dx, py = ge * dy;
            sx += px;
            sy += py;
            sxx = fmaf(px, ct.dx, sxx);
            sxy = fmaf(px, dy, sxy);
            syy = fmaf(py, dy, syy);
            W[i] = fmaf(-qc, aT, W[i]);
            T[i] = Ti;
          }
        }
      }
      const unsigned am = __ballot_sync(0xffffffffu, act);
      if (am) {
        if (__popc(am) <= kDirectLanes) {
          // up to kDirectLanes lanes hold the warp's contribution: their own atomics cost
          // the L2 more operations than the reduction's nine but skip its shuffles, and
          // the kernel is bound by instruction issue, not by the L2
          if (act) {
            float4* dst = g2 + (int64_t)sG[jj] * 3;
            atomicAdd(dst, make_float4(sx, sy, sxx, sxy));
            atomicAdd(dst + 1, make_float4(syy, go, gr, gg));
            atomicAdd(&dst[2].x, gb);
          }
        } else {
          float v[9] = {sx, sy, sxx, sxy, syy, go, gr, gg, gb};
          float mine, v8;
          warp_reduce9(v, lane, mine, v8);
          // lanes 0, 4, ..., 28 hold the sums of values 0..7, lane 0 also value 8; the
          // 2-D gradient record is 12 floats (sx, sy, sxx, sxy, syy, go, gr, gg, gb, -, -, -)
          float* dst = reinterpret_cast<float*>(g2 + (int64_t)sG[jj] * 3);
          if ((lane & 3) == 0) atomicAdd(dst + (lane >> 2), mine);
          if (lane == 0) atomicAdd(dst + 8, v8);
        }
      }
    }
  }
  if (kCount) {
    flush_counter(b.counters, 3, n_evalb);
    flush_counter(b.counters, 4, n_pixb);
    flush_counter(b.counters, 5, n_actb);
  }
}

// One CTA per work item, or (kPersist) a grid sized to the SMs whose CTAs take work items
// in order from a device counter until none is left.
// (16x16 tiles: 128 threads held to 48 registers, 10 resident CTAs per SM; 32x32 tiles:
// 256 threads at 64 registers, 4 CTAs)
template <int TS>
constexpr int kMinBlocksFwd = TS == 16 ? 10 : (TS == 32 ? 4 : 1);

template <int TS, int PPT, bool kCount, bool kPersist>
__global__ void __launch_bounds__(TS * TS / PPT, kMinBlocksFwd<TS>) k_raster_fwd(const BatchDev b) {
  __shared__ float4 sA[kNB], sB[kNB], sC[kNB];
  __shared__ uint32_t sL[(TS * TS / PPT / 32) * kNB];  // per-warp compacted entry lists
  if constexpr (!kPersist) {
    fwd_item<TS, PPT, kCount>(b, item_of(b, blockIdx.x), sA, sB, sC, sL);
  } else {
    __shared__ long long s_id;
    for (;;) {
      __syncthreads();  // the previous item is done with shared memory and s_id
      if (threadIdx.x == 0) s_id = (long long)atomicAdd(b.work_ctr, 1ull);
      __syncthreads();
      const int64_t id = s_id;
      if (id >= items_of_launch(b)) return;
      fwd_item<TS, PPT, kCount>(b, item_of(b, id), sA, sB, sC, sL);
    }
  }
}

// Second forward of the items the first one handed back (b.retry, after their full sort):
// a fixed grid whose CTAs take the list's items in a grid-stride loop (few items, each a
// long walk: no register cap for occupancy).
template <int TS, int PPT, bool kCount>
__global__ void __launch_bounds__(TS * TS / PPT) k_raster_fwd_retry(const BatchDev b) {
  __shared__ float4 sA[kNB], sB[kNB], sC[kNB];
  __shared__ uint32_t sL[(TS * TS / PPT / 32) * kNB];
  const unsigned n = *b.retry_count;
  for (unsigned w = blockIdx.x; w < n; w += gridDim.x) {
    __syncthreads();  // the previous item is done with shared memory
    fwd_item<TS, PPT, kCount>(b, (int64_t)b.retry[w], sA, sB, sC, sL);
  }
}

template <int TS, int PPT, bool kCount, bool kPersist>
__global__ void __launch_bounds__(TS * TS / PPT, (kMinBlocksBwd<TS, PPT>)) k_raster_bwd(const BatchDev b) {
  __shared__ float4 sA[kNBBwd<TS, PPT>], sB[kNBBwd<TS, PPT>], sC[kNBBwd<TS, PPT>];
  __shared__ uint32_t sG[kNBBwd<TS, PPT>];
  __shared__ float4 sQ[TS * TS];  // composite adjoint per pixel slot
  __shared__ int s_maxlast;
  if constexpr (!kPersist) {
    bwd_item<TS, PPT, kCount>(b, blockIdx.x, sA, sB, sC, sG, s_maxlast, sQ);
  } else {
    __shared__ long long s_id;
    for (;;) {
      __syncthreads();
      if (threadIdx.x == 0) s_id = (long long)atomicAdd(b.work_ctr + 1, 1ull);
      __syncthreads();
      const int64_t id = s_id;
      if (id >= b.n_tiles) return;
      bwd_item<TS, PPT, kCount>(b, id, sA, sB, sC, sG, s_maxlast, sQ);
    }
  }
}

// Tile side -> pixels per thread.  Forward: 2 (8 x 8 regions per warp) for 8x8 and 16x16
// tiles, 4 for 32x32; backward: 2 for 8x8, 8 (one warp per 16x16 tile) for 16x16, 4 (16 x 8
// regions) for 32x32.  At 16x16 the forward's smaller per-thread state gives 40 resident
// warps per SM instead of 30 and beats the 4-pixel mapping (15.8 vs 17.1 ms on the 10M
// step); the backward's per-entry work (record loads, rectangle tests, the warp reduction
// and its atomics) favours more pixels per lane: one warp per tile does it once per entry
// instead of twice (21.0 ms at 8 pixels and 27 CTAs per SM, 22.0 at 4, 29.2 at 2).
template <int TS>
struct PptFwd {
  static constexpr int value = TS == 32 ? 4 : 2;
};
template <int TS>
struct PptBwd {
  static constexpr int value = TS == 8 ? 2 : (TS == 16 ? 8 : 4);
};

// Work is counted only by eager runs with a counter buffer: a captured graph launches the
// plain variants, so replays carry no counting instructions (and keep the eager counts).
static bool counting(const BatchDev& b, cudaStream_t s) {
  return b.counters && !stream_capturing(s);
}

template <int TS, bool kCount, bool kPersist>
static void launch_fwd_k(const BatchDev& b, cudaStream_t s) {
  constexpr int P = PptFwd<TS>::value;
  const int64_t items = b.order ? b.item_n : b.n_tiles;
  const unsigned grid = kPersist ? (unsigned)std::min<int64_t>(items, (int64_t)b.persist_grid)
                                 : (unsigned)items;
  k_raster_fwd<TS, P, kCount, kPersist><<<grid, TS * TS / P, 0, s>>>(b);
}
template <int TS, bool kCount, bool kPersist>
static void launch_bwd_k(const BatchDev& b, cudaStream_t s) {
  constexpr int P = PptBwd<TS>::value;
  const unsigned grid = kPersist ? (unsigned)std::min<int64_t>(b.n_tiles, (int64_t)b.persist_grid)
                                 : (unsigned)b.n_tiles;
  k_raster_bwd<TS, P, kCount, kPersist><<<grid, TS * TS / P, 0, s>>>(b);
}
template <int TS>
static void launch_fwd_t(const BatchDev& b, cudaStream_t s) {
  const bool c = counting(b, s), p = b.persist_grid > 0 && b.work_ctr;
  if (p) cudaMemsetAsync(b.work_ctr, 0, sizeof(unsigned long long), s);
  if (c) { if (p) launch_fwd_k<TS, true, true>(b, s); else launch_fwd_k<TS, true, false>(b, s); }
  else   { if (p) launch_fwd_k<TS, false, true>(b, s); else launch_fwd_k<TS, false, false>(b, s); }
}
template <int TS>
static void launch_bwd_t(const BatchDev& b, cudaStream_t s) {
  const bool c = counting(b, s), p = b.persist_grid > 0 && b.work_ctr;
  if (p) cudaMemsetAsync(b.work_ctr + 1, 0, sizeof(unsigned long long), s);
  if (c) { if (p) launch_bwd_k<TS, true, true>(b, s); else launch_bwd_k<TS, true, false>(b, s); }
  else   { if (p) launch_bwd_k<TS, false, true>(b, s); else launch_bwd_k<TS, false, false>(b, s); }
}

template <int TS>
static int max_ctas_t(bool bwd) {
  constexpr int PF = PptFwd<TS>::value, PB = PptBwd<TS>::value;
  int n = 0;
  cudaError_t e =
      bwd ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_raster_bwd<TS, PB, false, true>,
                                                          TS * TS / PB, 0)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_raster_fwd<TS, PF, false, true>,
                                                          TS * TS / PF, 0);
  return e == cudaSuccess ? n : 0;
}

int raster_max_ctas_per_sm(int tile, bool bwd) {
  switch (tile) {
    case 8: return max_ctas_t<8>(bwd);
    case 32: return max_ctas_t<32>(bwd);
    default: return max_ctas_t<16>(bwd);
  }
}

void launch_raster_fwd(const BatchDev& b, cudaStream_t s) {
  if (b.n_tiles == 0) return;
  switch (b.tile) {
    case 8: launch_fwd_t<8>(b, s); break;
    case 32: launch_fwd_t<32>(b, s); break;
    default: launch_fwd_t<16>(b, s); break;
  }
  count_launch();
}

template <int TS>
static void launch_fwd_retry_t(const BatchDev& b, cudaStream_t s) {
  constexpr int P = PptFwd<TS>::value;
  const unsigned grid = (unsigned)device_sm_count() * 2;
  if (counting(b, s)) k_raster_fwd_retry<TS, P, true><<<grid, TS * TS / P, 0, s>>>(b);
  else k_raster_fwd_retry<TS, P, false><<<grid, TS * TS / P, 0, s>>>(b);
}

void launch_raster_fwd_retry(const BatchDev& b, cudaStream_t s) {
  if (!b.sel || b.n_tiles == 0) return;
  switch (b.tile) {
    case 8: launch_fwd_retry_t<8>(b, s); break;
    case 32: launch_fwd_retry_t<32>(b, s); break;
    default: launch_fwd_retry_t<16>(b, s); break;
  }
  count_launch();
}

void launch_raster_bwd(const BatchDev& b, cudaStream_t s) {
  if (b.n_tiles == 0) return;
  switch (b.tile) {
    case 8: launch_bwd_t<8>(b, s); break;
    case 32: launch_bwd_t<32>(b, s); break;
    default: launch_bwd_t<16>(b, s); break;
  }
  count_launch();
}

}  // namespace splx
