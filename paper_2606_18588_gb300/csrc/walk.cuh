// Balanced walk over a warp's (lane, j) tasks, j < cnt of that lane: the projection's and
// the fill's loops over the tiles of each lane's Gaussian.  A loop to the warp's largest
// count leaves most lanes idle (on the 10M workload the largest of 32 counts is about three
// times their mean); here every round gives each active lane one task of the warp's
// concatenated list, so the walk takes ceil(total / lanes) rounds.
#pragma once

#include <cuda_runtime.h>

namespace splx {

struct WarpWalk {
  unsigned lanes;  // active lanes (0 .. nact-1)
  int nact, lane, cnt, pre, total;
};

// Exclusive prefix of the counts over the active lanes.
__device__ __forceinline__ WarpWalk warp_walk_begin(unsigned lanes, int cnt) {
  WarpWalk w;
  w.lanes = lanes;
  w.nact = __popc(lanes);
  w.lane = (int)(threadIdx.x & 31);
  w.cnt = cnt;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(lanes, incl, o);
    if (w.lane >= o) incl += n;
  }
  w.pre = incl - cnt;
  w.total = __shfl_sync(lanes, incl, w.nact - 1);
  return w;
}

// The task of this lane in the round that starts at list position `base`: returns the
// owning lane (or -1 past the end) and sets j.  Lanes whose range starts inside the round
// mark their first position; a position's owner is the last mark at or before it, or the
// lane whose range runs into the round.  s_own: 32 ints of this warp's shared memory.
// Orders this warp's earlier shared-memory writes before its later reads.
__device__ __forceinline__ int warp_walk_owner(const WarpWalk& w, int base, int* s_own, int& j) {
  const bool starts = w.cnt > 0 && w.pre >= base && w.pre < base + w.nact;
  if (starts) s_own[w.pre - base] = w.lane;
  const unsigned marks = __reduce_or_sync(w.lanes, starts ? 1u << (w.pre - base) : 0u);
  const unsigned carry = __ballot_sync(w.lanes, w.cnt > 0 && w.pre < base && w.pre + w.cnt > base);
  __syncwarp(w.lanes);
  const int q = base + w.lane;
  int owner = -1;
  if (q < w.total) {
    const unsigned le = marks & (0xFFFFFFFFu >> (31 - w.lane));
    owner = le ? s_own[31 - __clz(le)] : __ffs(carry) - 1;
  }
  const int opre = __shfl_sync(w.lanes, w.pre, owner < 0 ? w.lane : owner);
  j = q - opre;
  __syncwarp(w.lanes);  // s_own is rewritten by the next round
  return owner;
}

// j = jy * tw + jx for a rectangle tw tiles wide (rcp_tw = 1/tw; exact for j < 2^21).
__device__ __forceinline__ void walk_tile(int j, int tw, float rcp_tw, int& jx, int& jy) {
  jy = (int)(((float)j + 0.5f) * rcp_tw);
  jx = j - jy * tw;
}

}  // namespace splx
