// FP32 binning specification on the GPU.
//
// The discrete structure of the render (cull decision, integer 3-sigma pixel
// rectangle, tile rectangle, depth sort key) must match the CPU reference bit for bit,
// so it is computed here with explicitly rounded IEEE operations (__fmul_rn, __fadd_rn,
// __fsub_rn, __fdiv_rn, __fsqrt_rn: no contraction into FMA, no approximate division)
// in a fixed evaluation order.  Projection follows Sec. 2 step 1: Sigma2D = J W Sigma
// W^T J^T with Sigma = R S S^T R^T, plus a 0.3 px^2 low-pass dilation; the determinant
// uses the Cauchy-Binet sum of squared 2x2 minors so it never cancels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace splx {

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }

// Exponential from basic operations only: Cody-Waite range reduction with ln 2 split
// as in Moshier's Cephes library, degree-7 Taylor polynomial of e^r (Horner), exact
// power-of-two scaling.  Within a few ulp of e^x on [-87, 88].
__device__ __forceinline__ float exp_spec(float x) {
  x = fminf(fmaxf(x, -87.0f), 88.0f);
  const float k = rintf(fm(x, 1.44269502f));
  float r = fs(x, fm(k, 0.693359375f));
  r = fs(r, fm(k, -2.12194440e-4f));
  float p = 1.98412698e-4f;
  p = fa(fm(p, r), 1.38888889e-3f);
  p = fa(fm(p, r), 8.33333377e-3f);
  p = fa(fm(p, r), 4.16666679e-2f);
  p = fa(fm(p, r), 1.66666672e-1f);
  p = fa(fm(p, r), 0.5f);
  p = fa(fm(p, r), 1.0f);
  p = fa(fm(p, r), 1.0f);
  const float scale = __int_as_float(((int)k + 127) << 23);
  return fm(p, scale);
}

struct SpecOut {
  bool visible;
  int x0, x1, y0, y1;
  float tz;         // camera depth (its bits are the sort key)
  float tx, ty;     // camera-space x, y
  float ex, ey, ez; // rounding errors of tx, ty, tz (for the blend's centre, not the spec)
  float u, v;       // 2-D mean
  float a, b, c;    // dilated Sigma2D
  float det;        // det(Sigma2D)
  float sx, sy, sz; // activated scales
};

// View-independent part of the specification: M = R(q) diag(exp(log_scale)).  `ok` is
// false for a zero quaternion (never visible).
struct SpecG {
  bool ok;
  float M[9];
  float sx, sy, sz;
};

__device__ __forceinline__ SpecG spec_gaussian(const float ls[3], const float q[4]) {
  SpecG G;
  G.ok = false;
  G.sx = G.sy = G.sz = 0.0f;
  const float qn = fa(fa(fa(fm(q[0], q[0]), fm(q[1], q[1])), fm(q[2], q[2])), fm(q[3], q[3]));
  if (!(qn > 0.0f)) return G;
  G.ok = true;
  const float inv = fd(1.0f, __fsqrt_rn(qn));
  const float w = fm(q[0], inv), x = fm(q[1], inv), y = fm(q[2], inv), z = fm(q[3], inv);
  float Rq[9];
  Rq[0] = fs(1.0f, fm(2.0f, fa(fm(y, y), fm(z, z))));
  Rq[1] = fm(2.0f, fs(fm(x, y), fm(w, z)));
  Rq[2] = fm(2.0f, fa(fm(x, z), fm(w, y)));
  Rq[3] = fm(2.0f, fa(fm(x, y), fm(w, z)));
  Rq[4] = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(z, z))));
  Rq[5] = fm(2.0f, fs(fm(y, z), fm(w, x)));
  Rq[6] = fm(2.0f, fs(fm(x, z), fm(w, y)));
  Rq[7] = fm(2.0f, fa(fm(y, z), fm(w, x)));
  Rq[8] = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(y, y))));
  const float s[3] = {exp_spec(ls[0]), exp_spec(ls[1]), exp_spec(ls[2])};
  G.sx = s[0]; G.sy = s[1]; G.sz = s[2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) G.M[3 * i + j] = fm(Rq[3 * i + j], s[j]);
  return G;
}

// Per-view part; cam: R[9], t[3], fx, fy, cx, cy, W, H, near.
// Knuth's TwoSum: s = fl(a + b) and its exact rounding error e (s + e = a + b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = fa(a, b);
  const float bb = fs(s, a);
  e = fa(fs(a, fs(s, bb)), fs(b, bb));
}

// Camera-space position of a mean in the specification's arithmetic,
// t_i = ((R_i0 m_0 + R_i1 m_1) + R_i2 m_2) + tc_i, each step rounded.  err, if the caller
// uses it, receives the sum of those steps' exact rounding errors (Dot2 of Ogita, Rump and
// Oishi, "Accurate sum and dot product", 2005: products split by an FMA, sums by TwoSum),
// so that t_i + err_i is R m + tc to about twice the precision; it is not part of the
// specification and leaves t_i as it is.
__device__ __forceinline__ void spec_camera(const float m[3], const float* R, const float* tc,
                                            float t[3], float err[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float p0 = fm(R[3 * i], m[0]), p1 = fm(R[3 * i + 1], m[1]), p2 = fm(R[3 * i + 2], m[2]);
    float s1, s2, s3, e1, e2, e3;
    two_sum(p0, p1, s1, e1);
    two_sum(s1, p2, s2, e2);
    two_sum(s2, tc[i], s3, e3);
    const float ep = fa(fa(__fmaf_rn(R[3 * i], m[0], -p0), __fmaf_rn(R[3 * i + 1], m[1], -p1)),
                        __fmaf_rn(R[3 * i + 2], m[2], -p2));
    t[i] = s3;
    err[i] = fa(ep, fa(fa(e1, e2), e3));
  }
}
// Its 2-D mean (the centre of the pixel rectangle).
__device__ __forceinline__ void spec_center(float tx, float ty, float tz, float fx, float fy,
                                            float cx, float cy, float& u, float& v) {
  u = fa(fd(fm(fx, tx), tz), cx);
  v = fa(fd(fm(fy, ty), tz), cy);
}

__device__ __forceinline__ SpecOut bin_spec(const float m[3], const SpecG& G, const float* R,
                                            const float* tc, float fx, float fy, float cx,
                                            float cy, int W, int H, float near_plane) {
  SpecOut o;
  o.visible = false;
  o.x0 = 0; o.x1 = -1; o.y0 = 0; o.y1 = -1;
  float t[3], terr[3];
  spec_camera(m, R, tc, t, terr);
  const float tx = t[0], ty = t[1], tz = t[2];
  o.ex = terr[0]; o.ey = terr[1]; o.ez = terr[2];
  o.tz = tz; o.tx = tx; o.ty = ty;
  o.sx = G.sx; o.sy = G.sy; o.sz = G.sz;
  if (!(tz > near_plane)) return o;
  if (!G.ok) return o;
  {
    // Early exit, outside the specification (it only leaves out work): the rectangle is
    // empty when the 2-D mean lies farther outside the image than a bound on the radius.
    // The dilated covariance's largest eigenvalue is at most |J|_F^2 s_max^2 (the view and
    // the Gaussian's rotations are orthonormal up to FP32 rounding) + 0.6 (the dilation of
    // both diagonal entries) + 0.32 (the 0.1 floor under the root), and
    // |J|_F^2 <= (fx^2 (1 + limx^2) + fy^2 (1 + limy^2)) / tz^2 with the clamped x/z, y/z,
    // where fx limx = 0.65 W; a 0.5 % and 2-pixel margin covers rounding, the approximate
    // reciprocal, root and 2-D mean used here, and the ceil.
    const float smax = fmaxf(fmaxf(G.sx, G.sy), G.sz);
    const float itz = __fdividef(1.0f, tz);
    const float k2 = fx * fx + fy * fy + 0.4225f * ((float)W * (float)W + (float)H * (float)H);
    const float q = 1.005f * k2 * itz * itz * smax * smax + 0.93f;
    const float rb = 3.0f * q * rsqrtf(q) + 2.0f;
    const float u0 = fx * tx * itz + cx, v0 = fy * ty * itz + cy;
    if (u0 + rb < 0.0f || u0 - rb > (float)W || v0 + rb < 0.0f || v0 - rb > (float)H) return o;
  }
  const float* M = G.M;
  float V[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      V[3 * i + j] = fa(fa(fm(R[3 * i + 0], M[j]), fm(R[3 * i + 1], M[3 + j])),
                        fm(R[3 * i + 2], M[6 + j]));
  const float limx = fd(fm(1.3f, fm(0.5f, (float)W)), fx);
  const float limy = fd(fm(1.3f, fm(0.5f, (float)H)), fy);
  const float rx = fminf(limx, fmaxf(-limx, fd(tx, tz)));
  const float ry = fminf(limy, fmaxf(-limy, fd(ty, tz)));
  const float j00 = fd(fx, tz);
  const float j02 = -fd(fm(fx, rx), tz);
  const float j11 = fd(fy, tz);
  const float j12 = -fd(fm(fy, ry), tz);
  float P0[3], P1[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    P0[j] = fa(fm(j00, V[j]), fm(j02, V[6 + j]));
    P1[j] = fa(fm(j11, V[3 + j]), fm(j12, V[6 + j]));
  }
  const float a0 = fa(fa(fm(P0[0], P0[0]), fm(P0[1], P0[1])), fm(P0[2], P0[2]));
  const float c0 = fa(fa(fm(P1[0], P1[0]), fm(P1[1], P1[1])), fm(P1[2], P1[2]));
  const float b0 = fa(fa(fm(P0[0], P1[0]), fm(P0[1], P1[1])), fm(P0[2], P1[2]));
  const float d01 = fs(fm(P0[0], P1[1]), fm(P0[1], P1[0]));
  const float d02 = fs(fm(P0[0], P1[2]), fm(P0[2], P1[0]));
  const float d12 = fs(fm(P0[1], P1[2]), fm(P0[2], P1[1]));
  const float det0 = fa(fa(fm(d01, d01), fm(d02, d02)), fm(d12, d12));
  const float a = fa(a0, 0.3f), c = fa(c0, 0.3f);
  const float det = fa(fa(det0, fm(0.3f, fa(a0, c0))), 0.09f);
  o.a = a; o.b = b0; o.c = c; o.det = det;
  if (!(det > 0.0f)) return o;
  const float mid = fm(0.5f, fa(a, c));
  const float lam = fa(mid, __fsqrt_rn(fmaxf(0.1f, fs(fm(mid, mid), det))));
  if (!(lam < 1.0e30f)) return o;
  const float r = ceilf(fm(3.0f, __fsqrt_rn(lam)));
  if (!(r > 0.0f)) return o;
  float u, v;
  spec_center(tx, ty, tz, fx, fy, cx, cy, u, v);
  o.u = u; o.v = v;
  if (!(fabsf(u) < 1.0e7f) || !(fabsf(v) < 1.0e7f)) return o;
  const float xlo = ceilf(fs(fs(u, r), 0.5f)), xhi = floorf(fs(fa(u, r), 0.5f));
  const float ylo = ceilf(fs(fs(v, r), 0.5f)), yhi = floorf(fs(fa(v, r), 0.5f));
  const float x0 = fmaxf(xlo, 0.0f), x1 = fminf(xhi, (float)(W - 1));
  const float y0 = fmaxf(ylo, 0.0f), y1 = fminf(yhi, (float)(H - 1));
  if (x0 > x1 || y0 > y1) return o;
  o.visible = true;
  o.x0 = (int)x0; o.x1 = (int)x1; o.y0 = (int)y0; o.y1 = (int)y1;
  return o;
}

// ---- the blend's 2-D mean, outside the specification ----------------------------------
// The specification's u, v round each of its steps, so with a mean hundreds of metres from
// the camera they can be off by several 1e-4 pixels, which a footprint of a pixel turns
// into alpha errors of that order.  The blend therefore takes u = fx (tx + ex)/(tz + ez) + cx
// (and v alike) from the camera-space position with its rounding errors (spec_camera),
// the quotient with its remainder and one final rounding: within half an ulp of the exact
// projection of the FP32 inputs.
__device__ __forceinline__ float project_df(float f, float nh, float nl, float dh, float dl,
                                            float c) {
  const float q = fd(nh, dh);
  // remainder n - q d: exact for the high parts, then the low parts
  float r = __fmaf_rn(-q, dh, nh);
  r = fa(r, fs(nl, fm(q, dl)));
  const float ql = fd(r, dh);
  const float p = fm(f, q);
  const float pe = __fmaf_rn(f, ql, __fmaf_rn(f, q, -p));
  float s, e;
  two_sum(p, c, s, e);
  return fa(s, fa(e, pe));
}
__device__ __forceinline__ void blend_center(const SpecOut& so, float fx, float fy, float cx,
                                             float cy, float& u, float& v) {
  u = project_df(fx, so.tx, so.ex, so.tz, so.ez, cx);
  v = project_df(fy, so.ty, so.ey, so.tz, so.ez, cy);
}

// Conic of the dilated Sigma2D and opacity in the specification's arithmetic.
__device__ __forceinline__ void spec_conic(const SpecOut& so, float& A, float& B, float& C) {
  A = fd(so.c, so.det);
  B = -fd(so.b, so.det);
  C = fd(so.a, so.det);
}
__device__ __forceinline__ float spec_opacity(float logit) {
  return fd(1.0f, fa(1.0f, exp_spec(-logit)));
}

// Natural logarithm of x >= 1 from basic operations only: x = m 2^e with m in
// [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s), s = (m - 1)/(m + 1), by its odd series through
// s^9, and ln 2 split as in exp_spec.
__device__ __forceinline__ float log_spec(float x) {
  uint32_t bits = __float_as_uint(x);
  int e = (int)(bits >> 23) - 127;
  float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
  if (m > 1.41421354f) { m = fm(m, 0.5f); e += 1; }
  const float s = fd(fs(m, 1.0f), fa(m, 1.0f));
  const float s2 = fm(s, s);
  float p = 0.222222222f;
  p = fa(fm(p, s2), 0.285714287f);
  p = fa(fm(p, s2), 0.400000006f);
  p = fa(fm(p, s2), 0.666666687f);
  p = fa(fm(p, s2), 2.0f);
  const float fe = (float)e;
  return fa(fm(fe, 0.693359375f), fa(fm(s, p), fm(fe, -2.12194440e-4f)));
}

// Tile culling, part of the binning specification.  A (Gaussian, tile) pair is listed
// only if the conic's quadratic form q = A x^2 + 2B xy + C y^2 (offsets from the mean)
// reaches q_max = 2 ln(o / (0.999 alpha_min)) on the box spanned by the pixel centres the
// Gaussian's rectangle [x0,x1]x[y0,y1] shares with the tile, i.e. only if alpha can reach
// 0.999 alpha_min there; the 0.1% margin makes every culled pair one that the per-pixel
// alpha >= alpha_min test rejects at every pixel.  The minimum of the convex q over the
// box is 0 if the mean lies inside, else it lies on an edge whose outer side holds the
// mean, at the clamped stationary point of that edge.  q_max < 0 marks a Gaussian with
// o < 0.999 alpha_min, which reaches no tile.
struct TileCull {
  float u, v, A, B, C, qmax, rBC, rBA;
};

__device__ __forceinline__ float tile_cull_qmax(float o, float amin) {
  const float thr = fm(amin, 0.999f);
  if (!(o >= thr)) return -1.0f;
  return fm(2.0f, log_spec(fd(o, thr)));
}

__device__ __forceinline__ TileCull tile_cull_prep(float u, float v, float A, float B, float C,
                                                   float qmax) {
  TileCull t;
  t.u = u; t.v = v; t.A = A; t.B = B; t.C = C; t.qmax = qmax;
  t.rBC = fd(B, C);
  t.rBA = fd(B, A);
  return t;
}

__device__ __forceinline__ bool tile_hits_spec(const TileCull& t, int x0, int x1, int y0, int y1,
                                               int tx, int ty, int T) {
  if (!(t.qmax >= 0.0f)) return false;
  const int px0 = max(tx * T, x0), px1 = min(tx * T + T - 1, x1);
  const int py0 = max(ty * T, y0), py1 = min(ty * T + T - 1, y1);
  const float xa = fs(fa((float)px0, 0.5f), t.u), xb = fs(fa((float)px1, 0.5f), t.u);
  const float ya = fs(fa((float)py0, 0.5f), t.v), yb = fs(fa((float)py1, 0.5f), t.v);
  const bool xout = xa > 0.0f || xb < 0.0f, yout = ya > 0.0f || yb < 0.0f;
  if (!xout && !yout) return true;  // q = 0 at the mean
  const float twoB = fm(2.0f, t.B);
  float q = __int_as_float(0x7f800000);
  if (xout) {
    const float x = xa > 0.0f ? xa : xb;
    const float y = fminf(fmaxf(-fm(t.rBC, x), ya), yb);
    q = fa(fa(fm(fm(t.A, x), x), fm(fm(twoB, x), y)), fm(fm(t.C, y), y));
  }
  if (yout) {
    const float y = ya > 0.0f ? ya : yb;
    const float x = fminf(fmaxf(-fm(t.rBA, y), xa), xb);
    q = fminf(q, fa(fa(fm(fm(t.A, x), x), fm(fm(twoB, x), y)), fm(fm(t.C, y), y)));
  }
  return q <= t.qmax;
}

}  // namespace splx
