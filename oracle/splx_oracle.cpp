// Splaxel hot path: plain, slow, FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this library: only
// the tests, the smoke check and the benchmark's CPU-baseline leg load it.  It shares no
// code, header, table or constant with the CUDA path.
//
// What it computes (paper passages in brackets):
//   * FP32 binning specification: near-plane cull, EWA 2-D covariance, 3-sigma pixel
//     rectangle, tile rectangle and depth key, in IEEE basic operations with a fixed
//     evaluation order and no contraction (built with -ffp-contract=off) so that the
//     GPU's independent implementation can be compared bit for bit [Sec. 2, steps 1-2].
//   * FP64 projection: mean, EWA covariance Sigma2D = J W Sigma W^T J^T, conic, SH colour,
//     opacity [Sec. 2 step 1; Theta_i = {mu, R, S, o, c}].
//   * FP64 local render of one subset into premultiplied colour C^m, transmittance T^m
//     and alpha-weighted depth D^m [Eq. 1-4].
//   * FP64 global composition of K partials in per-pixel depth order [Eq. 5].
//   * FP64 backward through Eq. 5 and the local render [Eq. 6-7] and the projection.
//   * FP64 Adam.
//
// Readings of the paper used here (the paper leaves these to "standard 3DGS"):
//   D^m = sum_i d_i alpha_i T_i (Eq. 4 as printed omits alpha_i); subsets are ordered per
//   pixel by the normalised depth D^m / (1 - T^m), ties to the lower subset index, empty
//   subsets last; pixel centres at +0.5; a Gaussian touches only the pixels of its integer
//   3-sigma rectangle; alpha in [1/255, 0.99]; a pixel stops before the Gaussian that would
//   take its transmittance below eps_T; colour = max(0, SH + 0.5).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

typedef struct {
  float R[9];   // world -> camera rotation, row-major
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float near_plane;
} orc_camera;

typedef struct {
  int32_t tile;          // tile side in pixels
  double eps_T;          // local-render termination threshold on transmittance
  double eps_comp;       // composition saturation threshold on the prefix transmittance
  double alpha_min, alpha_max;
  double bg[3];
  // Ambiguity margins: a pixel whose result hinges on a decision closer than this to
  // its threshold is flagged, because FP32 and FP64 may legitimately take either side.
  double amb_alpha;      // relative margin on alpha vs alpha_min
  double amb_power;      // relative margin on the sign of the Gaussian exponent
  double amb_T;          // relative margin on T*(1-alpha) vs eps_T and prefix vs eps_comp
  double amb_key;        // relative margin between two subsets' composite keys
} orc_opts;

typedef struct {
  const double *means, *log_scales, *quats, *opacity_logits, *sh;
  int64_t n;
  int32_t sh_degree;
} orc_params;

typedef struct {
  double *means, *log_scales, *quats, *opacity_logits, *sh;
} orc_grads;

// Flip bounds of a render (every pointer nullable).  On a pixel with an ambiguous decision
// an FP32 implementation may legitimately take the other side; these bound how far that
// moves each output (blend_pixel and composite_bounds say how they are derived).
typedef struct {
  double* image;   // [H][W] bound on |delta| of each channel of the composited image
  double* T;       // [H][W] bound on |delta| of the composited transmittance
  double* partC;   // [K][H][W] per partial: |delta C^m| <= partC cmax, |delta D^m| <= partC dmax
  double* partT;   // [K][H][W] per partial: |delta T^m| <= partT
  double cmax;     // out: largest colour channel of a visible Gaussian (and of the background)
  double dmax;     // out: largest depth of a visible Gaussian
} orc_bounds;

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------------
// FP32 binning specification.  Every line is one correctly rounded IEEE operation in
// the order written; the CUDA side implements the same specification independently.
// ---------------------------------------------------------------------------------

// Fixed-formula exponential from basic operations (Cody-Waite reduction with a split
// ln 2 as in Moshier's Cephes expf, then the degree-7 Taylor polynomial of e^r in
// Horner form, then an exact power-of-two scale).  Only used where a value feeds the
// discrete pixel rectangle, so that both sides agree bit for bit.
float exp_spec(float x) {
  x = std::fmin(std::fmax(x, -87.0f), 88.0f);
  const float k = std::rint(x * 1.44269502f);
  float r = x - k * 0.693359375f;
  r = r - k * -2.12194440e-4f;
  float p = 1.98412698e-4f;            // 1/7!
  p = p * r + 1.38888889e-3f;          // 1/6!
  p = p * r + 8.33333377e-3f;          // 1/5!
  p = p * r + 4.16666679e-2f;          // 1/4!
  p = p * r + 1.66666672e-1f;          // 1/3!
  p = p * r + 0.5f;                    // 1/2!
  p = p * r + 1.0f;
  p = p * r + 1.0f;
  const int ki = (int)k;
  uint32_t bits = (uint32_t)(ki + 127) << 23;
  float scale;
  std::memcpy(&scale, &bits, 4);
  return p * scale;
}

struct BinRec {
  int visible;
  int x0, x1, y0, y1;     // inclusive pixel rectangle, clipped to the image
  uint32_t depth_bits;    // bit pattern of the FP32 camera-space depth
  float u, v;             // 2-D mean
  float A, B, C;          // conic of the dilated Sigma2D
  float o;                // opacity sigmoid(logit)
};

// Natural logarithm of x >= 1 from basic operations only: x = m 2^e with m in
// [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s) with s = (m - 1)/(m + 1) as its odd series
// through s^9 (truncation below 1e-9 for |s| <= 0.172), ln 2 split as in exp_spec.
float log_spec(float x) {
  uint32_t bits;
  std::memcpy(&bits, &x, 4);
  int e = (int)(bits >> 23) - 127;
  bits = (bits & 0x7FFFFFu) | 0x3F800000u;
  float m;
  std::memcpy(&m, &bits, 4);
  if (m > 1.41421354f) { m = m * 0.5f; e += 1; }
  const float s = (m - 1.0f) / (m + 1.0f);
  const float s2 = s * s;
  float p = 0.222222222f;
  p = p * s2 + 0.285714287f;
  p = p * s2 + 0.400000006f;
  p = p * s2 + 0.666666687f;
  p = p * s2 + 2.0f;
  const float fe = (float)e;
  return fe * 0.693359375f + (s * p + fe * -2.12194440e-4f);
}

// Tile culling, part of the binning specification.  A (Gaussian, tile) pair is listed
// only if the conic's quadratic form q = A x^2 + 2B xy + C y^2 (offsets from the mean)
// reaches q_max = 2 ln(o / (0.999 alpha_min)) somewhere on the box spanned by the pixel
// centres that the Gaussian's rectangle shares with the tile, i.e. only if alpha can
// reach 0.999 alpha_min there; the 0.1% margin makes every culled pair one that the
// per-pixel alpha >= alpha_min test rejects at every pixel of the tile.  The minimum of
// the convex q over the box is 0 if the mean lies inside; otherwise it lies on an edge
// whose outer side holds the mean, and along such an edge at the clamped stationary
// point.  TileCull holds the per-Gaussian part; a Gaussian with o < 0.999 alpha_min
// reaches no tile.
struct TileCull {
  bool any;
  float qmax, rBC, rBA;  // q_max, B/C, B/A
};

TileCull tile_cull_prep(const BinRec& b, float amin) {
  TileCull t{false, 0.0f, 0.0f, 0.0f};
  const float thr = amin * 0.999f;
  if (!(b.o >= thr)) return t;
  t.any = true;
  t.qmax = 2.0f * log_spec(b.o / thr);
  t.rBC = b.B / b.C;
  t.rBA = b.B / b.A;
  return t;
}

bool tile_hits_spec(const BinRec& b, const TileCull& t, int tx, int ty, int B_) {
  if (!t.any) return false;
  const int px0 = std::max(tx * B_, b.x0), px1 = std::min(tx * B_ + B_ - 1, b.x1);
  const int py0 = std::max(ty * B_, b.y0), py1 = std::min(ty * B_ + B_ - 1, b.y1);
  const float xa = ((float)px0 + 0.5f) - b.u, xb = ((float)px1 + 0.5f) - b.u;
  const float ya = ((float)py0 + 0.5f) - b.v, yb = ((float)py1 + 0.5f) - b.v;
  const bool xout = xa > 0.0f || xb < 0.0f, yout = ya > 0.0f || yb < 0.0f;
  if (!xout && !yout) return true;  // q = 0 at the mean
  const float twoB = 2.0f * b.B;
  float q = INFINITY;
  if (xout) {
    const float x = xa > 0.0f ? xa : xb;
    const float y = std::fmin(std::fmax(-(t.rBC * x), ya), yb);
    q = ((b.A * x) * x + (twoB * x) * y) + (b.C * y) * y;
  }
  if (yout) {
    const float y = ya > 0.0f ? ya : yb;
    const float x = std::fmin(std::fmax(-(t.rBA * y), xa), xb);
    q = std::fmin(q, ((b.A * x) * x + (twoB * x) * y) + (b.C * y) * y);
  }
  return q <= t.qmax;
}

BinRec bin_spec(const float m[3], const float ls[3], const float q[4], float logit,
                const orc_camera& c) {
  BinRec b{0, 0, -1, 0, -1, 0u, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  const float* R = c.R;
  const float tx = ((R[0] * m[0] + R[1] * m[1]) + R[2] * m[2]) + c.t[0];
  const float ty = ((R[3] * m[0] + R[4] * m[1]) + R[5] * m[2]) + c.t[1];
  const float tz = ((R[6] * m[0] + R[7] * m[1]) + R[8] * m[2]) + c.t[2];
  if (!(tz > c.near_plane)) return b;

  const float qn = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
  if (!(qn > 0.0f)) return b;
  const float inv = 1.0f / std::sqrt(qn);
  const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
  float Rq[9];
  Rq[0] = 1.0f - 2.0f * (y * y + z * z);
  Rq[1] = 2.0f * (x * y - w * z);
  Rq[2] = 2.0f * (x * z + w * y);
  Rq[3] = 2.0f * (x * y + w * z);
  Rq[4] = 1.0f - 2.0f * (x * x + z * z);
  Rq[5] = 2.0f * (y * z - w * x);
  Rq[6] = 2.0f * (x * z - w * y);
  Rq[7] = 2.0f * (y * z + w * x);
  Rq[8] = 1.0f - 2.0f * (x * x + y * y);
  const float s[3] = {exp_spec(ls[0]), exp_spec(ls[1]), exp_spec(ls[2])};
  float M[9];  // M = Rq diag(s)
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[3 * i + j] = Rq[3 * i + j] * s[j];
  float V[9];  // V = W M, W = camera rotation
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      V[3 * i + j] = (R[3 * i + 0] * M[j] + R[3 * i + 1] * M[3 + j]) + R[3 * i + 2] * M[6 + j];

  const float limx = (1.3f * (0.5f * (float)c.width)) / c.fx;
  const float limy = (1.3f * (0.5f * (float)c.height)) / c.fy;
  const float rx = std::fmin(limx, std::fmax(-limx, tx / tz));
  const float ry = std::fmin(limy, std::fmax(-limy, ty / tz));
  const float j00 = c.fx / tz;
  const float j02 = -(c.fx * rx) / tz;
  const float j11 = c.fy / tz;
  const float j12 = -(c.fy * ry) / tz;
  float P0[3], P1[3];  // P = J V (2x3)
  for (int j = 0; j < 3; ++j) {
    P0[j] = j00 * V[j] + j02 * V[6 + j];
    P1[j] = j11 * V[3 + j] + j12 * V[6 + j];
  }
  const float a0 = (P0[0] * P0[0] + P0[1] * P0[1]) + P0[2] * P0[2];
  const float c0 = (P1[0] * P1[0] + P1[1] * P1[1]) + P1[2] * P1[2];
  const float b0 = (P0[0] * P1[0] + P0[1] * P1[1]) + P0[2] * P1[2];
  const float d01 = P0[0] * P1[1] - P0[1] * P1[0];
  const float d02 = P0[0] * P1[2] - P0[2] * P1[0];
  const float d12 = P0[1] * P1[2] - P0[2] * P1[1];
  const float det0 = (d01 * d01 + d02 * d02) + d12 * d12;  // Cauchy-Binet: det(P P^T)
  const float a = a0 + 0.3f, cc = c0 + 0.3f;
  const float det = (det0 + 0.3f * (a0 + c0)) + 0.09f;
  if (!(det > 0.0f)) return b;
  const float mid = 0.5f * (a + cc);
  const float lam = mid + std::sqrt(std::fmax(0.1f, mid * mid - det));
  if (!(lam < 1.0e30f)) return b;
  const float r = std::ceil(3.0f * std::sqrt(lam));
  if (!(r > 0.0f)) return b;
  const float u = (c.fx * tx) / tz + c.cx;
  const float v = (c.fy * ty) / tz + c.cy;
  if (!(std::fabs(u) < 1.0e7f) || !(std::fabs(v) < 1.0e7f)) return b;
  const float xlo = std::ceil((u - r) - 0.5f), xhi = std::floor((u + r) - 0.5f);
  const float ylo = std::ceil((v - r) - 0.5f), yhi = std::floor((v + r) - 0.5f);
  const float x0 = std::fmax(xlo, 0.0f), x1 = std::fmin(xhi, (float)(c.width - 1));
  const float y0 = std::fmax(ylo, 0.0f), y1 = std::fmin(yhi, (float)(c.height - 1));
  if (x0 > x1 || y0 > y1) return b;
  b.visible = 1;
  b.x0 = (int)x0; b.x1 = (int)x1; b.y0 = (int)y0; b.y1 = (int)y1;
  std::memcpy(&b.depth_bits, &tz, 4);
  b.u = u;
  b.v = v;
  b.A = cc / det;
  b.B = -(b0 / det);
  b.C = a / det;
  b.o = 1.0f / (1.0f + exp_spec(-logit));
  return b;
}

BinRec bin_of(const orc_params& p, int64_t i, const orc_camera& c) {
  float m[3], ls[3], q[4];
  for (int k = 0; k < 3; ++k) {
    m[k] = (float)p.means[3 * i + k];
    ls[k] = (float)p.log_scales[3 * i + k];
  }
  for (int k = 0; k < 4; ++k) q[k] = (float)p.quats[4 * i + k];
  return bin_spec(m, ls, q, (float)p.opacity_logits[i], c);
}

// ---------------------------------------------------------------------------------
// Real spherical harmonics, degrees 0-3, with the Condon-Shortley phase:
//   Y_{l,m} = sqrt(2) Re Y_l^m (m > 0), Y_l^0 (m = 0), sqrt(2) Im Y_l^{|m|} (m < 0),
// written as homogeneous polynomials in the unit direction (x, y, z), ordered
// m = -l..l within each degree.  Normalisations from the closed form
// N_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
// ---------------------------------------------------------------------------------
void sh_basis(const double d[3], double Y[16], double dY[16][3]) {
  const double x = d[0], y = d[1], z = d[2];
  const double PI = 3.14159265358979323846;
  const double k0 = 0.5 / std::sqrt(PI);
  const double k1 = std::sqrt(3.0 / (4.0 * PI));
  const double k2a = std::sqrt(15.0 / (4.0 * PI));
  const double k2b = std::sqrt(5.0 / (16.0 * PI));
  const double k2c = std::sqrt(15.0 / (16.0 * PI));
  const double k3a = std::sqrt(35.0 / (32.0 * PI));
  const double k3b = std::sqrt(105.0 / (4.0 * PI));
  const double k3c = std::sqrt(21.0 / (32.0 * PI));
  const double k3d = std::sqrt(7.0 / (16.0 * PI));
  const double k3e = std::sqrt(105.0 / (16.0 * PI));
  // value, d/dx, d/dy, d/dz of each polynomial
  auto set = [&](int i, double v, double gx, double gy, double gz) {
    Y[i] = v;
    if (dY) { dY[i][0] = gx; dY[i][1] = gy; dY[i][2] = gz; }
  };
  set(0, k0, 0, 0, 0);
  set(1, -k1 * y, 0, -k1, 0);
  set(2, k1 * z, 0, 0, k1);
  set(3, -k1 * x, -k1, 0, 0);
  set(4, k2a * x * y, k2a * y, k2a * x, 0);
  set(5, -k2a * y * z, 0, -k2a * z, -k2a * y);
  set(6, k2b * (2 * z * z - x * x - y * y), -2 * k2b * x, -2 * k2b * y, 4 * k2b * z);
  set(7, -k2a * x * z, -k2a * z, 0, -k2a * x);
  set(8, k2c * (x * x - y * y), 2 * k2c * x, -2 * k2c * y, 0);
  set(9, -k3a * y * (3 * x * x - y * y), -6 * k3a * x * y, -k3a * (3 * x * x - 3 * y * y), 0);
  set(10, k3b * x * y * z, k3b * y * z, k3b * x * z, k3b * x * y);
  set(11, -k3c * y * (4 * z * z - x * x - y * y), 2 * k3c * x * y,
      -k3c * (4 * z * z - x * x - 3 * y * y), -8 * k3c * y * z);
  set(12, k3d * z * (2 * z * z - 3 * x * x - 3 * y * y), -6 * k3d * x * z, -6 * k3d * y * z,
      k3d * (6 * z * z - 3 * x * x - 3 * y * y));
  set(13, -k3c * x * (4 * z * z - x * x - y * y), -k3c * (4 * z * z - 3 * x * x - y * y),
      2 * k3c * x * y, -8 * k3c * x * z);
  set(14, k3e * z * (x * x - y * y), 2 * k3e * x * z, -2 * k3e * y * z, k3e * (x * x - y * y));
  set(15, -k3a * x * (x * x - 3 * y * y), -k3a * (3 * x * x - 3 * y * y), 6 * k3a * x * y, 0);
}

// ---------------------------------------------------------------------------------
// FP64 projection of one Gaussian (continuous quantities; the discrete ones come from
// bin_spec).  Keeps the intermediates the backward needs.
// ---------------------------------------------------------------------------------
struct Proj {
  double t[3];               // camera-space mean
  double u, v;               // 2-D mean (pixels)
  double a, b, c;            // Sigma2D (dilated)
  double A, B, C;            // conic = Sigma2D^{-1}
  double o;                  // opacity
  double col[3];             // colour after clamp
  int col_clamped[3];
  double depth;
  // intermediates
  double qhat[4], qnorm, Rq[9], s[3], M[9], V[9], P0[3], P1[3];
  double j00, j02, j11, j12, rx, ry;
  int clx, cly;
  double dir[3], dist, Y[16], dY[16][3];
};

Proj project64(const orc_params& p, int64_t i, const orc_camera& c) {
  Proj g;
  double R[9], tc[3];
  for (int k = 0; k < 9; ++k) R[k] = c.R[k];
  for (int k = 0; k < 3; ++k) tc[k] = c.t[k];
  const double* mu = p.means + 3 * i;
  for (int r = 0; r < 3; ++r) g.t[r] = R[3 * r] * mu[0] + R[3 * r + 1] * mu[1] + R[3 * r + 2] * mu[2] + tc[r];
  const double* q = p.quats + 4 * i;
  g.qnorm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) g.qhat[k] = q[k] / g.qnorm;
  const double w = g.qhat[0], x = g.qhat[1], y = g.qhat[2], z = g.qhat[3];
  double* Rq = g.Rq;
  Rq[0] = 1 - 2 * (y * y + z * z); Rq[1] = 2 * (x * y - w * z);     Rq[2] = 2 * (x * z + w * y);
  Rq[3] = 2 * (x * y + w * z);     Rq[4] = 1 - 2 * (x * x + z * z); Rq[5] = 2 * (y * z - w * x);
  Rq[6] = 2 * (x * z - w * y);     Rq[7] = 2 * (y * z + w * x);     Rq[8] = 1 - 2 * (x * x + y * y);
  for (int k = 0; k < 3; ++k) g.s[k] = std::exp(p.log_scales[3 * i + k]);
  for (int r = 0; r < 3; ++r)
    for (int j = 0; j < 3; ++j) g.M[3 * r + j] = Rq[3 * r + j] * g.s[j];
  for (int r = 0; r < 3; ++r)
    for (int j = 0; j < 3; ++j)
      g.V[3 * r + j] = R[3 * r] * g.M[j] + R[3 * r + 1] * g.M[3 + j] + R[3 * r + 2] * g.M[6 + j];
  const double fx = c.fx, fy = c.fy, tz = g.t[2];
  const double limx = 1.3 * (0.5 * c.width) / fx, limy = 1.3 * (0.5 * c.height) / fy;
  const double rx = g.t[0] / tz, ry = g.t[1] / tz;
  g.clx = (rx < -limx || rx > limx);
  g.cly = (ry < -limy || ry > limy);
  g.rx = std::min(limx, std::max(-limx, rx));
  g.ry = std::min(limy, std::max(-limy, ry));
  g.j00 = fx / tz; g.j02 = -fx * g.rx / tz; g.j11 = fy / tz; g.j12 = -fy * g.ry / tz;
  for (int j = 0; j < 3; ++j) {
    g.P0[j] = g.j00 * g.V[j] + g.j02 * g.V[6 + j];
    g.P1[j] = g.j11 * g.V[3 + j] + g.j12 * g.V[6 + j];
  }
  const double a0 = g.P0[0] * g.P0[0] + g.P0[1] * g.P0[1] + g.P0[2] * g.P0[2];
  const double c0 = g.P1[0] * g.P1[0] + g.P1[1] * g.P1[1] + g.P1[2] * g.P1[2];
  const double b0 = g.P0[0] * g.P1[0] + g.P0[1] * g.P1[1] + g.P0[2] * g.P1[2];
  g.a = a0 + 0.3; g.b = b0; g.c = c0 + 0.3;
  const double det = g.a * g.c - g.b * g.b;
  g.A = g.c / det; g.B = -g.b / det; g.C = g.a / det;
  g.u = fx * g.t[0] / tz + c.cx;
  g.v = fy * g.t[1] / tz + c.cy;
  g.depth = tz;
  g.o = 1.0 / (1.0 + std::exp(-p.opacity_logits[i]));
  // colour from SH at the viewing direction (mean minus camera centre)
  double eye[3];
  for (int k = 0; k < 3; ++k) eye[k] = -(R[k] * tc[0] + R[3 + k] * tc[1] + R[6 + k] * tc[2]);
  double dv[3] = {mu[0] - eye[0], mu[1] - eye[1], mu[2] - eye[2]};
  g.dist = std::sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  for (int k = 0; k < 3; ++k) g.dir[k] = dv[k] / g.dist;
  sh_basis(g.dir, g.Y, g.dY);
  const int nc = (p.sh_degree + 1) * (p.sh_degree + 1);
  const double* sh = p.sh + i * (int64_t)nc * 3;
  for (int ch = 0; ch < 3; ++ch) {
    double acc = 0.5;
    for (int k = 0; k < nc; ++k) acc += g.Y[k] * sh[3 * k + ch];
    g.col_clamped[ch] = acc < 0.0;
    g.col[ch] = acc < 0.0 ? 0.0 : acc;
  }
  return g;
}

// ---------------------------------------------------------------------------------
// Tile lists: every (Gaussian, tile) pair of the Gaussian's tile rectangle, each tile's
// list sorted by (depth bits, Gaussian index) [Sec. 2 step 2].
// ---------------------------------------------------------------------------------
struct Tiles {
  int tw, th;
  std::vector<int64_t> start;   // tw*th + 1
  std::vector<int32_t> list;    // Gaussian indices
};

Tiles build_tiles(const std::vector<BinRec>& bins, int W, int H, int B, float amin) {
  Tiles T;
  T.tw = (W + B - 1) / B;
  T.th = (H + B - 1) / B;
  const int nt = T.tw * T.th;
  std::vector<std::vector<std::pair<uint64_t, int32_t>>> per(nt);
  for (size_t i = 0; i < bins.size(); ++i) {
    const BinRec& b = bins[i];
    if (!b.visible) continue;
    const TileCull tc = tile_cull_prep(b, amin);
    for (int ty = b.y0 / B; ty <= b.y1 / B; ++ty)
      for (int tx = b.x0 / B; tx <= b.x1 / B; ++tx)
        if (tile_hits_spec(b, tc, tx, ty, B))
          per[ty * T.tw + tx].push_back({((uint64_t)b.depth_bits << 32) | (uint64_t)i, (int32_t)i});
  }
  T.start.assign(nt + 1, 0);
  for (int t = 0; t < nt; ++t) {
    std::sort(per[t].begin(), per[t].end());
    T.start[t + 1] = T.start[t] + (int64_t)per[t].size();
  }
  T.list.resize(T.start[nt]);
  for (int t = 0; t < nt; ++t)
    for (size_t j = 0; j < per[t].size(); ++j) T.list[T.start[t] + j] = per[t][j].second;
  return T;
}

// Per-pixel record of one included Gaussian (for the backward).
struct Frag {
  int32_t g;
  double alpha, T, dx, dy, ex;  // ex = e^power
  int clamped;
};

enum { AMB_ALPHA = 1, AMB_POWER = 2, AMB_TSTOP = 4, AMB_KEY = 8, AMB_SAT = 16 };

// Blend one pixel of one subset front to back.  Returns flags of ambiguous decisions.
//
// flip (nullable) receives a bound on how far an implementation that takes any flagged
// decision the other way (and any later transmittance stop that such a change can move)
// may end from this result: |delta C| <= flip[0] max c, |delta D| <= flip[0] max d,
// |delta T| <= flip[1].  Taking the decisions in list order, with rho = prod 1/(1 - alpha)
// - 1 over the alpha_min decisions flipped so far (the most any transmittance can have
// grown or shrunk by then):
//   * an alpha_min decision at Gaussian i moves C by alpha_i T_i (c_i - X) with X the
//     normalised colour behind i, at most alpha_i T_i (1 + rho) max c, and multiplies
//     every later transmittance by (1 - alpha_i)^(+-1), which rho accumulates;
//   * a flagged power sign or transmittance stop at Gaussian k, or an unflagged stop test
//     that the accumulated rho can move (relative margin <= rho + its own margin), leaves
//     everything from k on within [0, T_k (1 + rho) max c] in both results: that amount
//     bounds the rest, and later decisions add nothing;
//   * T_final moves by at most T_final rho plus the stop amounts.
// flip[2], flip[3] receive the depth range of the Gaussians that may contribute in either
// result (those blended, flagged, or in the rectangle after a bounded rest), within which
// the subset's composite key D / (1 - T) stays whichever of them contribute (+inf, -inf if
// none may).
int blend_pixel(int px, int py, const int32_t* lst, int64_t cnt, const std::vector<BinRec>& bins,
                const std::vector<Proj>& pr, const orc_opts& o, double C[3], double& T,
                double& D, int32_t& last, int32_t& ncontrib, int64_t& evaluated,
                std::vector<Frag>* frags, double* flip = nullptr) {
  int amb = 0;
  T = 1.0; D = 0.0; C[0] = C[1] = C[2] = 0.0; last = -1; ncontrib = 0;
  const double pcx = px + 0.5, pcy = py + 0.5;
  double rho = 0.0, massC = 0.0, massT = 0.0;
  bool rest_bounded = false;  // a stop amount already bounds everything from here on
  int64_t rest_from = cnt;    // list position where the rest became bounded
  double dlo = INFINITY, dhi = -INFINITY;
  int64_t j = 0;
  auto bound_rest = [&](double Tk) {
    if (rest_bounded) return;
    massC += Tk * (1.0 + rho);
    massT += Tk * (1.0 + rho);
    rest_bounded = true;
    rest_from = j;
  };
  for (; j < cnt; ++j) {
    const int32_t g = lst[j];
    const BinRec& b = bins[g];
    ++evaluated;
    if (px < b.x0 || px > b.x1 || py < b.y0 || py > b.y1) continue;
    const Proj& q = pr[g];
    const double dx = pcx - q.u, dy = pcy - q.v;
    const double t1 = q.A * dx * dx, t2 = q.C * dy * dy, t3 = 2.0 * q.B * dx * dy;
    const double power = -0.5 * (t1 + t2) - 0.5 * t3;
    if (std::fabs(power) <= o.amb_power * (std::fabs(t1) + std::fabs(t2) + std::fabs(t3)) &&
        (t1 + t2 + std::fabs(t3)) > 0.0) {
      amb |= AMB_POWER;
      bound_rest(T);
      dlo = std::min(dlo, q.depth);
      dhi = std::max(dhi, q.depth);
    }
    if (power > 0.0) continue;
    const double ex = std::exp(power);
    const double raw = q.o * ex;
    const int clamped = raw > o.alpha_max;
    const double alpha = clamped ? o.alpha_max : raw;
    // alpha's relative error in FP32 is the exponent's absolute error, which grows with
    // the magnitude of its terms (they cancel for elongated Gaussians): the alpha and
    // T-stop margins include it
    const double rel_alpha = clamped ? 0.0 : 0.5 * o.amb_power * (std::fabs(t1) + std::fabs(t2) + std::fabs(t3));
    if (std::fabs(alpha - o.alpha_min) <= (o.amb_alpha + rel_alpha) * o.alpha_min) {
      amb |= AMB_ALPHA;
      if (!rest_bounded) {
        massC += alpha * T * (1.0 + rho);
        rho = (1.0 + rho) / (1.0 - alpha) - 1.0;
      }
      dlo = std::min(dlo, q.depth);
      dhi = std::max(dhi, q.depth);
    }
    if (alpha < o.alpha_min) continue;
    dlo = std::min(dlo, q.depth);
    dhi = std::max(dhi, q.depth);
    const double Tn = T * (1.0 - alpha);
    const double rel_T = o.amb_T + rel_alpha * alpha / (1.0 - alpha);
    if (o.eps_T > 0.0) {
      const double margin = std::fabs(Tn - o.eps_T);
      if (margin <= rel_T * o.eps_T) {
        amb |= AMB_TSTOP;
        bound_rest(T);
      } else if (rho > 0.0 && margin <= (rel_T + 1.001 * rho) * o.eps_T) {
        bound_rest(T);
      }
    }
    if (Tn < o.eps_T) break;
    const double w = alpha * T;
    for (int ch = 0; ch < 3; ++ch) C[ch] += q.col[ch] * w;
    D += q.depth * w;
    if (frags) frags->push_back(Frag{g, alpha, T, dx, dy, ex, clamped});
    T = Tn;
    last = g;
    ++ncontrib;
  }
  if (flip) {
    flip[0] = massC;
    flip[1] = massT + (rest_bounded ? 0.0 : T * rho);
    // after a bounded rest or an early stop any later Gaussian of the rectangle may
    // contribute in the other result
    const int64_t from = rest_bounded ? rest_from : cnt;
    for (int64_t k = from; k < cnt; ++k) {
      const BinRec& b = bins[lst[k]];
      if (px < b.x0 || px > b.x1 || py < b.y0 || py > b.y1) continue;
      dlo = std::min(dlo, pr[lst[k]].depth);
      dhi = std::max(dhi, pr[lst[k]].depth);
    }
    flip[2] = dlo;
    flip[3] = dhi;
  }
  return amb;
}

struct Subset {
  std::vector<BinRec> bins;
  std::vector<Proj> pr;
  Tiles tiles;
};

// Cross-boundary per-ray filtering (Sec. 8.1, appendix "Cross-boundary Gaussians
// Handling"), in one view.  Q_cross: a Gaussian of cell k whose support box
// mu +- 3 s_max (FP32; s_max its largest activated scale) meets another cell s.  D_m: the
// range of the specification's FP32 depths of subset m's kept Gaussians; Omega_m: the
// bounding rectangle of the tile rectangles of its Gaussians that have a (Gaussian, tile)
// pair.  The Gaussian leaves the rays of
// tile t (a tile of its own pairs, hence of Omega_k) when, for some such s, t lies in
// Omega_s and its depth in D_k n D_s.
struct CrossFilter {
  std::vector<uint64_t> cross;       // per global Gaussian: bit s, the support meets cell s
  std::vector<int> omega;            // [K][4] tx0, ty0, tx1, ty1 (tx0 > tx1: empty)
  std::vector<uint32_t> dmin, dmax;  // [K] depth bits (dmin > dmax: no kept Gaussian)
  bool removes(int64_t g, int k, int tx, int ty, uint32_t dbits) const {
    const uint64_t c = cross[g];
    for (int s = 0; s < 64; ++s) {
      if (!((c >> s) & 1ull)) continue;
      const int* o = &omega[4 * s];
      if (tx < o[0] || tx > o[2] || ty < o[1] || ty > o[3]) continue;
      const uint32_t lo = std::max(dmin[k], dmin[s]), hi = std::min(dmax[k], dmax[s]);
      if (dbits >= lo && dbits <= hi) return true;
    }
    return false;
  }
};

// Removes from subset m's tile lists the pairs the filter takes out (global index goff + i).
void apply_filter(Subset& s, const CrossFilter& f, int m, int64_t goff) {
  const int nt = s.tiles.tw * s.tiles.th;
  std::vector<int64_t> start(nt + 1, 0);
  std::vector<int32_t> list;
  list.reserve(s.tiles.list.size());
  for (int t = 0; t < nt; ++t) {
    const int tx = t % s.tiles.tw, ty = t / s.tiles.tw;
    for (int64_t j = s.tiles.start[t]; j < s.tiles.start[t + 1]; ++j) {
      const int32_t i = s.tiles.list[j];
      if (!f.removes(goff + i, m, tx, ty, s.bins[i].depth_bits)) list.push_back(i);
    }
    start[t + 1] = (int64_t)list.size();
  }
  s.tiles.start.swap(start);
  s.tiles.list.swap(list);
}

Subset prepare(const orc_params& p, const orc_camera& cam, int B, float amin,
               const CrossFilter* f = nullptr, int m = 0, int64_t goff = 0) {
  Subset s;
  s.bins.resize(p.n);
  s.pr.resize(p.n);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t i = 0; i < p.n; ++i) {
    s.bins[i] = bin_of(p, i, cam);
    if (s.bins[i].visible) s.pr[i] = project64(p, i, cam);
  }
  s.tiles = build_tiles(s.bins, cam.width, cam.height, B, amin);
  if (f) apply_filter(s, *f, m, goff);
  return s;
}

orc_params slice(const orc_params& p, int64_t lo, int64_t hi) {
  const int nc = (p.sh_degree + 1) * (p.sh_degree + 1);
  orc_params q = p;
  q.means = p.means + 3 * lo;
  q.log_scales = p.log_scales + 3 * lo;
  q.quats = p.quats + 4 * lo;
  q.opacity_logits = p.opacity_logits + lo;
  q.sh = p.sh + lo * nc * 3;
  q.n = hi - lo;
  return q;
}

// The filter of one view over K contiguous subsets; cells [K][6] = (lo x, y, z, hi x, y, z)
// of the k-d boxes (infinite on open sides).
CrossFilter make_filter(const orc_params& p, const int64_t* offsets, int K, const orc_camera& cam,
                        const orc_opts& o, const float* cells) {
  CrossFilter f;
  f.cross.assign((size_t)p.n, 0ull);
  f.omega.assign((size_t)4 * K, 0);
  f.dmin.assign(K, 0xFFFFFFFFu);
  f.dmax.assign(K, 0u);
  for (int m = 0; m < K; ++m) {
    orc_params q = slice(p, offsets[m], offsets[m + 1]);
    const Subset s = prepare(q, cam, o.tile, (float)o.alpha_min);
    // Omega (the visible region of Sec. 4.2, read on one GPU as a tile rectangle): the
    // bounding rectangle of the tile rectangles of the subset's Gaussians that have at
    // least one (Gaussian, tile) pair
    int* om = &f.omega[(size_t)4 * m];
    om[0] = om[1] = INT_MAX;
    om[2] = om[3] = -1;
    std::vector<uint8_t> paired((size_t)q.n, 0);
    for (size_t j = 0; j < s.tiles.list.size(); ++j) paired[s.tiles.list[j]] = 1;
    const int B = o.tile;
    for (int64_t i = 0; i < q.n; ++i) {
      if (!paired[i]) continue;
      const BinRec& b = s.bins[i];
      om[0] = std::min(om[0], b.x0 / B); om[1] = std::min(om[1], b.y0 / B);
      om[2] = std::max(om[2], b.x1 / B); om[3] = std::max(om[3], b.y1 / B);
    }
    for (int64_t i = 0; i < q.n; ++i) {
      if (!s.bins[i].visible) continue;
      f.dmin[m] = std::min(f.dmin[m], s.bins[i].depth_bits);
      f.dmax[m] = std::max(f.dmax[m], s.bins[i].depth_bits);
    }
    for (int64_t i = 0; i < q.n; ++i) {
      float smax = 0.0f;
      for (int a = 0; a < 3; ++a) smax = std::max(smax, exp_spec((float)q.log_scales[3 * i + a]));
      const float r3 = 3.0f * smax;
      float lo[3], hi[3];
      for (int a = 0; a < 3; ++a) {
        lo[a] = (float)q.means[3 * i + a] - r3;
        hi[a] = (float)q.means[3 * i + a] + r3;
      }
      uint64_t mask = 0;
      for (int c = 0; c < K; ++c) {
        if (c == m) continue;
        const float* b = cells + 6 * c;
        if (lo[0] <= b[3] && hi[0] >= b[0] && lo[1] <= b[4] && hi[1] >= b[1] && lo[2] <= b[5] &&
            hi[2] >= b[2])
          mask |= 1ull << c;
      }
      f.cross[(size_t)(offsets[m] + i)] = mask;
    }
  }
  return f;
}

// Composite order of one pixel (Eq. 5 with the normalised-depth reading).  Fills `ord`
// with subset indices front to back; returns ambiguity flags for near-tied keys.
int composite_order(int K, const double* Tm, const double* Dm, const orc_opts& o, int* ord) {
  std::vector<std::pair<double, int>> keys(K);
  for (int m = 0; m < K; ++m) {
    const double occ = 1.0 - Tm[m];
    const double key = (Tm[m] < 1.0) ? Dm[m] / occ : INFINITY;
    keys[m] = {key, m};
  }
  std::stable_sort(keys.begin(), keys.end(),
                   [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
                     return a.first < b.first;
                   });
  int amb = 0;
  for (int j = 0; j < K; ++j) ord[j] = keys[j].second;
  for (int j = 0; j + 1 < K; ++j) {
    const double ka = keys[j].first, kb = keys[j + 1].first;
    if (!std::isfinite(kb)) break;
    const double occ = std::min(1.0 - Tm[keys[j].second], 1.0 - Tm[keys[j + 1].second]);
    const double tol = (o.amb_key + 1e-6 / occ) * std::max(std::fabs(ka), std::fabs(kb));
    if (std::fabs(kb - ka) <= tol) amb |= AMB_KEY;
  }
  return amb;
}

// Eq. 5 at one pixel, in the order ord, with the saturation cut: image rgb and
// transmittance.
void composite_one(int K, const double* Tm, const double* Cm, const int* ord, const orc_opts& o,
                   double out[3], double& Tout) {
  double P = 1.0;
  out[0] = out[1] = out[2] = 0.0;
  for (int j = 0; j < K; ++j) {
    if (P < o.eps_comp) break;
    const int m = ord[j];
    for (int ch = 0; ch < 3; ++ch) out[ch] += Cm[3 * m + ch] * P;
    P *= Tm[m];
  }
  for (int ch = 0; ch < 3; ++ch) out[ch] += o.bg[ch] * P;
  Tout = P;
}

// Flip bound of one composited pixel (Eq. 5), from the K partials (Tm, Dm, Cm [K][3]),
// their flip bounds fC, fT (|delta C^m| <= fC cmax, |delta T^m| <= fT) and the depth
// range [dlo, dhi] of the Gaussians that may contribute to each (blend_pixel).  With P_j
// the prefix transmittance at rank j of the composite order and L the ranks before the
// saturation cut:
//   * a partial's own change moves the image by at most P_j (fC + fT) cmax (its colour,
//     and its transmittance times the normalised colour behind it, background included)
//     and the transmittance by P_j fT;
//   * a partial with a flagged decision keeps its key D/(1 - T) within [dlo, dhi] (the key
//     is an alpha-weighted mean of contributor depths) and within the first-order reach
//     (|delta D| + key |delta T|) / (1 - T - |delta T|), or becomes empty (key +inf, placed
//     last) if its change can reach its whole occupancy 1 - T; two neighbours whose key
//     ranges meet (with the FP32 margin of composite_order) may be composited the other
//     way round, which moves the image by P_j |C_a (1 - T_b) - C_b (1 - T_a)| (Eq. 5); in a
//     run of three or more, each subset m adds between C_m prod_{k != m} T_k and C_m
//     whatever the order, so the run moves it by at most P_j sum_m C_m (1 - prod T_k);
//   * the saturation cut leaves out at most Pu cmax of colour and Pu of transmittance, Pu
//     the largest prefix, under the partials' flips, at the first rank where the cut can
//     fall.
void composite_bounds(int K, const double* Tm, const double* Dm, const double* Cm,
                      const double* fC, const double* fT, const double* dlo, const double* dhi,
                      const orc_opts& o, double cmax, double dmax, const int* ord, double& bimg,
                      double& bT) {
  bimg = 0.0;
  bT = 0.0;
  std::vector<double> P(K + 1, 1.0);
  int L = 0;
  for (int j = 0; j < K; ++j) {
    if (P[j] < o.eps_comp) break;
    P[j + 1] = P[j] * Tm[ord[j]];
    ++L;
  }
  for (int j = 0; j < L; ++j) {
    const int m = ord[j];
    bimg += P[j] * (fC[m] + fT[m]) * cmax;
    bT += P[j] * fT[m];
  }
  // the cut may fall at the first rank whose prefix, moved by the partials' flips before it
  // (between Pl and Pu: products of T -+ fT), can lie below eps_comp (within amb_T);
  // everything from there on lies within [0, Pu cmax] in both results
  if (L < K || o.eps_comp > 0.0) {
    double Pl = 1.0, Pu = 1.0;
    for (int j = 0; j <= L && j < K + 1; ++j) {
      if (j == K) break;
      if (Pl < o.eps_comp * (1.0 + o.amb_T) || j == L) {
        if (j < K) {
          bimg += Pu * cmax;
          bT += Pu;
        }
        break;
      }
      const int m = ord[j];
      Pl *= std::max(0.0, Tm[m] - fT[m]);
      Pu *= std::min(1.0, Tm[m] + fT[m]);
    }
  }
  // the range each key may take
  std::vector<double> klo(K), khi(K);
  for (int m = 0; m < K; ++m) {
    const double key = Tm[m] < 1.0 ? Dm[m] / (1.0 - Tm[m]) : INFINITY;
    klo[m] = khi[m] = key;
    if (fC[m] == 0.0 && fT[m] == 0.0) continue;  // no flagged decision: the key stays
    if (fT[m] >= 1.0 - Tm[m]) {  // may become empty (or, if empty, take any contributor)
      klo[m] = std::min(std::isfinite(key) ? key : INFINITY, dlo[m]);
      khi[m] = INFINITY;
      continue;
    }
    // both the contributors' depth range and the first-order reach
    // (|delta D| + key |delta T|) / (occupancy - |delta T|) bound the key's change
    const double reach = (fC[m] * dmax + std::fabs(key) * fT[m]) / ((1.0 - Tm[m]) - fT[m]);
    klo[m] = std::max(key - reach, std::min(key, dlo[m]));
    khi[m] = std::min(key + reach, std::max(key, dhi[m]));
  }
  std::vector<uint8_t> near(K, 0);  // near[j]: ranks j and j + 1 may swap
  for (int j = 0; j + 1 < K && j < L; ++j) {
    const int a = ord[j], b = ord[j + 1];
    if (!std::isfinite(klo[a]) && !std::isfinite(klo[b])) break;  // both stay empty
    const double occ = std::max(std::min(1.0 - Tm[a], 1.0 - Tm[b]), 1e-300);
    const double ref = std::max(std::isfinite(khi[a]) ? std::fabs(khi[a]) : 0.0,
                                std::isfinite(klo[b]) ? std::fabs(klo[b]) : 0.0);
    const double tol = (o.amb_key + 1e-6 / occ) * ref;
    near[j] = khi[a] + tol >= klo[b];
  }
  for (int j = 0; j < K && j < L;) {
    if (!near[j]) { ++j; continue; }
    int e = j;
    while (e < K && near[e]) ++e;  // ranks j .. e may be reordered among themselves
    double sw = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
      double d = 0.0;
      if (e == j + 1) {
        const int a = ord[j], b = ord[j + 1];
        d = std::fabs(Cm[3 * a + ch] * (1.0 - Tm[b]) - Cm[3 * b + ch] * (1.0 - Tm[a]));
      } else {
        for (int r = j; r <= e && r < K; ++r) {
          double others = 1.0;
          for (int r2 = j; r2 <= e && r2 < K; ++r2)
            if (r2 != r) others *= Tm[ord[r2]];
          d += Cm[3 * ord[r] + ch] * (1.0 - others);
        }
      }
      sw = std::max(sw, d);
    }
    bimg += P[j] * sw;
    j = e + 1;
  }
}

}  // namespace

// Local render of one subset (filtered by f as subset m with global offset goff, if given).
int render_subset(const orc_params* p, const orc_camera* cam, const orc_opts* o,
                  const uint8_t* tile_mask, double* C, double* T, double* D, int32_t* last,
                  int32_t* ncontrib, uint8_t* amb, int64_t* stats, const CrossFilter* f, int m,
                  int64_t goff, const uint8_t* pix_open = nullptr, double* flips = nullptr,
                  double* cdmax = nullptr, const uint8_t* pix_alt = nullptr,
                  double* alt = nullptr);

namespace {

// Saturation skipping (Sec. 4.2 ②, with the composite's threshold eps_comp): the K
// partials of a view are rendered in the given front-to-back subset order, and the subset
// at rank r leaves a pixel empty (C = 0, T = 1, D = 0, no contributor) where the product
// of the transmittances of the subsets ranked before it is below eps_comp: the saturated
// pixels leave the subset's pixel set.  A tile all of whose pixels are saturated is not
// rendered at all (skip[m * nt + t] = 1).  A pixel whose prefix lies within the relative
// margin amb_T of eps_comp is flagged AMB_SAT.  Renders into C, T, D (planar per subset)
// and, if pskip is given, sets pskip[m * HW + pixel] for the pixels left empty.  With
// order == nullptr every subset is rendered on every pixel of tile_mask's tiles.
// With flips given, flips[0..3] ([K][H][W] each) receive each partial's flip bounds and
// contributor depth range (blend_pixel) and cdmax (2) the largest colour and depth.  With
// saturation skipping, a pixel's skip decision for a subset is ambiguous when its prefix
// lies within amb_T of eps_comp, widened by the relative change that the flip bounds of the
// subsets before it allow (sum of fT / (T - fT)); for such pixels sat_alt ([K][H][W])
// is set and alt ([K][5][H][W]: C rgb, T, D) holds the partial's other outcome.
//
// Stale saturation state (Sec. 4.2 step 2: a view's pixels found saturated by the
// composition of one visit are left out of the next one).  With sat_in ([H][W], used
// with order) the subset at rank r leaves pixel i empty exactly when r >= sat_in[i] (a
// value >= K prunes nothing): the decision is the input's, not the current prefix's.
// With sat_out ([H][W]) each pixel's state for the next visit is re-evaluated from this
// visit's partials: r + 1 for the first rank r below min(sat_in, K) whose prefix (the
// product of the transmittances of ranks 0..r in order) is below eps_comp, or 255 (none)
// if there is no such rank or r + 1 = K.  Pruned ranks are transparent here, so once the
// prefix stays above eps_comp up to the old state every pruned rank comes back.  sat_amb
// (nullable) marks pixels where a prefix examined lies within the AMB_SAT band of
// eps_comp.
void render_partials(const orc_params& p, const int64_t* offsets, int K, const orc_camera& cam,
                     const orc_opts& o, const uint8_t* tile_mask, const int32_t* order,
                     std::vector<double>& C, std::vector<double>& T, std::vector<double>& D,
                     std::vector<uint8_t>& skip, uint8_t* amb, int64_t* stats,
                     const CrossFilter* f, std::vector<uint8_t>* pskip = nullptr,
                     std::vector<double>* flips = nullptr, double* cdmax = nullptr,
                     std::vector<uint8_t>* sat_alt = nullptr, std::vector<double>* alt = nullptr,
                     const uint8_t* sat_in = nullptr, uint8_t* sat_out = nullptr,
                     uint8_t* sat_amb_out = nullptr) {
  const int W = cam.width, H = cam.height, B = o.tile;
  const int64_t HW = (int64_t)W * H;
  const int tw = (W + B - 1) / B, th = (H + B - 1) / B, nt = tw * th;
  C.assign((size_t)K * 3 * HW, 0.0);
  T.assign((size_t)K * HW, 1.0);
  D.assign((size_t)K * HW, 0.0);
  skip.assign((size_t)K * nt, 0);
  if (pskip) pskip->assign((size_t)K * HW, 0);
  if (flips) {
    flips[0].assign((size_t)K * HW, 0.0);
    flips[1].assign((size_t)K * HW, 0.0);
    flips[2].assign((size_t)K * HW, INFINITY);
    flips[3].assign((size_t)K * HW, -INFINITY);
  }
  std::vector<double> fl1(flips ? (size_t)4 * HW : 0);
  std::vector<double> prefix(HW, 1.0), prefix_rel(HW, 0.0);
  std::vector<uint8_t> sat_amb(HW, 0);
  if (!order) sat_in = nullptr;
  const bool want_alt = flips && order && sat_alt && alt && !sat_in;
  std::vector<uint8_t> decided(sat_out ? HW : 0, 0);
  if (sat_out) std::fill(sat_out, sat_out + HW, (uint8_t)255);
  if (sat_amb_out) std::fill(sat_amb_out, sat_amb_out + HW, (uint8_t)0);
  if (want_alt) {
    sat_alt->assign((size_t)K * HW, 0);
    alt->assign((size_t)K * 5 * HW, 0.0);
  }
  std::vector<uint8_t> mask(nt), a1(HW, 0), open(HW, 1);
  for (int r = 0; r < K; ++r) {
    const int m = order ? order[r] : r;
    const bool skipping = order && (r > 0 || sat_in);
    if (skipping)
      for (int64_t i = 0; i < HW; ++i) {
        if (sat_in) {
          open[i] = (uint8_t)(r < (int)sat_in[i]);
        } else {
          open[i] = (uint8_t)(prefix[i] >= o.eps_comp);
          sat_amb[i] = std::fabs(prefix[i] - o.eps_comp) <=
                       (o.amb_T + prefix_rel[i] * (1.0 + o.amb_T)) * o.eps_comp;
          if (amb && sat_amb[i]) amb[i] |= AMB_SAT;
        }
        if (pskip && !open[i]) (*pskip)[(size_t)m * HW + i] = 1;
      }
    for (int t = 0; t < nt; ++t) {
      mask[t] = (uint8_t)(!tile_mask || tile_mask[t]);
      if (skipping && mask[t]) {
        // a tile with no open pixel is not rendered
        const int tx = t % tw, ty = t / tw;
        bool any_open = false;
        for (int py = ty * B; py < std::min(H, (ty + 1) * B); ++py)
          for (int px = tx * B; px < std::min(W, (tx + 1) * B); ++px)
            any_open = any_open || open[(int64_t)py * W + px];
        if (!any_open) {
          mask[t] = 0;
          skip[(size_t)m * nt + t] = 1;
        }
      }
    }
    orc_params q = slice(p, offsets[m], offsets[m + 1]);
    std::fill(a1.begin(), a1.end(), 0);
    render_subset(&q, &cam, &o, mask.data(), C.data() + (size_t)m * 3 * HW,
                  T.data() + (size_t)m * HW, D.data() + (size_t)m * HW, nullptr, nullptr,
                  a1.data(), stats, f, m, offsets[m], skipping ? open.data() : nullptr,
                  flips ? fl1.data() : nullptr, cdmax,
                  want_alt && r > 0 ? sat_amb.data() : nullptr,
                  want_alt ? alt->data() + (size_t)m * 5 * HW : nullptr);
    if (flips)
      for (int64_t i = 0; i < HW; ++i)
        for (int k = 0; k < 4; ++k) flips[k][(size_t)m * HW + i] = fl1[(size_t)k * HW + i];
    if (want_alt && r > 0)
      for (int64_t i = 0; i < HW; ++i) (*sat_alt)[(size_t)m * HW + i] = sat_amb[i];
    if (amb)
      for (int64_t i = 0; i < HW; ++i) amb[i] |= a1[i];
    if (order)
      for (int64_t i = 0; i < HW; ++i) {
        const double Tb = T[(size_t)m * HW + i];
        prefix[i] *= Tb;
        if (flips) {
          // relative change of the prefix that this subset's flips (or other outcome) allow
          double dT = flips[1][(size_t)m * HW + i];
          if (want_alt && r > 0 && sat_amb[i])
            dT = std::max(dT, std::fabs(alt->at(((size_t)m * 5 + 3) * HW + i) - Tb));
          prefix_rel[i] += dT > 0.0 ? (Tb - dT > 0.0 ? dT / (Tb - dT) : INFINITY) : 0.0;
        }
      }
    if (order && sat_out)
      for (int64_t i = 0; i < HW; ++i) {
        const int lim = sat_in ? std::min((int)sat_in[i], K) : K;
        if (decided[i] || r >= lim) continue;
        if (sat_amb_out && std::fabs(prefix[i] - o.eps_comp) <=
                               (o.amb_T + prefix_rel[i] * (1.0 + o.amb_T)) * o.eps_comp)
          sat_amb_out[i] = 1;
        if (prefix[i] < o.eps_comp) {
          decided[i] = 1;
          sat_out[i] = r + 1 < K ? (uint8_t)(r + 1) : (uint8_t)255;
        }
      }
  }
}

}  // namespace

extern "C" {

float orc_exp_spec(float x) { return exp_spec(x); }

void orc_exp_spec_n(const float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = exp_spec(x[i]);
}

void orc_log_spec_n(const float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = log_spec(x[i]);
}

void orc_sh_basis(const double* dirs, int64_t n, double* Y) {
  for (int64_t i = 0; i < n; ++i) sh_basis(dirs + 3 * i, Y + 16 * i, nullptr);
}

void orc_sh_basis_grad(const double* dirs, int64_t n, double* dY) {
  double Y[16];
  for (int64_t i = 0; i < n; ++i) sh_basis(dirs + 3 * i, Y, (double(*)[3])(dY + 48 * i));
}

// FP32 binning spec per Gaussian.  rect: [n][4] (x0,x1,y0,y1), visible: [n].
void orc_bin(const orc_params* p, const orc_camera* cam, int32_t* visible, int32_t* rect,
             uint32_t* depth_bits) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < p->n; ++i) {
    const BinRec b = bin_of(*p, i, *cam);
    visible[i] = b.visible;
    rect[4 * i + 0] = b.x0; rect[4 * i + 1] = b.x1;
    rect[4 * i + 2] = b.y0; rect[4 * i + 3] = b.y1;
    depth_bits[i] = b.depth_bits;
  }
}

// Sorted tile lists.  Pass list == NULL to get the pair count; tile_start has
// ceil(W/B)*ceil(H/B)+1 entries.
int64_t orc_tile_lists(const orc_params* p, const orc_camera* cam, int32_t tile, double alpha_min,
                       int64_t* tile_start, int32_t* list, int64_t capacity) {
  std::vector<BinRec> bins(p->n);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < p->n; ++i) bins[i] = bin_of(*p, i, *cam);
  Tiles T = build_tiles(bins, cam->width, cam->height, tile, (float)alpha_min);
  const int64_t total = (int64_t)T.list.size();
  if (tile_start) std::memcpy(tile_start, T.start.data(), T.start.size() * sizeof(int64_t));
  if (list) {
    if (capacity < total) return -total;
    std::memcpy(list, T.list.data(), total * sizeof(int32_t));
  }
  return total;
}

// FP64 projection: out[n][12] = (u, v, A, B, C, o, r, g, b, depth, a, c) for visible
// Gaussians (zeros otherwise); visible as in orc_bin.
void orc_project(const orc_params* p, const orc_camera* cam, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < p->n; ++i) {
    double* r = out + 12 * i;
    std::fill(r, r + 12, 0.0);
    if (!bin_of(*p, i, *cam).visible) continue;
    const Proj g = project64(*p, i, *cam);
    r[0] = g.u; r[1] = g.v; r[2] = g.A; r[3] = g.B; r[4] = g.C; r[5] = g.o;
    r[6] = g.col[0]; r[7] = g.col[1]; r[8] = g.col[2]; r[9] = g.depth; r[10] = g.a; r[11] = g.c;
  }
}

// Local render of one subset [Eq. 3-4].  Outputs planar C[3][H][W], T[H][W], D[H][W],
// last Gaussian index [H][W] (-1 if none), contributor count [H][W], ambiguity flags
// [H][W].  tile_mask (nullable) restricts the work to tiles with a nonzero entry; other
// pixels are left untouched.  stats[0] += evaluated (pixel, list entry) steps.
// bd (nullable): flip bounds of the subset (partC, partT [H][W]; cmax, dmax).
int orc_render(const orc_params* p, const orc_camera* cam, const orc_opts* o,
               const uint8_t* tile_mask, double* C, double* T, double* D, int32_t* last,
               int32_t* ncontrib, uint8_t* amb, int64_t* stats, orc_bounds* bd) {
  double cd[2] = {0.0, 0.0};
  const int64_t HW = (int64_t)cam->width * cam->height;
  std::vector<double> fl(bd ? (size_t)4 * HW : 0);
  const int r = render_subset(p, cam, o, tile_mask, C, T, D, last, ncontrib, amb, stats, nullptr,
                              0, 0, nullptr, bd ? fl.data() : nullptr, cd);
  if (bd) {
    if (bd->partC) std::memcpy(bd->partC, fl.data(), HW * sizeof(double));
    if (bd->partT) std::memcpy(bd->partT, fl.data() + HW, HW * sizeof(double));
    bd->cmax = std::max(cd[0], std::max(o->bg[0], std::max(o->bg[1], o->bg[2])));
    bd->dmax = cd[1];
  }
  return r;
}
}  // extern "C"

// pix_open (nullable, [H][W]): a pixel with a zero entry is left empty (C = 0, T = 1,
// D = 0, no contributor) without being evaluated.  flips (nullable, [4][H][W]): the
// pixel's flip bounds and contributor depth range (blend_pixel's flip[0..3]).  cdmax
// (nullable, 2): raised to the largest colour channel and the largest depth of the
// subset's visible Gaussians.  pix_alt (nullable, [H][W]): pixels whose saturation decision
// is ambiguous; alt ([5][H][W]: C rgb, T, D) receives their other outcome (empty where the
// pixel is rendered, rendered where it is left empty), in tiles outside tile_mask too.
int render_subset(const orc_params* p, const orc_camera* cam, const orc_opts* o,
                  const uint8_t* tile_mask, double* C, double* T, double* D, int32_t* last,
                  int32_t* ncontrib, uint8_t* amb, int64_t* stats, const CrossFilter* f, int m,
                  int64_t goff, const uint8_t* pix_open, double* flips, double* cdmax,
                  const uint8_t* pix_alt, double* alt) {
  const int W = cam->width, H = cam->height, B = o->tile;
  Subset s = prepare(*p, *cam, B, (float)o->alpha_min, f, m, goff);
  if (cdmax)
    for (int64_t i = 0; i < p->n; ++i) {
      if (!s.bins[i].visible) continue;
      for (int ch = 0; ch < 3; ++ch) cdmax[0] = std::max(cdmax[0], s.pr[i].col[ch]);
      cdmax[1] = std::max(cdmax[1], s.pr[i].depth);
    }
  const int nt = s.tiles.tw * s.tiles.th;
  int64_t evaluated = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : evaluated)
  for (int t = 0; t < nt; ++t) {
    const int tx = t % s.tiles.tw, ty = t / s.tiles.tw;
    const bool main_t = !tile_mask || tile_mask[t];
    bool alt_t = false;
    if (pix_alt)
      for (int py = ty * B; py < std::min(H, (ty + 1) * B); ++py)
        for (int px = tx * B; px < std::min(W, (tx + 1) * B); ++px)
          alt_t = alt_t || pix_alt[(int64_t)py * W + px];
    if (!main_t && !alt_t) continue;
    const int32_t* lst = s.tiles.list.data() + s.tiles.start[t];
    const int64_t cnt = s.tiles.start[t + 1] - s.tiles.start[t];
    for (int py = ty * B; py < std::min(H, (ty + 1) * B); ++py)
      for (int px = tx * B; px < std::min(W, (tx + 1) * B); ++px) {
        const int64_t pi = (int64_t)py * W + px;
        const bool rendered = main_t && (!pix_open || pix_open[pi]);
        if (pix_alt && pix_alt[pi]) {
          double a3[3] = {0.0, 0.0, 0.0}, at = 1.0, ad = 0.0;
          int32_t alg = -1, anc = 0;
          int64_t aev = 0;
          if (!rendered)
            blend_pixel(px, py, lst, cnt, s.bins, s.pr, *o, a3, at, ad, alg, anc, aev, nullptr);
          for (int ch = 0; ch < 3; ++ch) alt[(int64_t)ch * H * W + pi] = a3[ch];
          alt[(int64_t)3 * H * W + pi] = at;
          alt[(int64_t)4 * H * W + pi] = ad;
        }
        if (!main_t) continue;
        double c3[3] = {0.0, 0.0, 0.0}, tt = 1.0, dd = 0.0;
        int32_t lg = -1, nc = 0;
        int a = 0;
        double fl[4] = {0.0, 0.0, INFINITY, -INFINITY};
        if (!pix_open || pix_open[pi])
          a = blend_pixel(px, py, lst, cnt, s.bins, s.pr, *o, c3, tt, dd, lg, nc, evaluated,
                          nullptr, fl);
        if (flips)
          for (int k = 0; k < 4; ++k) flips[(int64_t)k * H * W + pi] = fl[k];
        for (int ch = 0; ch < 3; ++ch) C[(int64_t)ch * H * W + pi] = c3[ch];
        T[pi] = tt; D[pi] = dd;
        if (last) last[pi] = lg;
        if (ncontrib) ncontrib[pi] = nc;
        if (amb) amb[pi] = (uint8_t)a;
      }
  }
  if (stats) stats[0] += evaluated;
  return 0;
}

extern "C" {

// Global composition of K partials [Eq. 5].  Partials planar: C[K][3][H][W],
// T[K][H][W], D[K][H][W].  Outputs image [3][H][W], total transmittance [H][W], the
// number of subsets composited [H][W] and ambiguity flags (OR-ed into amb).  bimg, bT
// (nullable, [H][W]): flip bounds of the image and transmittance for exactly given
// partials (near-tied keys and the saturation cut; composite_bounds).
int orc_composite(int32_t K, int32_t H, int32_t W, const double* Cp, const double* Tp,
                  const double* Dp, const orc_opts* o, double* out, double* Tout,
                  int32_t* nused, uint8_t* amb, double* bimg, double* bT) {
  const int64_t HW = (int64_t)H * W;
#pragma omp parallel for schedule(static)
  for (int64_t pi = 0; pi < HW; ++pi) {
    std::vector<double> Tm(K), Dm(K);
    std::vector<int> ord(K);
    for (int m = 0; m < K; ++m) { Tm[m] = Tp[m * HW + pi]; Dm[m] = Dp[m * HW + pi]; }
    int a = composite_order(K, Tm.data(), Dm.data(), *o, ord.data());
    double c[3] = {0, 0, 0}, P = 1.0;
    int used = 0;
    for (int j = 0; j < K; ++j) {
      if (o->eps_comp > 0.0 && std::fabs(P - o->eps_comp) <= o->amb_T * o->eps_comp) a |= AMB_SAT;
      if (P < o->eps_comp) break;
      const int m = ord[j];
      for (int ch = 0; ch < 3; ++ch) c[ch] += Cp[((int64_t)m * 3 + ch) * HW + pi] * P;
      P *= Tm[m];
      ++used;
    }
    for (int ch = 0; ch < 3; ++ch) out[ch * HW + pi] = c[ch] + o->bg[ch] * P;
    Tout[pi] = P;
    if (nused) nused[pi] = used;
    if (amb) amb[pi] |= (uint8_t)a;
    if (bimg || bT) {
      std::vector<double> Cm((size_t)3 * K), zero(K, 0.0);
      double cmax = std::max(o->bg[0], std::max(o->bg[1], o->bg[2]));
      for (int m = 0; m < K; ++m)
        for (int ch = 0; ch < 3; ++ch) {
          Cm[3 * m + ch] = Cp[((int64_t)m * 3 + ch) * HW + pi];
          // a partial's colour is at most its occupancy times its largest colour; its
          // normalised colour bounds what lies behind
          if (Tm[m] < 1.0) cmax = std::max(cmax, Cm[3 * m + ch] / (1.0 - Tm[m]));
        }
      double bi, bt;
      composite_bounds(K, Tm.data(), Dm.data(), Cm.data(), zero.data(), zero.data(), zero.data(),
                       zero.data(), *o, cmax, 0.0, ord.data(), bi, bt);
      if (bimg) bimg[pi] = bi;
      if (bT) bT[pi] = bt;
    }
  }
  return 0;
}

// Render K contiguous subsets (offsets[K+1] into p) of one view and composite them.
// Partial outputs (nullable) as in orc_composite.  sep (nullable): 1 where the pixel is
// separable, i.e. its monolithic contributor list (all Gaussians, no termination) is a
// concatenation of per-subset runs in composite order (where Eq. 5 equals Eq. 2).
// bd (nullable): flip bounds of the image and of every partial (orc_bounds).
static int render_view_impl(const orc_params* p, const int64_t* offsets, int32_t K,
                            const orc_camera* cam, const orc_opts* o, const uint8_t* tile_mask,
                            const int32_t* order, const float* cells, double* out, double* Tout,
                            double* Cp, double* Tp, double* Dp, uint8_t* amb, uint8_t* sep,
                            uint8_t* skip_out, int64_t* stats, orc_bounds* bd,
                            const uint8_t* sat_in, uint8_t* sat_out, uint8_t* sat_amb) {
  const int64_t HW = (int64_t)cam->width * cam->height;
  std::vector<double> C, T, D;
  std::vector<uint8_t> a(HW, 0), skip;
  CrossFilter cf;
  if (cells) cf = make_filter(*p, offsets, K, *cam, *o, cells);
  std::vector<double> flips[4], alt;
  std::vector<uint8_t> sat_alt;
  double cd[2] = {0.0, 0.0};
  render_partials(*p, offsets, K, *cam, *o, tile_mask, order, C, T, D, skip, a.data(), stats,
                  cells ? &cf : nullptr, nullptr, bd ? flips : nullptr, cd, &sat_alt, &alt,
                  sat_in, sat_out, sat_amb);
  if (skip_out) std::memcpy(skip_out, skip.data(), skip.size());
  orc_composite(K, cam->height, cam->width, C.data(), T.data(), D.data(), o, out, Tout, nullptr,
                a.data(), nullptr, nullptr);
  if (bd) {
    const double cmax = std::max(cd[0], std::max(o->bg[0], std::max(o->bg[1], o->bg[2])));
    bd->cmax = cmax;
    bd->dmax = cd[1];
    const bool has_alt = !sat_alt.empty();
    // a partial whose saturation decision is ambiguous may end as its other outcome
    std::vector<double> pC = flips[0], pT = flips[1];
    if (has_alt)
      for (int m = 0; m < K; ++m)
        for (int64_t i = 0; i < HW; ++i) {
          const size_t mi = (size_t)m * HW + i;
          if (!sat_alt[mi]) continue;
          double dc = std::fabs(alt[((size_t)m * 5 + 4) * HW + i] - D[mi]) / std::max(cd[1], 1e-300);
          for (int ch = 0; ch < 3; ++ch)
            dc = std::max(dc, std::fabs(alt[((size_t)m * 5 + ch) * HW + i] -
                                        C[((size_t)m * 3 + ch) * HW + i]) / std::max(cmax, 1e-300));
          pC[mi] = std::max(pC[mi], dc);
          pT[mi] = std::max(pT[mi], std::fabs(alt[((size_t)m * 5 + 3) * HW + i] - T[mi]));
        }
    if (bd->partC) std::memcpy(bd->partC, pC.data(), pC.size() * sizeof(double));
    if (bd->partT) std::memcpy(bd->partT, pT.data(), pT.size() * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t pi = 0; pi < HW; ++pi) {
      if (tile_mask) {
        const int B = o->tile, tw = (cam->width + B - 1) / B;
        const int px = (int)(pi % cam->width), py = (int)(pi / cam->width);
        if (!tile_mask[(py / B) * tw + px / B]) continue;
      }
      std::vector<double> Tm(K), Dm(K), Cm((size_t)3 * K), fC(K), fT(K), dlo(K), dhi(K);
      std::vector<int> ord(K);
      for (int m = 0; m < K; ++m) {
        Tm[m] = T[(size_t)m * HW + pi];
        Dm[m] = D[(size_t)m * HW + pi];
        for (int ch = 0; ch < 3; ++ch) Cm[3 * m + ch] = C[((size_t)m * 3 + ch) * HW + pi];
        fC[m] = flips[0][(size_t)m * HW + pi];
        fT[m] = flips[1][(size_t)m * HW + pi];
        dlo[m] = flips[2][(size_t)m * HW + pi];
        dhi[m] = flips[3][(size_t)m * HW + pi];
      }
      composite_order(K, Tm.data(), Dm.data(), *o, ord.data());
      double bi, bt;
      composite_bounds(K, Tm.data(), Dm.data(), Cm.data(), fC.data(), fT.data(), dlo.data(),
                       dhi.data(), *o, cmax, cd[1], ord.data(), bi, bt);
      // each ambiguous saturation decision: the composite with that partial's other
      // outcome, exactly
      if (has_alt) {
        double base3[3], baseT;
        composite_one(K, Tm.data(), Cm.data(), ord.data(), *o, base3, baseT);
        for (int m = 0; m < K; ++m) {
          if (!sat_alt[(size_t)m * HW + pi]) continue;
          std::vector<double> T2 = Tm, D2 = Dm, C2 = Cm;
          for (int ch = 0; ch < 3; ++ch) C2[3 * m + ch] = alt[((size_t)m * 5 + ch) * HW + pi];
          T2[m] = alt[((size_t)m * 5 + 3) * HW + pi];
          D2[m] = alt[((size_t)m * 5 + 4) * HW + pi];
          std::vector<int> ord2(K);
          composite_order(K, T2.data(), D2.data(), *o, ord2.data());
          double alt3[3], altT;
          composite_one(K, T2.data(), C2.data(), ord2.data(), *o, alt3, altT);
          double d = 0.0;
          for (int ch = 0; ch < 3; ++ch) d = std::max(d, std::fabs(alt3[ch] - base3[ch]));
          bi += d;
          bt += std::fabs(altT - baseT);
        }
      }
      if (bd->image) bd->image[pi] = bi;
      if (bd->T) bd->T[pi] = bt;
    }
  }
  if (Cp) std::memcpy(Cp, C.data(), C.size() * sizeof(double));
  if (Tp) std::memcpy(Tp, T.data(), T.size() * sizeof(double));
  if (Dp) std::memcpy(Dp, D.data(), D.size() * sizeof(double));
  if (amb) std::memcpy(amb, a.data(), HW);
  if (sep) {
    // monolithic contributor lists without termination, subset id per contributor
    orc_opts o2 = *o;
    o2.eps_T = 0.0;
    Subset s = prepare(*p, *cam, o->tile, (float)o->alpha_min);
    const int W = cam->width, H = cam->height, B = o->tile;
    const int nt = s.tiles.tw * s.tiles.th;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nt; ++t) {
      if (tile_mask && !tile_mask[t]) continue;
      const int tx = t % s.tiles.tw, ty = t / s.tiles.tw;
      const int32_t* lst = s.tiles.list.data() + s.tiles.start[t];
      const int64_t cnt = s.tiles.start[t + 1] - s.tiles.start[t];
      std::vector<Frag> fr;
      std::vector<double> Tm(K), Dm(K);
      std::vector<int> ord(K), rank(K);
      for (int py = ty * B; py < std::min(H, (ty + 1) * B); ++py)
        for (int px = tx * B; px < std::min(W, (tx + 1) * B); ++px) {
          const int64_t pi = (int64_t)py * W + px;
          fr.clear();
          double c3[3], tt, dd;
          int32_t lg, nc;
          int64_t ev = 0;
          blend_pixel(px, py, lst, cnt, s.bins, s.pr, o2, c3, tt, dd, lg, nc, ev, &fr);
          for (int m = 0; m < K; ++m) { Tm[m] = T[(size_t)m * HW + pi]; Dm[m] = D[(size_t)m * HW + pi]; }
          composite_order(K, Tm.data(), Dm.data(), *o, ord.data());
          for (int j = 0; j < K; ++j) rank[ord[j]] = j;
          int ok = 1, prev_rank = -1, prev_m = -1;
          for (const Frag& f : fr) {
            int m = (int)(std::upper_bound(offsets, offsets + K + 1, (int64_t)f.g) - offsets) - 1;
            if (m == prev_m) continue;
            if (rank[m] <= prev_rank) { ok = 0; break; }
            prev_rank = rank[m];
            prev_m = m;
          }
          sep[pi] = (uint8_t)ok;
        }
    }
  }
  return 0;
}

int orc_render_view(const orc_params* p, const int64_t* offsets, int32_t K, const orc_camera* cam,
                    const orc_opts* o, const uint8_t* tile_mask, const int32_t* order,
                    const float* cells, double* out, double* Tout, double* Cp, double* Tp,
                    double* Dp, uint8_t* amb, uint8_t* sep, uint8_t* skip_out, int64_t* stats,
                    orc_bounds* bd) {
  return render_view_impl(p, offsets, K, cam, o, tile_mask, order, cells, out, Tout, Cp, Tp, Dp,
                          amb, sep, skip_out, stats, bd, nullptr, nullptr, nullptr);
}

// orc_render_view with the view's stale saturation state (Sec. 4.2 step 2; render_partials
// gives the rule): sat_in [H][W] (required, with order) prunes ranks >= sat_in at each
// pixel; sat_out [H][W] receives the state re-evaluated from this render's partials and
// sat_amb [H][W] (nullable) the pixels whose re-evaluation met a prefix within the AMB_SAT
// band of eps_comp.
int orc_render_view_pruned(const orc_params* p, const int64_t* offsets, int32_t K,
                           const orc_camera* cam, const orc_opts* o, const uint8_t* tile_mask,
                           const int32_t* order, const float* cells, double* out, double* Tout,
                           double* Cp, double* Tp, double* Dp, uint8_t* amb, uint8_t* skip_out,
                           int64_t* stats, orc_bounds* bd, const uint8_t* sat_in,
                           uint8_t* sat_out, uint8_t* sat_amb) {
  if (!order || !sat_in) return -1;
  return render_view_impl(p, offsets, K, cam, o, tile_mask, order, cells, out, Tout, Cp, Tp, Dp,
                          amb, nullptr, skip_out, stats, bd, sat_in, sat_out, sat_amb);
}

// Backward of one view [Eq. 6-7 and the chain through Eq. 1-4 and the projection].
// dLdC [3][H][W] and dLdT [H][W] (nullable) are the loss gradients w.r.t. the composited
// image and total transmittance.  Gradients are written (not accumulated) to g.
// tile_mask (nullable) restricts the adjoint to pixels of tiles with a nonzero entry,
// as if dLdC and dLdT were zero elsewhere.
static int backward_view_impl(const orc_params* p, const int64_t* offsets, int32_t K,
                              const orc_camera* cam, const orc_opts* o, const double* dLdC,
                              const double* dLdT, const uint8_t* tile_mask, const int32_t* order,
                              const float* cells, const orc_grads* gr, const uint8_t* sat_in) {
  const int W = cam->width, H = cam->height, B = o->tile;
  const int64_t HW = (int64_t)W * H;
  const int nc = (p->sh_degree + 1) * (p->sh_degree + 1);
  CrossFilter cf;
  if (cells) cf = make_filter(*p, offsets, K, *cam, *o, cells);
  const CrossFilter* fp = cells ? &cf : nullptr;
  std::vector<Subset> subs(K);
  for (int m = 0; m < K; ++m) {
    orc_params q = slice(*p, offsets[m], offsets[m + 1]);
    subs[m] = prepare(q, *cam, B, (float)o->alpha_min, fp, m, offsets[m]);
  }
  std::vector<double> C, T, D;
  std::vector<uint8_t> skip, pskip;
  render_partials(*p, offsets, K, *cam, *o, tile_mask, order, C, T, D, skip, nullptr, nullptr, fp,
                  &pskip, nullptr, nullptr, nullptr, nullptr, sat_in);
  // per-Gaussian 2-D gradients: u, v, A, B, C, o, r, g, b (threads add atomically)
  std::vector<double> g2((size_t)p->n * 9, 0.0);
  const int tw = (W + B - 1) / B, th = (H + B - 1) / B;
#pragma omp parallel
  {
    std::vector<Frag> fr;
    std::vector<double> Tm(K), Dm(K), gT(K), gC((size_t)K * 3), Pj(K + 1);
    std::vector<int> ord(K);
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < tw * th; ++t) {
      if (tile_mask && !tile_mask[t]) continue;
      const int tx = t % tw, ty = t / tw;
      for (int py = ty * B; py < std::min(H, (ty + 1) * B); ++py)
        for (int px = tx * B; px < std::min(W, (tx + 1) * B); ++px) {
          const int64_t pi = (int64_t)py * W + px;
          const double g[3] = {dLdC[pi], dLdC[HW + pi], dLdC[2 * HW + pi]};
          const double gTo = dLdT ? dLdT[pi] : 0.0;
          // composite adjoint [Eq. 6-7]
          for (int m = 0; m < K; ++m) { Tm[m] = T[(size_t)m * HW + pi]; Dm[m] = D[(size_t)m * HW + pi]; }
          composite_order(K, Tm.data(), Dm.data(), *o, ord.data());
          int L = 0;
          double P = 1.0;
          for (int j = 0; j < K; ++j) {
            if (P < o->eps_comp) break;
            Pj[j] = P;
            P *= Tm[ord[j]];
            ++L;
          }
          std::fill(gT.begin(), gT.end(), 0.0);
          std::fill(gC.begin(), gC.end(), 0.0);
          double S[3] = {o->bg[0], o->bg[1], o->bg[2]}, Rt = 1.0;
          for (int j = L - 1; j >= 0; --j) {
            const int m = ord[j];
            for (int ch = 0; ch < 3; ++ch) gC[3 * m + ch] = g[ch] * Pj[j];
            gT[m] = (g[0] * S[0] + g[1] * S[1] + g[2] * S[2]) * Pj[j] + gTo * Pj[j] * Rt;
            for (int ch = 0; ch < 3; ++ch) S[ch] = C[((size_t)m * 3 + ch) * HW + pi] + Tm[m] * S[ch];
            Rt *= Tm[m];
          }
          // local-render adjoint per subset, back to front
          for (int j = 0; j < L; ++j) {
            const int m = ord[j];
            // not rendered (the tile or the pixel left empty): no contributors
            if (skip[(size_t)m * tw * th + t] || pskip[(size_t)m * HW + pi]) continue;
            const Subset& s = subs[m];
            const int32_t* lst = s.tiles.list.data() + s.tiles.start[t];
            const int64_t cnt = s.tiles.start[t + 1] - s.tiles.start[t];
            fr.clear();
            double c3[3], tt, dd;
            int32_t lg, ncn;
            int64_t ev = 0;
            blend_pixel(px, py, lst, cnt, s.bins, s.pr, *o, c3, tt, dd, lg, ncn, ev, &fr);
            const double Tf = tt;
            double Bc[3] = {0, 0, 0};
            for (int k = (int)fr.size() - 1; k >= 0; --k) {
              const Frag& f = fr[k];
              const Proj& q = s.pr[f.g];
              double ga = 0.0;
              for (int ch = 0; ch < 3; ++ch)
                ga += gC[3 * m + ch] * (q.col[ch] * f.T - Bc[ch] / (1.0 - f.alpha));
              ga += gT[m] * (-Tf / (1.0 - f.alpha));
              double add[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
              for (int ch = 0; ch < 3; ++ch) add[6 + ch] = gC[3 * m + ch] * f.alpha * f.T;
              if (!f.clamped) {
                add[5] = ga * f.ex;
                const double gp = ga * f.alpha;
                add[0] = (q.A * f.dx + q.B * f.dy) * gp;
                add[1] = (q.C * f.dy + q.B * f.dx) * gp;
                add[2] = -0.5 * f.dx * f.dx * gp;
                add[3] = -f.dx * f.dy * gp;
                add[4] = -0.5 * f.dy * f.dy * gp;
              }
              double* G = g2.data() + (size_t)(offsets[m] + f.g) * 9;
              for (int e = 0; e < 9; ++e) {
#pragma omp atomic
                G[e] += add[e];
              }
              for (int ch = 0; ch < 3; ++ch) Bc[ch] += q.col[ch] * f.alpha * f.T;
            }
          }
        }
    }
  }
  // projection adjoint per Gaussian
  double Rc[9];
  for (int k = 0; k < 9; ++k) Rc[k] = cam->R[k];
  const double fx = cam->fx, fy = cam->fy;
#pragma omp parallel for schedule(static)
  for (int64_t gi = 0; gi < p->n; ++gi) {
    double* gm = gr->means + 3 * gi;
    double* gls = gr->log_scales + 3 * gi;
    double* gq = gr->quats + 4 * gi;
    double* gsh = gr->sh + gi * nc * 3;
    for (int k = 0; k < 3; ++k) { gm[k] = 0; gls[k] = 0; }
    for (int k = 0; k < 4; ++k) gq[k] = 0;
    gr->opacity_logits[gi] = 0;
    for (int k = 0; k < nc * 3; ++k) gsh[k] = 0;
    const double* G = g2.data() + (size_t)gi * 9;
    bool any = false;
    for (int k = 0; k < 9; ++k) any = any || G[k] != 0.0;
    if (!any) continue;
    int m = (int)(std::upper_bound(offsets, offsets + K + 1, gi) - offsets) - 1;
    orc_params q = slice(*p, offsets[m], offsets[m + 1]);
    const Proj& g = subs[m].pr[gi - offsets[m]];
    // opacity
    gr->opacity_logits[gi] = G[5] * g.o * (1.0 - g.o);
    // colour -> SH coefficients and viewing direction
    double gdir[3] = {0, 0, 0};
    const double* sh = q.sh + (gi - offsets[m]) * nc * 3;
    for (int ch = 0; ch < 3; ++ch) {
      if (g.col_clamped[ch]) continue;
      const double gc = G[6 + ch];
      for (int k = 0; k < nc; ++k) {
        gsh[3 * k + ch] = g.Y[k] * gc;
        for (int e = 0; e < 3; ++e) gdir[e] += sh[3 * k + ch] * g.dY[k][e] * gc;
      }
    }
    const double dd = g.dir[0] * gdir[0] + g.dir[1] * gdir[1] + g.dir[2] * gdir[2];
    for (int e = 0; e < 3; ++e) gm[e] += (gdir[e] - g.dir[e] * dd) / g.dist;
    // conic -> Sigma2D:  H = -Q Gq Q with Gq = [[gA, gB/2], [gB/2, gC]]
    const double Q[2][2] = {{g.A, g.B}, {g.B, g.C}};
    const double Gq[2][2] = {{G[2], 0.5 * G[3]}, {0.5 * G[3], G[4]}};
    double QG[2][2], Hm[2][2];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) QG[i][j] = Q[i][0] * Gq[0][j] + Q[i][1] * Gq[1][j];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) Hm[i][j] = -(QG[i][0] * Q[0][j] + QG[i][1] * Q[1][j]);
    // Sigma2D0 = P P^T  ->  gP = 2 H P
    double gP0[3], gP1[3];
    for (int j = 0; j < 3; ++j) {
      gP0[j] = 2.0 * (Hm[0][0] * g.P0[j] + Hm[0][1] * g.P1[j]);
      gP1[j] = 2.0 * (Hm[1][0] * g.P0[j] + Hm[1][1] * g.P1[j]);
    }
    // P = J V:  gJ = gP V^T,  gV = J^T gP
    double gj00 = 0, gj02 = 0, gj11 = 0, gj12 = 0;
    for (int j = 0; j < 3; ++j) {
      gj00 += gP0[j] * g.V[j];
      gj02 += gP0[j] * g.V[6 + j];
      gj11 += gP1[j] * g.V[3 + j];
      gj12 += gP1[j] * g.V[6 + j];
    }
    double gV[9];
    for (int j = 0; j < 3; ++j) {
      gV[j] = g.j00 * gP0[j];
      gV[3 + j] = g.j11 * gP1[j];
      gV[6 + j] = g.j02 * gP0[j] + g.j12 * gP1[j];
    }
    // J -> camera-space mean
    const double tx = g.t[0], ty = g.t[1], tz = g.t[2];
    double gt[3] = {0, 0, 0};
    gt[2] += -fx / (tz * tz) * gj00;
    gt[2] += -fy / (tz * tz) * gj11;
    if (!g.clx) { gt[0] += -fx / (tz * tz) * gj02; gt[2] += 2.0 * fx * tx / (tz * tz * tz) * gj02; }
    else { gt[2] += fx * g.rx / (tz * tz) * gj02; }
    if (!g.cly) { gt[1] += -fy / (tz * tz) * gj12; gt[2] += 2.0 * fy * ty / (tz * tz * tz) * gj12; }
    else { gt[2] += fy * g.ry / (tz * tz) * gj12; }
    // 2-D mean
    gt[0] += fx / tz * G[0];
    gt[2] += -fx * tx / (tz * tz) * G[0];
    gt[1] += fy / tz * G[1];
    gt[2] += -fy * ty / (tz * tz) * G[1];
    for (int e = 0; e < 3; ++e) gm[e] += Rc[e] * gt[0] + Rc[3 + e] * gt[1] + Rc[6 + e] * gt[2];
    // V = W M:  gM = W^T gV
    double gM[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        gM[3 * i + j] = Rc[i] * gV[j] + Rc[3 + i] * gV[3 + j] + Rc[6 + i] * gV[6 + j];
    // M = Rq diag(s)
    double gR[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) gR[3 * i + j] = gM[3 * i + j] * g.s[j];
    for (int j = 0; j < 3; ++j) {
      double gs = 0;
      for (int i = 0; i < 3; ++i) gs += gM[3 * i + j] * g.Rq[3 * i + j];
      gls[j] = gs * g.s[j];
    }
    // Rq(qhat)
    const double w = g.qhat[0], x = g.qhat[1], y = g.qhat[2], z = g.qhat[3];
    double gw = 0, gx = 0, gy = 0, gz = 0;
    gy += -4 * y * gR[0]; gz += -4 * z * gR[0];
    gx += 2 * y * gR[1]; gy += 2 * x * gR[1]; gw += -2 * z * gR[1]; gz += -2 * w * gR[1];
    gx += 2 * z * gR[2]; gz += 2 * x * gR[2]; gw += 2 * y * gR[2]; gy += 2 * w * gR[2];
    gx += 2 * y * gR[3]; gy += 2 * x * gR[3]; gw += 2 * z * gR[3]; gz += 2 * w * gR[3];
    gx += -4 * x * gR[4]; gz += -4 * z * gR[4];
    gy += 2 * z * gR[5]; gz += 2 * y * gR[5]; gw += -2 * x * gR[5]; gx += -2 * w * gR[5];
    gx += 2 * z * gR[6]; gz += 2 * x * gR[6]; gw += -2 * y * gR[6]; gy += -2 * w * gR[6];
    gy += 2 * z * gR[7]; gz += 2 * y * gR[7]; gw += 2 * x * gR[7]; gx += 2 * w * gR[7];
    gx += -4 * x * gR[8]; gy += -4 * y * gR[8];
    const double gqh[4] = {gw, gx, gy, gz};
    const double dq = w * gw + x * gx + y * gy + z * gz;
    for (int k = 0; k < 4; ++k) gq[k] = (gqh[k] - g.qhat[k] * dq) / g.qnorm;
  }
  return 0;
}

int orc_backward_view(const orc_params* p, const int64_t* offsets, int32_t K,
                      const orc_camera* cam, const orc_opts* o, const double* dLdC,
                      const double* dLdT, const uint8_t* tile_mask, const int32_t* order,
                      const float* cells, const orc_grads* gr) {
  return backward_view_impl(p, offsets, K, cam, o, dLdC, dLdT, tile_mask, order, cells, gr,
                            nullptr);
}

// orc_backward_view of the render with the stale saturation state sat_in [H][W] (the
// partials of orc_render_view_pruned).
int orc_backward_view_pruned(const orc_params* p, const int64_t* offsets, int32_t K,
                             const orc_camera* cam, const orc_opts* o, const double* dLdC,
                             const double* dLdT, const uint8_t* tile_mask, const int32_t* order,
                             const float* cells, const orc_grads* gr, const uint8_t* sat_in) {
  if (!order || !sat_in) return -1;
  return backward_view_impl(p, offsets, K, cam, o, dLdC, dLdT, tile_mask, order, cells, gr,
                            sat_in);
}

// Which clamp branches of the adjoint one view exercises, so that a finite-difference pin
// can show that it reaches each of them.  gflags[n] (visible Gaussians): bit 0 the
// Jacobian's x clamp, bit 1 its y clamp, bits 2-4 the colour clamp of r, g, b.  nclamp[n]:
// the number of pixels (over the K local renders) that blend the Gaussian with alpha held
// at alpha_max, i.e. where dL/do and dL/dpower vanish.
int orc_branch_stats(const orc_params* p, const int64_t* offsets, int32_t K,
                     const orc_camera* cam, const orc_opts* o, int32_t* gflags, int64_t* nclamp) {
  const int W = cam->width, H = cam->height, B = o->tile;
  std::fill(gflags, gflags + p->n, 0);
  std::fill(nclamp, nclamp + p->n, (int64_t)0);
  for (int m = 0; m < K; ++m) {
    orc_params q = slice(*p, offsets[m], offsets[m + 1]);
    const Subset s = prepare(q, *cam, B, (float)o->alpha_min);
    for (int64_t i = 0; i < q.n; ++i) {
      if (!s.bins[i].visible) continue;
      const Proj& g = s.pr[i];
      gflags[offsets[m] + i] = g.clx | (g.cly << 1) | (g.col_clamped[0] << 2) |
                               (g.col_clamped[1] << 3) | (g.col_clamped[2] << 4);
    }
    std::vector<Frag> fr;
    for (int t = 0; t < s.tiles.tw * s.tiles.th; ++t) {
      const int tx = t % s.tiles.tw, ty = t / s.tiles.tw;
      const int32_t* lst = s.tiles.list.data() + s.tiles.start[t];
      const int64_t cnt = s.tiles.start[t + 1] - s.tiles.start[t];
      for (int py = ty * B; py < std::min(H, (ty + 1) * B); ++py)
        for (int px = tx * B; px < std::min(W, (tx + 1) * B); ++px) {
          fr.clear();
          double c3[3], tt, dd;
          int32_t lg, nc;
          int64_t ev = 0;
          blend_pixel(px, py, lst, cnt, s.bins, s.pr, *o, c3, tt, dd, lg, nc, ev, &fr);
          for (const Frag& f : fr)
            if (f.clamped) ++nclamp[offsets[m] + f.g];
        }
    }
  }
  return 0;
}

// Adam with torch.optim.Adam semantics (bias-corrected, eps outside the square root).
void orc_adam(int64_t n, double* p, const double* g, double* m, double* v, double lr, double b1,
              double b2, double eps, int64_t step) {
  const double bc1 = 1.0 - std::pow(b1, (double)step);
  const double bc2 = 1.0 - std::pow(b2, (double)step);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    const double mh = m[i] / bc1;
    const double vh = v[i] / bc2;
    p[i] -= lr * mh / (std::sqrt(vh) + eps);
  }
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
