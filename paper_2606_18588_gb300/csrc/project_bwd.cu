// Backward of the projection (Sec. 2 step 1) and the parameter update (Sec. 2 step 4).
//
// project_bwd: one thread per Gaussian loops over the views of the batch.  For each view
// where the rasteriser left a nonzero 2-D gradient (the moments of dL/dpower / o over the
// pixels, dL/do, dL/dcolour) it recomputes the FP32 projection, consumes and clears that gradient, and
// chains it to the mean (through the 2-D mean, the EWA Jacobian J and the SH viewing
// direction), the SH coefficients, the opacity logit, and - accumulated over views as
// dL/dM for M = R(q) diag(s) - the log-scales and the quaternion.  Results are added
// to the caller's gradient arrays (one thread owns one Gaussian: no atomics), or, in the
// batch's update step, applied at once by Adam from shared memory (k_project_bwd<DEG,
// true>), the blocks without any gradient being left to a streaming zero-gradient pass.
// k_adam is the stand-alone Adam over gradient arrays; all routes share adam_elem.
#include "common.cuh"
#include "spec.cuh"

namespace splx {

namespace {
struct ShC {
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

// Y (value) and sum_k w_k grad Y_k for the real SH basis (same ordering as project.cu).
template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  Y[0] = 0.28209479177387814f;
  if (DEG >= 1) { Y[1] = -ShC::k1 * y; Y[2] = ShC::k1 * z; Y[3] = -ShC::k1 * x; }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = ShC::k2a * x * y; Y[5] = -ShC::k2a * y * z; Y[6] = ShC::k2b * (2.f * zz - xx - yy);
    Y[7] = -ShC::k2a * x * z; Y[8] = ShC::k2c * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -ShC::k3a * y * (3.f * xx - yy); Y[10] = ShC::k3b * x * y * z;
      Y[11] = -ShC::k3c * y * (4.f * zz - xx - yy);
      Y[12] = ShC::k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -ShC::k3c * x * (4.f * zz - xx - yy); Y[14] = ShC::k3e * z * (xx - yy);
      Y[15] = -ShC::k3a * x * (xx - 3.f * yy);
    }
  }
}

template <int DEG>
__device__ __forceinline__ void sh_dir_grad(float x, float y, float z, const float* w, float* gd) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (DEG >= 1) {
    gy += -ShC::k1 * w[1];
    gz += ShC::k1 * w[2];
    gx += -ShC::k1 * w[3];
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += ShC::k2a * y * w[4]; gy += ShC::k2a * x * w[4];
    gy += -ShC::k2a * z * w[5]; gz += -ShC::k2a * y * w[5];
    gx += -2.f * ShC::k2b * x * w[6]; gy += -2.f * ShC::k2b * y * w[6]; gz += 4.f * ShC::k2b * z * w[6];
    gx += -ShC::k2a * z * w[7]; gz += -ShC::k2a * x * w[7];
    gx += 2.f * ShC::k2c * x * w[8]; gy += -2.f * ShC::k2c * y * w[8];
    if (DEG >= 3) {
      gx += -6.f * ShC::k3a * x * y * w[9]; gy += -ShC::k3a * (3.f * xx - 3.f * yy) * w[9];
      gx += ShC::k3b * y * z * w[10]; gy += ShC::k3b * x * z * w[10]; gz += ShC::k3b * x * y * w[10];
      gx += 2.f * ShC::k3c * x * y * w[11]; gy += -ShC::k3c * (4.f * zz - xx - 3.f * yy) * w[11];
      gz += -8.f * ShC::k3c * y * z * w[11];
      gx += -6.f * ShC::k3d * x * z * w[12]; gy += -6.f * ShC::k3d * y * z * w[12];
      gz += ShC::k3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
      gx += -ShC::k3c * (4.f * zz - 3.f * xx - yy) * w[13]; gy += 2.f * ShC::k3c * x * y * w[13];
      gz += -8.f * ShC::k3c * x * z * w[13];
      gx += 2.f * ShC::k3e * x * z * w[14]; gy += -2.f * ShC::k3e * y * z * w[14];
      gz += ShC::k3e * (xx - yy) * w[14];
      gx += -ShC::k3a * (3.f * xx - 3.f * yy) * w[15]; gy += 6.f * ShC::k3a * x * y * w[15];
    }
  }
  gd[0] = gx; gd[1] = gy; gd[2] = gz;
}
}  // namespace

constexpr int kProjBwdThreads = 128;
// Row stride of the shared gradient columns: one float of padding, so that a warp reading
// one Gaussian's consecutive elements (the fused Adam epilogue) hits distinct banks, as do
// the threads writing one element of their own Gaussians.
constexpr int kGs = kProjBwdThreads + 1;
// The views' 2-D gradients of a thread's Gaussian stream through a ring of kRing slots of
// shared memory filled by asynchronous copies (cp.async), kRing - 1 views ahead of the one
// being processed, without holding registers for them.
constexpr int kRing = 3;


// The gradient of one Gaussian g over all views: mean, log-scale, quaternion and opacity
// logit in the outputs, the SH coefficients' in gsh (one column of shared memory, element e
// at gsh[e * kGs]); false (outputs untouched) where no view left a 2-D gradient, with gsh
// zeroed, or untouched when no view kept the Gaussian at all.  Consumes and clears the views' 2-D gradients.  ring / ringb: this
// thread's column of the kRing-slot ring (slot s: float4s at ring[(2 s + k) *
// kProjBwdThreads], k = 0, 1, and the ninth value at ringb[s * kProjBwdThreads]).
template <int DEG>
__device__ __forceinline__ bool proj_grads(const BatchDev& b, const int64_t g, float* gsh,
                                           float4* ring, float* ringb,
                                           float (&out_m)[3], float (&out_ls)[3],
                                           float (&out_q)[4], float& out_logit) {
  constexpr int NC = (DEG + 1) * (DEG + 1);
  if (b.counts) {
    // a Gaussian that no view kept has no 2-D gradient: leave before reading its
    // parameters (most of a large scene that a few views see); all counts loads in flight
    uint32_t seen = 0u;
    for (int v = 0; v < b.V; ++v) seen |= b.counts[(int64_t)v * b.N + g];
    if (!seen) return false;  // (gsh untouched)
  }
  const int k = subset_of(b, g);
  const SubsetDev& S = b.subsets[k];
  const int64_t i = g - b.goff[k];
  float m[3], ls[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) { m[e] = S.means[3 * i + e]; ls[e] = S.log_scales[3 * i + e]; }
  const float4 qv = reinterpret_cast<const float4*>(S.quats)[i];
  const float qn = sqrtf(qv.x * qv.x + qv.y * qv.y + qv.z * qv.z + qv.w * qv.w);
  const float qw = qv.x / qn, qx = qv.y / qn, qy = qv.z / qn, qz = qv.w / qn;
  float Rq[9];
  Rq[0] = 1.f - 2.f * (qy * qy + qz * qz); Rq[1] = 2.f * (qx * qy - qw * qz); Rq[2] = 2.f * (qx * qz + qw * qy);
  Rq[3] = 2.f * (qx * qy + qw * qz); Rq[4] = 1.f - 2.f * (qx * qx + qz * qz); Rq[5] = 2.f * (qy * qz - qw * qx);
  Rq[6] = 2.f * (qx * qz - qw * qy); Rq[7] = 2.f * (qy * qz + qw * qx); Rq[8] = 1.f - 2.f * (qx * qx + qy * qy);
  const float s[3] = {exp_spec(ls[0]), exp_spec(ls[1]), exp_spec(ls[2])};
  float M[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * s[c];
  const float o = 1.0f / (1.0f + __expf(-S.opacity_logits[i]));
  // SH coefficients are read per visible view (L1-resident) and their gradient sums live in
  // shared memory (one column per thread): 96 fewer registers, so more warps hide the
  // latency of the per-view 2-D gradient loads
  const float* shp = S.sh + i * NC * 3;

  float gm[3] = {0.f, 0.f, 0.f}, gM[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) gM[e] = 0.f;
  float glogit = 0.f;
#pragma unroll
  for (int e = 0; e < NC * 3; ++e) gsh[e * kGs] = 0.f;
  bool any = false;

  // Only views in which the Gaussian was projected (tile count > 0) can hold a 2-D
  // gradient.  Per chunk of up to 64 views: the counts give the chunk's mask of such views
  // (all loads in flight together), whose gradients then stream through the ring in view
  // order; a slot is refilled one view after it was read (its loads have returned: the
  // zero test below consumed them)
  auto seen_in = [&](int v) { return !b.counts || b.counts[(int64_t)v * b.N + g] != 0u; };
  for (int v0 = 0; v0 < b.V; v0 += 64) {
    const int vn = b.V - v0 < 64 ? b.V - v0 : 64;
    uint64_t vm = 0;
    for (int q = 0; q < vn; ++q)
      if (seen_in(v0 + q)) vm |= 1ull << q;
    uint64_t pend = vm;  // views not yet copied
    auto issue = [&](int s) {
      if (pend) {
        const int q = __ffsll((long long)pend) - 1;
        pend &= pend - 1;
        const float4* src = b.grad2d + ((int64_t)(v0 + q) * b.N + g) * 3;
        cp_async16(ring + (2 * s) * kProjBwdThreads, src);
        cp_async16(ring + (2 * s + 1) * kProjBwdThreads, src + 1);
        cp_async4(ringb + s * kProjBwdThreads, &src[2].x);
      }
      cp_async_commit();  // one group per call, empty or not
    };
#pragma unroll
    for (int s0 = 0; s0 < kRing; ++s0) issue(s0);
    int slot = 0;
    bool first = true;
    while (vm) {
      const int v = v0 + __ffsll((long long)vm) - 1;
      vm &= vm - 1;
      if (!first) issue(slot == 0 ? kRing - 1 : slot - 1);
      first = false;
      cp_async_wait<kRing - 1>();  // this view's group, the oldest outstanding, has landed
      const float4 G0 = ring[(2 * slot) * kProjBwdThreads];
      const float4 G1 = ring[(2 * slot + 1) * kProjBwdThreads];
      const float gbl = ringb[slot * kProjBwdThreads];
      slot = slot + 1 == kRing ? 0 : slot + 1;
      float4* gp = b.grad2d + ((int64_t)v * b.N + g) * 3;
      if (G0.x == 0.f && G0.y == 0.f && G0.z == 0.f && G0.w == 0.f && G1.x == 0.f && G1.y == 0.f &&
          G1.z == 0.f && G1.w == 0.f && gbl == 0.f)
        continue;
      any = true;
      gp[0] = make_float4(0.f, 0.f, 0.f, 0.f);
      gp[1] = make_float4(0.f, 0.f, 0.f, 0.f);
      gp[2].x = 0.f;
      const ViewDev& cam = b.views[v];
      const float* R = cam.R;
      const float tx = R[0] * m[0] + R[1] * m[1] + R[2] * m[2] + cam.t[0];
      const float ty = R[3] * m[0] + R[4] * m[1] + R[5] * m[2] + cam.t[1];
      const float tz = R[6] * m[0] + R[7] * m[1] + R[8] * m[2] + cam.t[2];
      const float fx = cam.fx, fy = cam.fy;
      const float itz = 1.0f / tz;
      const float limx = 1.3f * 0.5f * (float)cam.W / fx, limy = 1.3f * 0.5f * (float)cam.H / fy;
      const float rx = tx * itz, ry = ty * itz;
      const bool clx = rx < -limx || rx > limx, cly = ry < -limy || ry > limy;
      const float rxc = fminf(limx, fmaxf(-limx, rx)), ryc = fminf(limy, fmaxf(-limy, ry));
      const float j00 = fx * itz, j02 = -fx * rxc * itz, j11 = fy * itz, j12 = -fy * ryc * itz;
      float V[9];
  #pragma unroll
      for (int r = 0; r < 3; ++r)
  #pragma unroll
        for (int c = 0; c < 3; ++c)
          V[3 * r + c] = R[3 * r] * M[c] + R[3 * r + 1] * M[3 + c] + R[3 * r + 2] * M[6 + c];
      float P0[3], P1[3];
  #pragma unroll
      for (int c = 0; c < 3; ++c) {
        P0[c] = j00 * V[c] + j02 * V[6 + c];
        P1[c] = j11 * V[3 + c] + j12 * V[6 + c];
      }
      const float a0 = P0[0] * P0[0] + P0[1] * P0[1] + P0[2] * P0[2];
      const float c0 = P1[0] * P1[0] + P1[1] * P1[1] + P1[2] * P1[2];
      const float bb = P0[0] * P1[0] + P0[1] * P1[1] + P0[2] * P1[2];
      const float d01 = P0[0] * P1[1] - P0[1] * P1[0];
      const float d02 = P0[0] * P1[2] - P0[2] * P1[0];
      const float d12 = P0[1] * P1[2] - P0[2] * P1[1];
      const float det = d01 * d01 + d02 * d02 + d12 * d12 + 0.3f * (a0 + c0) + 0.09f;
      const float idet = 1.0f / det;
      const float QA = (c0 + 0.3f) * idet, QB = -bb * idet, QC = (a0 + 0.3f) * idet;
      // the rasteriser's moments of dL/dpower / o -> dL/du, dL/dv and dL/d(A, B, C) of the
      // conic: power = -(A dx^2 + 2 B dx dy + C dy^2) / 2 with (dx, dy) = pixel - (u, v)
      const float mx = o * G0.x, my = o * G0.y;
      const float gu = QA * mx + QB * my, gv = QB * mx + QC * my;
      const float gA = -0.5f * o * G0.z, gB = -o * G0.w, gCc = -0.5f * o * G1.x, go = G1.y;
      const float gcol[3] = {G1.z, G1.w, gbl};
      glogit += go * o * (1.0f - o);
      // colour -> SH coefficients and viewing direction
      float dx = m[0] - cam.eye[0], dy = m[1] - cam.eye[1], dz = m[2] - cam.eye[2];
      const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
      const float idist = 1.0f / dist;
      dx *= idist; dy *= idist; dz *= idist;
      float Y[NC];
      sh_basis<DEG>(dx, dy, dz, Y);
      float gc[3];
  #pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float raw = 0.5f;
  #pragma unroll
        for (int kk = 0; kk < NC; ++kk) raw = fmaf(Y[kk], __ldg(shp + 3 * kk + ch), raw);
        gc[ch] = raw < 0.0f ? 0.0f : gcol[ch];
      }
      float w[NC];
  #pragma unroll
      for (int kk = 0; kk < NC; ++kk) {
        gsh[(3 * kk + 0) * kGs] += Y[kk] * gc[0];
        gsh[(3 * kk + 1) * kGs] += Y[kk] * gc[1];
        gsh[(3 * kk + 2) * kGs] += Y[kk] * gc[2];
        w[kk] = __ldg(shp + 3 * kk) * gc[0] + __ldg(shp + 3 * kk + 1) * gc[1] +
                __ldg(shp + 3 * kk + 2) * gc[2];
      }
      if (DEG > 0) {
        float gd[3];
        sh_dir_grad<DEG>(dx, dy, dz, w, gd);
        const float dd = dx * gd[0] + dy * gd[1] + dz * gd[2];
        gm[0] += (gd[0] - dx * dd) * idist;
        gm[1] += (gd[1] - dy * dd) * idist;
        gm[2] += (gd[2] - dz * dd) * idist;
      }
      // conic -> Sigma2D:  H = -Q Gq Q,  Gq = [[gA, gB/2], [gB/2, gC]]
      const float hB = 0.5f * gB;
      const float QG00 = QA * gA + QB * hB, QG01 = QA * hB + QB * gCc;
      const float QG10 = QB * gA + QC * hB, QG11 = QB * hB + QC * gCc;
      const float H00 = -(QG00 * QA + QG01 * QB), H01 = -(QG00 * QB + QG01 * QC);
      const float H10 = -(QG10 * QA + QG11 * QB), H11 = -(QG10 * QB + QG11 * QC);
      // Sigma2D0 = P P^T  ->  gP = 2 H P
      float gP0[3], gP1[3];
  #pragma unroll
      for (int c = 0; c < 3; ++c) {
        gP0[c] = 2.f * (H00 * P0[c] + H01 * P1[c]);
        gP1[c] = 2.f * (H10 * P0[c] + H11 * P1[c]);
      }
      // P = J V
      const float gj00 = gP0[0] * V[0] + gP0[1] * V[1] + gP0[2] * V[2];
      const float gj02 = gP0[0] * V[6] + gP0[1] * V[7] + gP0[2] * V[8];
      const float gj11 = gP1[0] * V[3] + gP1[1] * V[4] + gP1[2] * V[5];
      const float gj12 = gP1[0] * V[6] + gP1[1] * V[7] + gP1[2] * V[8];
      float gV[9];
  #pragma unroll
      for (int c = 0; c < 3; ++c) {
        gV[c] = j00 * gP0[c];
        gV[3 + c] = j11 * gP1[c];
        gV[6 + c] = j02 * gP0[c] + j12 * gP1[c];
      }
      // J and the 2-D mean -> camera-space mean
      const float itz2 = itz * itz;
      float gtx = 0.f, gty = 0.f, gtz = 0.f;
      gtz += -fx * itz2 * gj00 - fy * itz2 * gj11;
      if (!clx) { gtx += -fx * itz2 * gj02; gtz += 2.f * fx * tx * itz2 * itz * gj02; }
      else { gtz += fx * rxc * itz2 * gj02; }
      if (!cly) { gty += -fy * itz2 * gj12; gtz += 2.f * fy * ty * itz2 * itz * gj12; }
      else { gtz += fy * ryc * itz2 * gj12; }
      gtx += fx * itz * gu;
      gtz += -fx * tx * itz2 * gu;
      gty += fy * itz * gv;
      gtz += -fy * ty * itz2 * gv;
  #pragma unroll
      for (int e = 0; e < 3; ++e) gm[e] += R[e] * gtx + R[3 + e] * gty + R[6 + e] * gtz;
      // V = W M  ->  gM += W^T gV
  #pragma unroll
      for (int r = 0; r < 3; ++r)
  #pragma unroll
        for (int c = 0; c < 3; ++c)
          gM[3 * r + c] += R[r] * gV[c] + R[3 + r] * gV[3 + c] + R[6 + r] * gV[6 + c];
    }
    cp_async_wait<0>();  // the chunk's ring is idle before the next chunk refills it
  }
  if (!any) return false;
  // M = Rq diag(s)
  float gR[9], gls[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) gR[3 * r + c] = gM[3 * r + c] * s[c];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    gls[c] = (gM[c] * Rq[c] + gM[3 + c] * Rq[3 + c] + gM[6 + c] * Rq[6 + c]) * s[c];
  float gw = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
  gy += -4.f * qy * gR[0]; gz += -4.f * qz * gR[0];
  gx += 2.f * qy * gR[1]; gy += 2.f * qx * gR[1]; gw += -2.f * qz * gR[1]; gz += -2.f * qw * gR[1];
  gx += 2.f * qz * gR[2]; gz += 2.f * qx * gR[2]; gw += 2.f * qy * gR[2]; gy += 2.f * qw * gR[2];
  gx += 2.f * qy * gR[3]; gy += 2.f * qx * gR[3]; gw += 2.f * qz * gR[3]; gz += 2.f * qw * gR[3];
  gx += -4.f * qx * gR[4]; gz += -4.f * qz * gR[4];
  gy += 2.f * qz * gR[5]; gz += 2.f * qy * gR[5]; gw += -2.f * qx * gR[5]; gx += -2.f * qw * gR[5];
  gx += 2.f * qz * gR[6]; gz += 2.f * qx * gR[6]; gw += -2.f * qy * gR[6]; gy += -2.f * qw * gR[6];
  gy += 2.f * qz * gR[7]; gz += 2.f * qy * gR[7]; gw += 2.f * qx * gR[7]; gx += 2.f * qw * gR[7];
  gx += -4.f * qx * gR[8]; gy += -4.f * qy * gR[8];
  const float dq = qw * gw + qx * gx + qy * gy + qz * gz;
  const float iqn = 1.0f / qn;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    out_m[e] = gm[e];
    out_ls[e] = gls[e];
  }
  out_q[0] = (gw - qw * dq) * iqn;
  out_q[1] = (gx - qx * dq) * iqn;
  out_q[2] = (gy - qy * dq) * iqn;
  out_q[3] = (gz - qz * dq) * iqn;
  out_logit = glogit;
  return true;
}

// One Adam element with torch.optim.Adam semantics (step_lr = lr / (1 - b1^t),
// bc2_sqrt_inv = 1 / sqrt(1 - b2^t)), each operation rounded as written, so that the
// stand-alone update and the one fused into the projection adjoint agree bit for bit.
__device__ __forceinline__ void adam_elem(float& p, const float g, float& m, float& v,
                                          const float step_lr, const float b1, const float b2,
                                          const float bc2_sqrt_inv, const float eps) {
  m = __fadd_rn(__fmul_rn(b1, m), __fmul_rn(__fsub_rn(1.0f, b1), g));
  v = __fadd_rn(__fmul_rn(b2, v), __fmul_rn(__fmul_rn(__fsub_rn(1.0f, b2), g), g));
  p = __fsub_rn(p, __fdiv_rn(__fmul_rn(step_lr, m),
                             __fadd_rn(__fmul_rn(__fsqrt_rn(v), bc2_sqrt_inv), eps)));
}

// Bias-corrected learning rates of a step, in double precision once per CTA (FP64 is
// slow on this part): [0] lr_group / bc1 for the 6 groups, [6] 1 / sqrt(bc2).
__device__ __forceinline__ void adam_scales(const AdamTable& at, float* sc) {
  if (threadIdx.x == 0) {
    const int64_t step = at.step_dev ? *at.step_dev : at.step;
    const double bc1 = 1.0 - pow((double)at.b1, (double)step);
    const double bc2 = 1.0 - pow((double)at.b2, (double)step);
    for (int j = 0; j < 6; ++j) sc[j] = (float)(at.lr[j] / bc1);
    sc[6] = (float)(1.0 / sqrt(bc2));
  }
  __syncthreads();
}

// The fused epilogue's view of one parameter array of the CTA's ng Gaussians (W floats
// each) when they all lie in one subset: E = ng W contiguous floats of p, m and v, and the
// gradient of element idx (CTA Gaussian j = idx / W, element e) at rows[e * kGs + j].
template <int W>
struct AdamSpan {
  float* p;
  float* m;
  float* v;
  const float* rows;
  int E;
  float lr_lo, lr_hi;  // elements e < 3, e >= 3 (the SH coefficients above degree 0)
};

template <int W>
__device__ __forceinline__ AdamSpan<W> adam_span(const AdamTable& at, const int a, const int k,
                                                 const int64_t i0, const float* rows, const int ng,
                                                 const float lr_lo, const float lr_hi) {
  const int64_t o = i0 * W;
  return AdamSpan<W>{at.p[k][a] + o, at.m[k][a] + o, at.v[k][a] + o, rows, ng * W, lr_lo, lr_hi};
}

// Loads kU elements of p, m and v per thread (elements base + u * kProjBwdThreads) ...
template <int W, int kU>
__device__ __forceinline__ void span_load(const AdamSpan<W>& sp, const int base, float (&pv)[kU],
                                          float (&mv)[kU], float (&vv)[kU]) {
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int idx = base + u * kProjBwdThreads;
    if (idx < sp.E) {
      pv[u] = sp.p[idx];
      mv[u] = sp.m[idx];
      vv[u] = sp.v[idx];
    }
  }
}

// ... and updates and stores them.
template <int W, int kU>
__device__ __forceinline__ void span_update(const AdamSpan<W>& sp, const int base, float (&pv)[kU],
                                            float (&mv)[kU], float (&vv)[kU], const float b1,
                                            const float b2, const float bci, const float eps) {
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int idx = base + u * kProjBwdThreads;
    if (idx < sp.E) {
      const int j = idx / W, e = idx - j * W;
      adam_elem(pv[u], sp.rows[e * kGs + j], mv[u], vv[u], e < 3 ? sp.lr_lo : sp.lr_hi, b1, b2,
                bci, eps);
      sp.p[idx] = pv[u];
      sp.m[idx] = mv[u];
      sp.v[idx] = vv[u];
    }
  }
}

// Adam over array a of the CTA's ng Gaussians (W floats each) element by element, for a CTA
// whose Gaussians straddle a subset boundary: element e of CTA Gaussian j lives in subset
// s_k[j] at local index s_i[j].
template <int W>
__device__ __forceinline__ void adam_rows_split(const AdamTable& at, const int a,
                                                const float* rows, const int* s_k,
                                                const int64_t* s_i, const int ng,
                                                const float lr_lo, const float lr_hi,
                                                const float b1, const float b2, const float bci,
                                                const float eps) {
  for (int idx = threadIdx.x; idx < ng * W; idx += kProjBwdThreads) {
    const int j = idx / W, e = idx - j * W;
    const int k = s_k[j];
    const int64_t off = s_i[j] * W + e;
    float* pp = at.p[k][a] + off;
    float* mp = at.m[k][a] + off;
    float* vp = at.v[k][a] + off;
    float pv = *pp, mv = *mp, vv = *vp;
    adam_elem(pv, rows[e * kGs + j], mv, vv, e < 3 ? lr_lo : lr_hi, b1, b2, bci, eps);
    *pp = pv;
    *mp = mv;
    *vp = vv;
  }
}

template <int DEG, bool kFuse>
__global__ void __launch_bounds__(kProjBwdThreads, 4)
    k_project_bwd(const BatchDev b, const GradTable gt, const AdamTable at) {
  constexpr int NC = (DEG + 1) * (DEG + 1);
  // gradient columns, one per thread: with kFuse rows 0-10 hold mean (3), log-scale (3),
  // quaternion (4) and opacity logit, the SH rows follow
  constexpr int kHead = kFuse ? 11 : 0;
  __shared__ float s_grad[(kHead + NC * 3) * kGs];
  __shared__ float4 s_ring[kRing * 2 * kProjBwdThreads];
  __shared__ float s_ringb[kRing * kProjBwdThreads];
  float* gsh = s_grad + kHead * kGs + threadIdx.x;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
  float glogit = 0.f;
  bool any = false;
  if (g < b.N) {
    any = proj_grads<DEG>(b, g, gsh, s_ring + threadIdx.x, s_ringb + threadIdx.x, gm, gls, gq,
                          glogit);
  }
  if constexpr (!kFuse) {
    // add into the caller's gradient arrays (one thread owns one Gaussian: no atomics)
    if (!any) return;
    const int k = subset_of(b, g);
    const int64_t i = g - b.goff[k];
    float* const* P = gt.p[k];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      P[0][3 * i + e] += gm[e];
      P[1][3 * i + e] += gls[e];
    }
    float4* gq4 = reinterpret_cast<float4*>(P[2]) + i;
    float4 cur = *gq4;
    cur.x += gq[0];
    cur.y += gq[1];
    cur.z += gq[2];
    cur.w += gq[3];
    *gq4 = cur;
    P[3][i] += glogit;
#pragma unroll
    for (int e = 0; e < NC * 3; ++e) P[4][i * NC * 3 + e] += gsh[e * kGs];
  } else {
    // Adam on every parameter of the CTA's Gaussians straight from these gradients (zero
    // where a Gaussian has none, as after zero_grad): no gradient array is written or read.
    // The CTA's Gaussians are contiguous within each subset's arrays, so the threads walk
    // each array's range with unit stride (coalesced loads and stores), taking the
    // gradients from the shared columns.
    __shared__ float s_sc[7];
    __shared__ int s_k[kProjBwdThreads];
    __shared__ int64_t s_i[kProjBwdThreads];
    if (at.defer) {
      // a block without any gradient (most of a large scene that few views see) is left
      // to the zero-gradient pass, which streams it at full occupancy
      const bool cta_any = __syncthreads_or(any) != 0;
      if (threadIdx.x == 0) at.defer[blockIdx.x] = cta_any ? 0 : 1;
      if (!cta_any) return;
    }
    if (!any) {  // a zero gradient (and a column proj_grads may have left untouched)
#pragma unroll
      for (int e = 0; e < NC * 3; ++e) gsh[e * kGs] = 0.f;
    }
    float* col = s_grad + threadIdx.x;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      col[e * kGs] = gm[e];
      col[(3 + e) * kGs] = gls[e];
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) col[(6 + e) * kGs] = gq[e];
    col[10 * kGs] = glogit;
    if (g < b.N) {
      const int k = subset_of(b, g);
      s_k[threadIdx.x] = k;
      s_i[threadIdx.x] = g - b.goff[k];
    }
    adam_scales(at, s_sc);  // (its barrier also publishes the columns above)
    const int64_t rest = b.N - (int64_t)blockIdx.x * kProjBwdThreads;
    const int ng = rest < kProjBwdThreads ? (int)rest : kProjBwdThreads;
    const float b1 = at.b1, b2 = at.b2, eps = at.eps, bci = s_sc[6];
    if (s_k[0] == s_k[ng - 1]) {
      // one subset: contiguous ranges.  The four small arrays hold at most 3 + 3 + 4 + 1
      // elements per thread, all loaded before any update (33 loads in flight per thread);
      // the SH array follows in batches of 16 elements per thread
      const int k = s_k[0];
      const int64_t i0 = s_i[0];
      const auto sm = adam_span<3>(at, 0, k, i0, s_grad, ng, s_sc[0], s_sc[0]);
      const auto sl = adam_span<3>(at, 1, k, i0, s_grad + 3 * kGs, ng, s_sc[1], s_sc[1]);
      const auto sq = adam_span<4>(at, 2, k, i0, s_grad + 6 * kGs, ng, s_sc[2], s_sc[2]);
      const auto so = adam_span<1>(at, 3, k, i0, s_grad + 10 * kGs, ng, s_sc[3], s_sc[3]);
      const int t = threadIdx.x;
      {
        float p0[3], m0[3], v0[3], p1[3], m1[3], v1[3], p2[4], m2[4], v2[4], p3[1], m3[1], v3[1];
        span_load<3, 3>(sm, t, p0, m0, v0);
        span_load<3, 3>(sl, t, p1, m1, v1);
        span_load<4, 4>(sq, t, p2, m2, v2);
        span_load<1, 1>(so, t, p3, m3, v3);
        span_update<3, 3>(sm, t, p0, m0, v0, b1, b2, bci, eps);
        span_update<3, 3>(sl, t, p1, m1, v1, b1, b2, bci, eps);
        span_update<4, 4>(sq, t, p2, m2, v2, b1, b2, bci, eps);
        span_update<1, 1>(so, t, p3, m3, v3, b1, b2, bci, eps);
      }
      constexpr int kU = 16;
      const auto ss = adam_span<NC * 3>(at, 4, k, i0, s_grad + 11 * kGs, ng, s_sc[4], s_sc[5]);
      for (int base = t; base < ss.E; base += kU * kProjBwdThreads) {
        float pv[kU], mv[kU], vv[kU];
        span_load<NC * 3, kU>(ss, base, pv, mv, vv);
        span_update<NC * 3, kU>(ss, base, pv, mv, vv, b1, b2, bci, eps);
      }
    } else {
      adam_rows_split<3>(at, 0, s_grad, s_k, s_i, ng, s_sc[0], s_sc[0], b1, b2, bci, eps);
      adam_rows_split<3>(at, 1, s_grad + 3 * kGs, s_k, s_i, ng, s_sc[1], s_sc[1], b1, b2, bci,
                         eps);
      adam_rows_split<4>(at, 2, s_grad + 6 * kGs, s_k, s_i, ng, s_sc[2], s_sc[2], b1, b2, bci,
                         eps);
      adam_rows_split<1>(at, 3, s_grad + 10 * kGs, s_k, s_i, ng, s_sc[3], s_sc[3], b1, b2, bci,
                         eps);
      adam_rows_split<NC * 3>(at, 4, s_grad + 11 * kGs, s_k, s_i, ng, s_sc[4], s_sc[5], b1, b2,
                              bci, eps);
    }
  }
}

// Adam with a zero gradient over the 128-Gaussian blocks that the fused projection adjoint
// deferred (at.defer[blk] = 1): the same element function and bias-corrected rates, so the
// result is bit for bit that of the fused epilogue.  A grid-stride loop over blocks at full
// occupancy; each block's ranges are contiguous within its subset (element by element when
// it straddles two subsets).
template <int NC3>
__global__ void __launch_bounds__(256) k_adam_zero(const BatchDev b, const AdamTable at) {
  __shared__ float s_sc[7];
  adam_scales(at, s_sc);
  const float b1 = at.b1, b2 = at.b2, eps = at.eps, bci = s_sc[6];
  const int64_t nblk = (b.N + kProjBwdThreads - 1) / kProjBwdThreads;
  constexpr int W[5] = {3, 3, 4, 1, NC3};
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    if (!at.defer[blk]) continue;
    const int64_t g0 = blk * kProjBwdThreads;
    const int ng = b.N - g0 < kProjBwdThreads ? (int)(b.N - g0) : kProjBwdThreads;
    const int k0 = subset_of(b, g0), k1 = subset_of(b, g0 + ng - 1);
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      const int w = W[a];
      const float lo = s_sc[a < 4 ? a : 4], hi = s_sc[a < 4 ? a : 5];
      const int E = ng * w;
      if (k0 == k1) {
        const int64_t o = (g0 - b.goff[k0]) * w;
        float* pb = at.p[k0][a] + o;
        float* mb = at.m[k0][a] + o;
        float* vb = at.v[k0][a] + o;
        constexpr int kU = 4;
        for (int base = threadIdx.x; base < E; base += kU * 256) {
          float pv[kU], mv[kU], vv[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int idx = base + u * 256;
            if (idx < E) {
              pv[u] = pb[idx];
              mv[u] = mb[idx];
              vv[u] = vb[idx];
            }
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int idx = base + u * 256;
            if (idx < E) {
              const int e = idx % w;
              adam_elem(pv[u], 0.0f, mv[u], vv[u], e < 3 ? lo : hi, b1, b2, bci, eps);
              pb[idx] = pv[u];
              mb[idx] = mv[u];
              vb[idx] = vv[u];
            }
          }
        }
      } else {
        for (int idx = threadIdx.x; idx < E; idx += 256) {
          const int j = idx / w, e = idx - j * w;
          const int64_t g = g0 + j;
          const int k = subset_of(b, g);
          const int64_t off = (g - b.goff[k]) * w + e;
          float* pp = at.p[k][a] + off;
          float* mp = at.m[k][a] + off;
          float* vp = at.v[k][a] + off;
          float pv = *pp, mv = *mp, vv = *vp;
          adam_elem(pv, 0.0f, mv, vv, e < 3 ? lo : hi, b1, b2, bci, eps);
          *pp = pv;
          *mp = mv;
          *vp = vv;
        }
      }
    }
  }
}

// The zero-gradient pass over one parameter array of the whole batch when the subsets'
// arrays are consecutive slices of one allocation (p, m, v of n = N W floats): a flat
// grid-stride stream of four floats at a time over the deferred blocks only (a 128-Gaussian
// block is 32 W float4s, so no float4 straddles two blocks).  Same element function and
// rates as the fused epilogue.
template <int W>
__global__ void __launch_bounds__(256) k_adam_zero_flat(const AdamTable at, int a,
                                                        float* __restrict__ p,
                                                        float* __restrict__ m,
                                                        float* __restrict__ v, int64_t n) {
  __shared__ float s_sc[7];
  adam_scales(at, s_sc);
  const float b1 = at.b1, b2 = at.b2, eps = at.eps, bci = s_sc[6];
  const float lo = s_sc[a < 4 ? a : 4], hi = s_sc[a < 4 ? a : 5];
  const int64_t n4 = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
    if (!at.defer[q / (32 * W)]) continue;
    float4 p4 = reinterpret_cast<float4*>(p)[q];
    float4 m4 = reinterpret_cast<float4*>(m)[q];
    float4 v4 = reinterpret_cast<float4*>(v)[q];
    float* pe = &p4.x;
    float* me = &m4.x;
    float* ve = &v4.x;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int e = (int)((4 * q + c) % W);
      adam_elem(pe[c], 0.0f, me[c], ve[c], e < 3 ? lo : hi, b1, b2, bci, eps);
    }
    reinterpret_cast<float4*>(p)[q] = p4;
    reinterpret_cast<float4*>(m)[q] = m4;
    reinterpret_cast<float4*>(v)[q] = v4;
  }
  for (int64_t idx = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += stride) {
    if (!at.defer[idx / (128 * W)]) continue;
    float pv = p[idx], mv = m[idx], vv = v[idx];
    adam_elem(pv, 0.0f, mv, vv, idx % W < 3 ? lo : hi, b1, b2, bci, eps);
    p[idx] = pv;
    m[idx] = mv;
    v[idx] = vv;
  }
}

template <bool kFuse>
static void launch_project_bwd_t(const BatchDev& b, const GradTable& gt, const AdamTable& at,
                                 cudaStream_t s) {
  const int threads = kProjBwdThreads;
  const int64_t blocks = (b.N + threads - 1) / threads;
  if (blocks == 0) return;
  switch (b.sh_degree) {
    case 0: k_project_bwd<0, kFuse><<<(unsigned)blocks, threads, 0, s>>>(b, gt, at); break;
    case 1: k_project_bwd<1, kFuse><<<(unsigned)blocks, threads, 0, s>>>(b, gt, at); break;
    case 2: k_project_bwd<2, kFuse><<<(unsigned)blocks, threads, 0, s>>>(b, gt, at); break;
    default: k_project_bwd<3, kFuse><<<(unsigned)blocks, threads, 0, s>>>(b, gt, at); break;
  }
  count_launch();
}

void launch_project_bwd(const BatchDev& b, const GradTable& gt, cudaStream_t s) {
  AdamTable at;
  memset(&at, 0, sizeof(at));
  launch_project_bwd_t<false>(b, gt, at, s);
}

void launch_project_bwd_adam(const BatchDev& b, const AdamTable& at, cudaStream_t s) {
  GradTable gt;
  memset(&gt, 0, sizeof(gt));
  if (at.step_dev) launch_step_increment(const_cast<int64_t*>(at.step_dev), s);
  launch_project_bwd_t<true>(b, gt, at, s);
  if (!at.defer || b.N == 0) return;
  // one allocation per array (each subset's slice right after the previous one, 16-byte
  // aligned): a flat stream per array, one wave of resident CTAs
  const int width[5] = {3, 3, 4, 1, 3 * n_sh(b.sh_degree)};
  bool flat = true;
  for (int a = 0; a < 5 && flat; ++a)
    for (int t = 0; t < 3 && flat; ++t) {
      float* const* base = t == 0 ? at.p[0] : t == 1 ? at.m[0] : at.v[0];
      if ((reinterpret_cast<uintptr_t>(base[a]) & 15) != 0) flat = false;
      for (int k = 1; k < b.K && flat; ++k) {
        if (b.goff[k + 1] == b.goff[k]) continue;  // an empty subset has no arrays
        float* const* tk = t == 0 ? at.p[k] : t == 1 ? at.m[k] : at.v[k];
        if (tk[a] != base[a] + b.goff[k] * width[a]) flat = false;
      }
    }
  if (flat) {
    for (int a = 0; a < 5; ++a) {
      const int64_t n = b.N * width[a];
      auto go = [&](auto kernel, int slot) {
        int64_t blocks =
            (int64_t)device_sm_count() * resident_ctas((const void*)kernel, 256, 0, slot);
        const int64_t need = ((n >> 2) + 255) / 256;
        if (blocks > need) blocks = need > 0 ? need : 1;
        kernel<<<(unsigned)blocks, 256, 0, s>>>(at, a, at.p[0][a], at.m[0][a], at.v[0][a], n);
      };
      switch (width[a]) {  // (a cache slot of resident_ctas per kernel)
        case 3: go(k_adam_zero_flat<3>, 8); break;
        case 4: go(k_adam_zero_flat<4>, 9); break;
        case 1: go(k_adam_zero_flat<1>, 10); break;
        case 12: go(k_adam_zero_flat<12>, 11); break;
        case 27: go(k_adam_zero_flat<27>, 12); break;
        default: go(k_adam_zero_flat<48>, 13); break;
      }
      count_launch();
    }
    return;
  }
  const int64_t nblk = (b.N + kProjBwdThreads - 1) / kProjBwdThreads;
  int64_t blocks = (int64_t)device_sm_count() * 8;  // one wave of 256-thread CTAs
  if (blocks > nblk) blocks = nblk;
  switch (b.sh_degree) {
    case 0: k_adam_zero<3><<<(unsigned)blocks, 256, 0, s>>>(b, at); break;
    case 1: k_adam_zero<12><<<(unsigned)blocks, 256, 0, s>>>(b, at); break;
    case 2: k_adam_zero<27><<<(unsigned)blocks, 256, 0, s>>>(b, at); break;
    default: k_adam_zero<48><<<(unsigned)blocks, 256, 0, s>>>(b, at); break;
  }
  count_launch();
}

// ---------------------------------------------------------------- Adam
// torch.optim.Adam semantics: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= (lr / bc1) * m / (sqrt(v) / sqrt(bc2) + eps), bc_i = 1 - b_i^step.  sh_stride > 0
// selects lr_rest for elements whose index modulo sh_stride is >= 3 (SH coefficients
// above degree 0).  With zero_grad the gradient is cleared after it is read.
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, float* __restrict__ g,
                                              float* __restrict__ m, float* __restrict__ v, int64_t n,
                                              int64_t sh_stride, float lr_in, float lr_rest_in,
                                              float b1, float b2, float eps, int64_t step_host,
                                              const int64_t* __restrict__ step_dev, bool zero_grad,
                                              bool vec4) {
  // bias corrections in double precision, once per CTA (FP64 is slow on this part)
  __shared__ float s_sc[3];
  if (threadIdx.x == 0) {
    const int64_t step = step_dev ? *step_dev : step_host;
    const double bc1 = 1.0 - pow((double)b1, (double)step);
    const double bc2 = 1.0 - pow((double)b2, (double)step);
    s_sc[0] = (float)(lr_in / bc1);
    s_sc[1] = (float)(lr_rest_in / bc1);
    s_sc[2] = (float)(1.0 / sqrt(bc2));
  }
  __syncthreads();
  const float step_lr = s_sc[0], step_lr_rest = s_sc[1], bc2_sqrt_inv = s_sc[2];
  const int64_t n4 = vec4 ? (n >> 2) : 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // SH learning rates: element idx takes lr_rest when idx % sh_stride >= 3.  When
  // sh_stride is a multiple of 4 the float4 q starts at (q % (sh_stride / 4)) * 4 within
  // its Gaussian, kept incrementally (no division per element)
  const bool sh4 = sh_stride > 0 && (sh_stride & 3) == 0;
  const int64_t m4 = sh4 ? (sh_stride >> 2) : 1;
  const int64_t q0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t rem = q0 % m4;
  const int64_t rem_step = stride % m4;
  for (int64_t q = q0; q < n4; q += stride) {
    float4 pp = reinterpret_cast<float4*>(p)[q];
    const float4 gg = reinterpret_cast<const float4*>(g)[q];
    float4 mm = reinterpret_cast<float4*>(m)[q];
    float4 vv = reinterpret_cast<float4*>(v)[q];
    float* pe = &pp.x;
    const float* ge = &gg.x;
    float* me = &mm.x;
    float* ve = &vv.x;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float lr = step_lr;
      if (sh4) {
        if (rem != 0 || e >= 3) lr = step_lr_rest;
      } else if (sh_stride > 0 && ((4 * q + e) % sh_stride) >= 3) {
        lr = step_lr_rest;
      }
      adam_elem(pe[e], ge[e], me[e], ve[e], lr, b1, b2, bc2_sqrt_inv, eps);
    }
    reinterpret_cast<float4*>(p)[q] = pp;
    reinterpret_cast<float4*>(m)[q] = mm;
    reinterpret_cast<float4*>(v)[q] = vv;
    if (zero_grad) reinterpret_cast<float4*>(g)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    rem += rem_step;
    if (rem >= m4) rem -= m4;
  }
  for (int64_t idx = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
    const float lr = (sh_stride > 0 && (idx % sh_stride) >= 3) ? step_lr_rest : step_lr;
    float pp = p[idx], mm = m[idx], vv = v[idx];
    adam_elem(pp, g[idx], mm, vv, lr, b1, b2, bc2_sqrt_inv, eps);
    p[idx] = pp;
    m[idx] = mm;
    v[idx] = vv;
    if (zero_grad) g[idx] = 0.0f;
  }
}

__global__ void k_step_increment(int64_t* step) { *step += 1; }

void launch_step_increment(int64_t* step_dev, cudaStream_t s) {
  k_step_increment<<<1, 1, 0, s>>>(step_dev);
  count_launch();
}

void launch_adam(float* p, float* g, float* m, float* v, int64_t n, int64_t sh_stride,
                 float lr, float lr_rest, float b1, float b2, float eps, int64_t step,
                 const int64_t* step_dev, bool zero_grad, bool vec4, cudaStream_t s) {
  if (n <= 0) return;
  int64_t blocks = ((n >> 2) + 255) / 256;
  if (blocks < 1) blocks = 1;
  const int64_t cap = (int64_t)device_sm_count() * 32;
  if (blocks > cap) blocks = cap;
  k_adam<<<(unsigned)blocks, 256, 0, s>>>(p, g, m, v, n, sh_stride, lr, lr_rest, b1, b2, eps, step,
                                          step_dev, zero_grad, vec4);
  count_launch();
}

}  // namespace splx
