// project.cu -- per-Gaussian activation + EWA projection (forward) and its
// adjoint, including the SE(3) pose gradient.
//
// Forward (Sec. 3.3: the projection f_i^proj of each Gaussian onto the image
// plane; the frustum cull of the candidate selection of Sec. 3.4 step 1):
// one thread per Gaussian, 56 B read, 56 B written.  Every operation follows
// the written operation order (plain IEEE mul/add/div/sqrt, no contraction),
// so that the rect, the depth key and the alpha inputs agree bit for bit with
// any implementation of the same order.
//
// Adjoint (map optimisation by differentiable rendering, Sec. 3.4 step 4;
// pose gradients for render-driven tracking and the relative transform of
// Sec. 3.5 step 3): one thread per Gaussian chains the screen-space gradients
// (du, dv, d conic, d opacity, d depth) back to mean, log-scale, quaternion and
// opacity logit, and the pose 6-vector is reduced per block before one atomic
// per component.
#include <algorithm>

#include "common.cuh"
#include "internal.cuh"

namespace splat {

struct ProjMath {
  float s[3], qn[4], qnorm;
  float R[9], M[9], Sig[9];
  float p[3];
  float J00, J02, J11, J12, tx, ty;
  bool clamp_x, clamp_y;
  float Tm[6];
  float ca, cb, cc, det;
  float u, v, lam, radius;
  int rect[4];
  int tiles;
  bool visible;
};

__device__ __forceinline__ void project_math(const float* __restrict__ mean,
                                             const float* __restrict__ log_scale,
                                             const float* __restrict__ quat, float logit,
                                             const float* W, const CamK& cam, ProjMath& m) {
  m.visible = false;
  m.tiles = 0;
  // camera transform and the near / distance culls first: a culled Gaussian
  // needs none of the activation below (the results are the same either way)
#pragma unroll
  for (int i = 0; i < 3; ++i)
    m.p[i] = ((W[4 * i] * mean[0] + W[4 * i + 1] * mean[1]) + W[4 * i + 2] * mean[2]) + W[4 * i + 3];
  if (!(m.p[2] > cam.znear)) return;
  if (cam.maxd2 > 0.f &&
      __fadd_rn(__fadd_rn(__fmul_rn(m.p[0], m.p[0]), __fmul_rn(m.p[1], m.p[1])), __fmul_rn(m.p[2], m.p[2])) >
          cam.maxd2)
    return;  // outside the selection distance
  for (int k = 0; k < 3; ++k) m.s[k] = exp_full(log_scale[k]);
  const float z = m.p[2];
  const float lim_x = kClip * ((float)cam.width / (2.0f * cam.fx));
  const float lim_y = kClip * ((float)cam.height / (2.0f * cam.fy));
  const float txz = m.p[0] / z;
  const float tyz = m.p[1] / z;
  m.clamp_x = !(txz >= -lim_x && txz <= lim_x);
  m.clamp_y = !(tyz >= -lim_y && tyz <= lim_y);
  m.tx = fminf(lim_x, fmaxf(-lim_x, txz)) * z;
  m.ty = fminf(lim_y, fmaxf(-lim_y, tyz)) * z;
  const float zz = z * z;
  m.J00 = cam.fx / z;
  m.J02 = -(cam.fx * m.tx) / zz;
  m.J11 = cam.fy / z;
  m.J12 = -(cam.fy * m.ty) / zz;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    m.Tm[j] = m.J00 * W[j] + m.J02 * W[8 + j];
    m.Tm[3 + j] = m.J11 * W[4 + j] + m.J12 * W[8 + j];
  }
  m.u = cam.fx * txz + cam.cx;
  m.v = cam.fy * tyz + cam.cy;
  {
    // Centre cull, conservative: the largest eigenvalue of the screen
    // covariance Tm Sigma Tm^T + 0.3 I is at most |Tm|_F^2 s_max^2 + 0.3, so
    // the 3-sigma radius is at most rb (0.1% and 2 px above, far beyond the
    // rounding of the exact radius); a centre more than rb outside the tile
    // grid gives an empty rect, exactly what the full computation below would
    // find.  The rest is skipped for such Gaussians.
    float f2 = 0.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) f2 += m.Tm[j] * m.Tm[j];
    const float smax = fmaxf(m.s[0], fmaxf(m.s[1], m.s[2]));
    const float rb = 3.0f * sqrtf((f2 * (smax * smax) + kLowPass) * 1.001f) + 2.0f;
    const float gxp = (float)(kTile * cam.tiles_x), gyp = (float)(kTile * cam.tiles_y);
    if (m.u + rb < 0.0f || m.u - rb >= gxp || m.v + rb < 0.0f || m.v - rb >= gyp) return;
  }
  const float4 q = *reinterpret_cast<const float4*>(quat);
  const float n2 = ((q.x * q.x + q.y * q.y) + q.z * q.z) + q.w * q.w;
  if (n2 == 0.0f) {
    m.qnorm = 0.0f;
    m.qn[0] = 1.0f; m.qn[1] = 0.0f; m.qn[2] = 0.0f; m.qn[3] = 0.0f;
  } else {
    m.qnorm = sqrtf(n2);
    m.qn[0] = q.x / m.qnorm; m.qn[1] = q.y / m.qnorm;
    m.qn[2] = q.z / m.qnorm; m.qn[3] = q.w / m.qnorm;
  }
  const float r = m.qn[0], a = m.qn[1], b = m.qn[2], c = m.qn[3];
  m.R[0] = 1.0f - 2.0f * (b * b + c * c);
  m.R[1] = 2.0f * (a * b - r * c);
  m.R[2] = 2.0f * (a * c + r * b);
  m.R[3] = 2.0f * (a * b + r * c);
  m.R[4] = 1.0f - 2.0f * (a * a + c * c);
  m.R[5] = 2.0f * (b * c - r * a);
  m.R[6] = 2.0f * (a * c - r * b);
  m.R[7] = 2.0f * (b * c + r * a);
  m.R[8] = 1.0f - 2.0f * (a * a + b * b);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) m.M[3 * i + j] = m.R[3 * i + j] * m.s[j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      m.Sig[3 * i + j] = (m.M[3 * i] * m.M[3 * j] + m.M[3 * i + 1] * m.M[3 * j + 1]) +
                         m.M[3 * i + 2] * m.M[3 * j + 2];
  float U[6];
#pragma unroll
  for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      U[3 * a2 + j] = (m.Tm[3 * a2] * m.Sig[j] + m.Tm[3 * a2 + 1] * m.Sig[3 + j]) +
                      m.Tm[3 * a2 + 2] * m.Sig[6 + j];
  const float s00 = (U[0] * m.Tm[0] + U[1] * m.Tm[1]) + U[2] * m.Tm[2];
  const float s01 = (U[0] * m.Tm[3] + U[1] * m.Tm[4]) + U[2] * m.Tm[5];
  const float s11 = (U[3] * m.Tm[3] + U[4] * m.Tm[4]) + U[5] * m.Tm[5];
  m.ca = s00 + kLowPass;
  m.cb = s01;
  m.cc = s11 + kLowPass;
  m.det = m.ca * m.cc - m.cb * m.cb;
  if (!(m.det > 0.0f)) return;
  const float mid = 0.5f * (m.ca + m.cc);
  const float disc = mid * mid - m.det;
  const float lmax = mid + sqrtf(fmaxf(disc, 0.0f));
  const float rr = ceilf(3.0f * sqrtf(lmax));
  m.radius = rr;
  const float gx = (float)cam.tiles_x, gy = (float)cam.tiles_y;
  m.rect[0] = (int)fminf(fmaxf(floorf((m.u - rr) / 16.0f), 0.0f), gx);
  m.rect[1] = (int)fminf(fmaxf(floorf((m.v - rr) / 16.0f), 0.0f), gy);
  m.rect[2] = (int)fminf(fmaxf(floorf((m.u + rr) / 16.0f) + 1.0f, 0.0f), gx);
  m.rect[3] = (int)fminf(fmaxf(floorf((m.v + rr) / 16.0f) + 1.0f, 0.0f), gy);
  m.tiles = (m.rect[2] - m.rect[0]) * (m.rect[3] - m.rect[1]);
  if (m.tiles == 0) return;
  m.lam = 1.0f / (1.0f + exp_full(-logit));
  m.visible = true;
}

// 8 resident CTAs of 256 threads (32 registers) per SM: a 300k-Gaussian
// launch (1172 CTAs) is one wave of the 152 SMs instead of 1.5 waves at 5.
__global__ void __launch_bounds__(256, 8) project_fwd_kernel(GaussiansK g, CamK cam, const float* __restrict__ w2c,
                                                             ProjectedK out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  float W[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) W[k] = __ldg(w2c + k);
  ProjMath m;
  project_math(g.mean + 3 * i, g.log_scale + 3 * i, g.quat + 4 * i, g.opacity_logit[i], W, cam, m);
  float4 xyzo = make_float4(0.f, 0.f, 0.f, 0.f), con = make_float4(0.f, 0.f, 0.f, 0.f);
  int4 rect = make_int4(0, 0, 0, 0);
  int radius = 0, tiles = 0;
  if (m.visible) {
    xyzo = make_float4(m.u, m.v, m.p[2], m.lam);
    con.x = m.cc / m.det;
    con.y = -m.cb / m.det;
    con.z = m.ca / m.det;
    // smallest exponent at which opacity * exp(power) can still reach 1/255
    con.w = (logf(kAlphaMin) - logf(m.lam)) - kPowerCutMargin;
    radius = (int)m.radius;
    rect = make_int4(m.rect[0], m.rect[1], m.rect[2], m.rect[3]);
    tiles = m.tiles;
  }
  reinterpret_cast<float4*>(out.xyzo)[i] = xyzo;
  reinterpret_cast<float4*>(out.conic)[i] = con;
  reinterpret_cast<int4*>(out.rect)[i] = rect;
  out.radius[i] = radius;
  out.tiles_touched[i] = tiles;
}

// ----------------------------------------------------------------------------
// Adjoint.
// ----------------------------------------------------------------------------
// The 14 parameter gradients of one Gaussian.
struct Grad14 {
  float mean[3], ls[3], q[4], logit, rgb[3];
};

// Adjoint of one Gaussian's projection (its screen-space gradients in g2):
// its parameter gradients in `o` (all 0 when the forward projection culled
// it) and its share of the pose gradient added to `pose`.
// Every caller passes a kept Gaussian (radius > 0), whose records are all
// read: they are requested together up front (the parameters into registers,
// the conic and the screen-space gradients into L1), so the adjoint waits for
// one round trip instead of one per early-return test of the projection.
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void project_adjoint_one(const GaussiansK& g, const CamK& cam, const float* W,
                                                    const float* __restrict__ conic, const float* __restrict__ g2,
                                                    int stride, int64_t i, Grad14& o, float (&pose)[6]) {
  float mean[3], ls[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    mean[k] = g.mean[3 * i + k];
    ls[k] = g.log_scale[3 * i + k];
  }
  const float4 quat = reinterpret_cast<const float4*>(g.quat)[i];
  const float logit = g.opacity_logit[i];
  prefetch_l1(conic + 4 * i);
  prefetch_l1(g2 + (size_t)stride * i);
  prefetch_l1(g2 + (size_t)stride * i + 9);
  ProjMath m;
  project_math(mean, ls, &quat.x, logit, W, cam, m);
#pragma unroll
  for (int k = 0; k < 3; ++k) o.mean[k] = o.ls[k] = o.rgb[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.q[k] = 0.f;
  o.logit = 0.f;
  if (m.visible) {
    const float* d = g2 + (size_t)stride * i;
    const float du = d[0], dv = d[1], dqa = d[2], dqb = d[3], dqc = d[4], dlam = d[5], dz = d[9];
    o.rgb[0] = d[6];
    o.rgb[1] = d[7];
    o.rgb[2] = d[8];
    o.logit = dlam * m.lam * (1.0f - m.lam);
    // conic Q = cov^-1 with cov = [[ca, cb], [cb, cc]]; the off-diagonal conic
    // entry is one scalar used twice, so the full-matrix gradient of Q is
    // [[dqa, dqb/2], [dqb/2, dqc]] and d cov = -Q dQ Q.
    const float4 Q = reinterpret_cast<const float4*>(conic)[i];
    const float qa = Q.x, qb = Q.y, qc = Q.z;
    const float h = 0.5f * dqb;
    const float t00 = qa * dqa + qb * h, t01 = qa * h + qb * dqc;
    const float t10 = qb * dqa + qc * h, t11 = qb * h + qc * dqc;
    const float g00 = -(t00 * qa + t01 * qb);
    const float g01 = -(t00 * qb + t01 * qc);
    const float g11 = -(t10 * qb + t11 * qc);
    // cov = Tm Sig Tm^T: dTm = 2 G Tm Sig, dSig = Tm^T G Tm  (G symmetric 2x2)
    float TS[6];
#pragma unroll
    for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        TS[3 * a2 + j] = m.Tm[3 * a2] * m.Sig[j] + m.Tm[3 * a2 + 1] * m.Sig[3 + j] + m.Tm[3 * a2 + 2] * m.Sig[6 + j];
    float dTm[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      dTm[j] = 2.0f * (g00 * TS[j] + g01 * TS[3 + j]);
      dTm[3 + j] = 2.0f * (g01 * TS[j] + g11 * TS[3 + j]);
    }
    float dSig[9];
#pragma unroll
    for (int a3 = 0; a3 < 3; ++a3)
#pragma unroll
      for (int b3 = 0; b3 < 3; ++b3) {
        const float x0 = m.Tm[a3], x1 = m.Tm[3 + a3];
        const float y0 = m.Tm[b3], y1 = m.Tm[3 + b3];
        dSig[3 * a3 + b3] = x0 * (g00 * y0 + g01 * y1) + x1 * (g01 * y0 + g11 * y1);
      }
    // Tm rows: (J00 W0 + J02 W2), (J11 W1 + J12 W2)
    const float dJ00 = dTm[0] * W[0] + dTm[1] * W[1] + dTm[2] * W[2];
    const float dJ02 = dTm[0] * W[8] + dTm[1] * W[9] + dTm[2] * W[10];
    const float dJ11 = dTm[3] * W[4] + dTm[4] * W[5] + dTm[5] * W[6];
    const float dJ12 = dTm[3] * W[8] + dTm[4] * W[9] + dTm[5] * W[10];
    // gradient of the rotation block through Tm: dW_ij = sum_a J_ai dTm_aj
    float dWr[9];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      dWr[j] = m.J00 * dTm[j];
      dWr[3 + j] = m.J11 * dTm[3 + j];
      dWr[6 + j] = m.J02 * dTm[j] + m.J12 * dTm[3 + j];
    }
    const float z = m.p[2];
    const float iz = 1.0f / z, iz2 = iz * iz, iz3 = iz2 * iz;
    float gz = -cam.fx * iz2 * dJ00 - cam.fy * iz2 * dJ11 + 2.0f * cam.fx * m.tx * iz3 * dJ02 +
               2.0f * cam.fy * m.ty * iz3 * dJ12;
    const float gtx = -cam.fx * iz2 * dJ02;
    const float gty = -cam.fy * iz2 * dJ12;
    float gp0 = 0.f, gp1 = 0.f;
    if (m.clamp_x) gz += gtx * (m.tx * iz); else gp0 += gtx;
    if (m.clamp_y) gz += gty * (m.ty * iz); else gp1 += gty;
    gp0 += du * cam.fx * iz;
    gp1 += dv * cam.fy * iz;
    gz -= (du * cam.fx * m.p[0] + dv * cam.fy * m.p[1]) * iz2;
    gz += dz;
    const float gp[3] = {gp0, gp1, gz};
#pragma unroll
    for (int j = 0; j < 3; ++j) o.mean[j] = W[j] * gp[0] + W[4 + j] * gp[1] + W[8 + j] * gp[2];
    // Sig = M M^T, M = R diag(s)
    float dM[9];
#pragma unroll
    for (int a3 = 0; a3 < 3; ++a3)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dM[3 * a3 + j] = 2.0f * (dSig[3 * a3] * m.M[j] + dSig[3 * a3 + 1] * m.M[3 + j] + dSig[3 * a3 + 2] * m.M[6 + j]);
    float dR[9];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float gs = dM[j] * m.R[j] + dM[3 + j] * m.R[3 + j] + dM[6 + j] * m.R[6 + j];
      o.ls[j] = gs * m.s[j];
      dR[j] = dM[j] * m.s[j];
      dR[3 + j] = dM[3 + j] * m.s[j];
      dR[6 + j] = dM[6 + j] * m.s[j];
    }
    if (m.qnorm > 0.0f) {
      const float r = m.qn[0], a = m.qn[1], b = m.qn[2], c = m.qn[3];
      float gq[4];
      gq[0] = 2.0f * (c * (dR[3] - dR[1]) + b * (dR[2] - dR[6]) + a * (dR[7] - dR[5]));
      gq[1] = 2.0f * (b * (dR[1] + dR[3]) + c * (dR[2] + dR[6]) + r * (dR[7] - dR[5])) - 4.0f * a * (dR[4] + dR[8]);
      gq[2] = 2.0f * (a * (dR[1] + dR[3]) + r * (dR[2] - dR[6]) + c * (dR[5] + dR[7])) - 4.0f * b * (dR[0] + dR[8]);
      gq[3] = 2.0f * (r * (dR[3] - dR[1]) + a * (dR[2] + dR[6]) + b * (dR[5] + dR[7])) - 4.0f * c * (dR[0] + dR[4]);
      const float dot = r * gq[0] + a * gq[1] + b * gq[2] + c * gq[3];
      const float inv = 1.0f / m.qnorm;
#pragma unroll
      for (int k = 0; k < 4; ++k) o.q[k] = (gq[k] - m.qn[k] * dot) * inv;
    }
    // pose: rho = dL/dp ; phi = p x dL/dp + vee(dW W^T)
    float A[9];
#pragma unroll
    for (int a3 = 0; a3 < 3; ++a3)
#pragma unroll
      for (int b3 = 0; b3 < 3; ++b3)
        A[3 * a3 + b3] = dWr[3 * a3] * W[4 * b3] + dWr[3 * a3 + 1] * W[4 * b3 + 1] + dWr[3 * a3 + 2] * W[4 * b3 + 2];
    pose[0] += gp[0];
    pose[1] += gp[1];
    pose[2] += gp[2];
    pose[3] += m.p[1] * gp[2] - m.p[2] * gp[1] + (A[7] - A[5]);
    pose[4] += m.p[2] * gp[0] - m.p[0] * gp[2] + (A[2] - A[6]);
    pose[5] += m.p[0] * gp[1] - m.p[1] * gp[0] + (A[3] - A[1]);
  }
}

// Accumulate one Gaussian's gradients into the gradient arrays (none when
// the arrays are null: the pose gradient alone is wanted).
__device__ __forceinline__ void add_grads(const GradK& out, int64_t i, const Grad14& o) {
  if (!out.mean) return;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    out.mean[3 * i + k] += o.mean[k];
    out.log_scale[3 * i + k] += o.ls[k];
    out.rgb[3 * i + k] += o.rgb[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) out.quat[4 * i + k] += o.q[k];
  out.opacity_logit[i] += o.logit;
}

// Gaussians the forward projection culled (radius 0) have no gradient.  Each
// warp scans its share of the map 32 at a time and queues the visible ones in
// shared memory; the adjoint runs whenever 32 are queued (and once more for
// the rest), so that no warp runs it for one or two visible lanes only.
constexpr int kPbThreads = 256;
constexpr int kPbWarps = kPbThreads / 32;
constexpr int kScanRuns = 8;  // runs of 32 radii a warp of the fused adjoint loads at once

__device__ __forceinline__ void adjoint_into(const GaussiansK& g, const CamK& cam, const float* W,
                                             const float* conic, const float* g2, int stride, const GradK& out,
                                             int64_t i, float (&pose)[6]) {
  Grad14 o;
  project_adjoint_one(g, cam, W, conic, g2, stride, i, o, pose);
  add_grads(out, i, o);
}

// Block reduction of the pose gradient (warp shuffles, then one warp) and
// one atomic per component.  Every thread of the block takes part.
__device__ __forceinline__ void add_pose(const float (&pose)[6], float* d_pose) {
  __shared__ float red[6][kPbWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float x = pose[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float x = lane < kPbWarps ? red[k][lane] : 0.0f;
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0 && x != 0.0f) atomicAdd(d_pose + k, x);
    }
  }
}

__global__ void __launch_bounds__(kPbThreads) project_bwd_kernel(GaussiansK g, CamK cam, const float* __restrict__ w2c,
                                                                 const float* __restrict__ conic,
                                                                 const int32_t* __restrict__ radius,
                                                                 const float* __restrict__ g2, int stride, GradK out,
                                                                 float* __restrict__ d_pose,
                                                                 float* __restrict__ d2d_out) {
  __shared__ int32_t queue[kPbWarps][64];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lower = (1u << lane) - 1u;
  float W[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) W[k] = __ldg(w2c + k);
  float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int qn = 0;  // warp-uniform
  const int64_t stride_all = (int64_t)gridDim.x * kPbThreads;
  for (int64_t base = ((int64_t)blockIdx.x * kPbWarps + warp) * 32; base < g.n; base += stride_all) {
    const int64_t i = base + lane;
    if (i < g.n && d2d_out) {
#pragma unroll
      for (int k = 0; k < 10; ++k) d2d_out[10 * i + k] = g2[(size_t)stride * i + k];
    }
    const bool vis = i < g.n && radius[i] != 0;
    const unsigned m = __ballot_sync(full, vis);
    if (vis) queue[warp][qn + __popc(m & lower)] = (int32_t)i;
    qn += __popc(m);
    __syncwarp();
    if (qn >= 32) {
      adjoint_into(g, cam, W, conic, g2, stride, out, queue[warp][lane], pose);
      __syncwarp();
      if (lane < qn - 32) queue[warp][lane] = queue[warp][32 + lane];
      __syncwarp();
      qn -= 32;
    }
  }
  if (lane < qn) adjoint_into(g, cam, W, conic, g2, stride, out, queue[warp][lane], pose);
  if (d_pose) add_pose(pose, d_pose);
}

// The fused projection adjoint + Adam step.  Blocks [0, n_kept_blocks) take
// the kept Gaussians: per warp, 32 consecutive Gaussians per pass; the kept
// ones (radius > 0) are queued and, 32 at a time, run the adjoint and then
// the Adam step of their 14 elements from the gradients in registers.  The
// other blocks take the culled Gaussians' zero-gradient step in element
// space (units of 4 consecutive elements of one parameter group; a unit whose
// moments are all +0 is left alone after reading them).  The two parts touch
// disjoint elements and run side by side in one launch.

template <int W>
struct GroupState {
  float p[W], m[W], v[W];
};

template <int W>
__device__ __forceinline__ void group_load(const AdamMapK& A, int grp, int64_t i, GroupState<W>& s) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const size_t at = (size_t)W * i + k;
    s.p[k] = A.p[grp][at];
    s.m[k] = A.m[grp][at];
    s.v[k] = A.v[grp][at];
  }
}

template <int W>
__device__ __forceinline__ void group_step_store(const AdamMapK& A, int grp, int64_t i, GroupState<W>& s,
                                                 const float* g, float ibc1, float ibc2) {
#pragma unroll
  for (int k = 0; k < W; ++k) adam_update(s.p[k], g[k], s.m[k], s.v[k], A.lr[grp], A.b1, A.b2, ibc1, ibc2, A.eps);
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const size_t at = (size_t)W * i + k;
    A.p[grp][at] = s.p[k];
    A.m[grp][at] = s.m[k];
    A.v[grp][at] = s.v[k];
  }
}

// The lines of a kept Gaussian's Adam moments (and of its colour, which the
// adjoint does not read) requested into L2 before its adjoint runs: its Adam
// step then finds them there instead of waiting on DRAM after the adjoint.
__device__ __forceinline__ void adam_prefetch(const AdamMapK& A, int64_t i) {
  constexpr int kW[5] = {3, 3, 4, 1, 3};
#pragma unroll
  for (int grp = 0; grp < 5; ++grp) {
    prefetch_l2(A.m[grp] + kW[grp] * i);
    prefetch_l2(A.v[grp] + kW[grp] * i);
  }
  prefetch_l2(A.p[4] + 3 * i);
}

// The Adam step of one kept Gaussian's 14 elements, group after group, each
// group's loads issued before the previous group's stores (the groups are
// distinct arrays, so the order is only a matter of latency).
__device__ __forceinline__ void adam_gaussian(const AdamMapK& A, int64_t i, const Grad14& o, float ibc1, float ibc2) {
  GroupState<3> s0, s1, s4;
  GroupState<4> s2;
  GroupState<1> s3;
  group_load<3>(A, 0, i, s0);
  group_load<3>(A, 1, i, s1);
  group_step_store<3>(A, 0, i, s0, o.mean, ibc1, ibc2);
  group_load<4>(A, 2, i, s2);
  group_step_store<3>(A, 1, i, s1, o.ls, ibc1, ibc2);
  group_load<1>(A, 3, i, s3);
  group_load<3>(A, 4, i, s4);
  group_step_store<4>(A, 2, i, s2, o.q, ibc1, ibc2);
  group_step_store<1>(A, 3, i, s3, &o.logit, ibc1, ibc2);
  group_step_store<3>(A, 4, i, s4, o.rgb, ibc1, ibc2);
  if (A.seen) {  // its moments are now nonzero (or may be): mark it once
    const uint32_t bit = 1u << (i & 31);
    if (!(A.seen[i >> 5] & bit)) atomicOr(&A.seen[i >> 5], bit);
  }
}

// With a seen bitmap: the zero-gradient step of culled Gaussian i (one thread
// per Gaussian, its 14 elements), taken only when its bit is set -- a clear
// bit promises zero moments, whose update is nothing -- so the culled part
// reads one bit per Gaussian that was never updated.
// The bits of kScanRuns strided Gaussians are loaded together; the Gaussians
// with a set bit are then taken one at a time.
__device__ __forceinline__ void culled_seen(const AdamMapK& A, const int32_t* __restrict__ radius, int64_t n,
                                            int64_t first, int64_t stride, float ibc1, float ibc2) {
  for (int64_t i0 = first; i0 < n; i0 += kScanRuns * stride) {
    unsigned set = 0u;
#pragma unroll
    for (int r = 0; r < kScanRuns; ++r) {
      const int64_t i = i0 + r * stride;
      if (i < n && ((__ldg(A.seen + (i >> 5)) >> (i & 31)) & 1u)) set |= 1u << r;
    }
    for (; set; set &= set - 1u) {
      const int64_t i = i0 + (int64_t)(__ffs(set) - 1) * stride;
      if (__ldg(radius + i) != 0) continue;
      const int W[5] = {3, 3, 4, 1, 3};
#pragma unroll
      for (int grp = 0; grp < 5; ++grp) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (k >= W[grp]) break;
          const size_t e = (size_t)W[grp] * i + k;
          float pj = A.p[grp][e], mj = A.m[grp][e], vj = A.v[grp][e];
          adam_update(pj, 0.0f, mj, vj, A.lr[grp], A.b1, A.b2, ibc1, ibc2, A.eps);
          A.p[grp][e] = pj;
          A.m[grp][e] = mj;
          A.v[grp][e] = vj;
        }
      }
    }
  }
}

// Zero-gradient Adam step of the culled Gaussians' elements of group GRP
// (W elements per Gaussian), in units of 4 consecutive elements, grid-strided
// over the culled part's threads (a few units per thread, all moment loads
// first).
constexpr int kCulledUnroll = 4;

template <int W>
__device__ __forceinline__ void culled_group(const AdamMapK& A, int grp, const int32_t* __restrict__ radius, int64_t n,
                                             int64_t u_first, int64_t u_stride, float ibc1, float ibc2) {
  const int64_t size = (int64_t)W * n;
  const int64_t units = (size + 3) / 4;
  const bool vec = A.vec[grp] != 0;
  for (int64_t u0 = u_first; u0 < units; u0 += kCulledUnroll * u_stride) {
    float m4[kCulledUnroll][4], v4[kCulledUnroll][4];
#pragma unroll
    for (int r = 0; r < kCulledUnroll; ++r) {  // all moment loads first
      const int64_t e0 = 4 * (u0 + r * u_stride);
      if (vec && e0 + 4 <= size) {
        const float4 a = *reinterpret_cast<const float4*>(A.m[grp] + e0);
        const float4 b = *reinterpret_cast<const float4*>(A.v[grp] + e0);
        m4[r][0] = a.x; m4[r][1] = a.y; m4[r][2] = a.z; m4[r][3] = a.w;
        v4[r][0] = b.x; v4[r][1] = b.y; v4[r][2] = b.z; v4[r][3] = b.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool in = e0 + j < size;
          m4[r][j] = in ? A.m[grp][e0 + j] : 0.f;
          v4[r][j] = in ? A.v[grp][e0 + j] : 0.f;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kCulledUnroll; ++r) {
      uint32_t any = 0u;
#pragma unroll
      for (int j = 0; j < 4; ++j) any |= __float_as_uint(m4[r][j]) | __float_as_uint(v4[r][j]);
      if (any == 0u) continue;  // never seen since its moments were zero: nothing changes
      const int64_t e0 = 4 * (u0 + r * u_stride);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t e = e0 + j;
        if (e >= size || radius[e / W] != 0) continue;  // a kept Gaussian's element: the other part's
        float pj = A.p[grp][e], mj = m4[r][j], vj = v4[r][j];
        adam_update(pj, 0.0f, mj, vj, A.lr[grp], A.b1, A.b2, ibc1, ibc2, A.eps);
        A.p[grp][e] = pj;
        A.m[grp][e] = mj;
        A.v[grp][e] = vj;
      }
    }
  }
}

__device__ __forceinline__ void culled_units(const AdamMapK& A, const int32_t* __restrict__ radius, int64_t n,
                                             int64_t u_first, int64_t u_stride, float ibc1, float ibc2) {
  culled_group<3>(A, 0, radius, n, u_first, u_stride, ibc1, ibc2);
  culled_group<3>(A, 1, radius, n, u_first, u_stride, ibc1, ibc2);
  culled_group<4>(A, 2, radius, n, u_first, u_stride, ibc1, ibc2);
  culled_group<1>(A, 3, radius, n, u_first, u_stride, ibc1, ibc2);
  culled_group<3>(A, 4, radius, n, u_first, u_stride, ibc1, ibc2);
}

__global__ void __launch_bounds__(kPbThreads, 2) project_bwd_adam_kernel(GaussiansK g, CamK cam,
                                                                         const float* __restrict__ w2c,
                                                                         const float* __restrict__ conic,
                                                                         const int32_t* __restrict__ radius,
                                                                         const float* __restrict__ g2, int stride,
                                                                         AdamMapK A, float* __restrict__ d_pose,
                                                                         PoseAdamK P, int kept_blocks) {
  const float ibc1 = 1.0f / bias_correction(A.b1, A.step);
  const float ibc2 = 1.0f / bias_correction(A.b2, A.step);
  if ((int)blockIdx.x >= kept_blocks) {  // the culled Gaussians
    const int64_t nb = (int64_t)gridDim.x - kept_blocks;
    const int64_t first = ((int64_t)blockIdx.x - kept_blocks) * kPbThreads + threadIdx.x;
    if (A.seen)
      culled_seen(A, radius, g.n, first, nb * kPbThreads, ibc1, ibc2);
    else
      culled_units(A, radius, g.n, first, nb * kPbThreads, ibc1, ibc2);
    return;
  }
  __shared__ int32_t queue[kPbWarps][32 * kScanRuns + 32];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lower = (1u << lane) - 1u;
  float W[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) W[k] = w2c[k];  // plain loads: the last CTA may update w2c
  float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int qn = 0;  // warp-uniform
  // each warp scans runs of 32 consecutive radii, the runs of all warps
  // interleaved over the map, queueing the kept Gaussians: the kept ones
  // cluster in index order (a map is built surface by surface), and short
  // interleaved runs spread each cluster over all warps.  The radii of
  // kScanRuns runs are loaded together, then queued, then the queue is worked
  // off 32 at a time (the rest carried to the next group of runs).
  const int64_t stride_all = (int64_t)kept_blocks * kPbThreads;
  for (int64_t base = ((int64_t)blockIdx.x * kPbWarps + warp) * 32; base < g.n; base += kScanRuns * stride_all) {
    int32_t rr[kScanRuns];
#pragma unroll
    for (int r = 0; r < kScanRuns; ++r) {
      const int64_t i = base + r * stride_all + lane;
      rr[r] = i < g.n ? __ldg(radius + i) : 0;
    }
#pragma unroll
    for (int r = 0; r < kScanRuns; ++r) {
      const bool vis = rr[r] != 0;
      const unsigned m = __ballot_sync(full, vis);
      if (vis) queue[warp][qn + __popc(m & lower)] = (int32_t)(base + r * stride_all + lane);
      qn += __popc(m);
    }
    __syncwarp();
    const bool last = base + kScanRuns * stride_all >= g.n;  // warp-uniform
#pragma unroll 1
    for (int k0 = 0; k0 < qn && (last || k0 + 32 <= qn); k0 += 32) {
      const bool take = k0 + lane < qn;
      const int64_t j = take ? queue[warp][k0 + lane] : 0;
      if (take) {
        adam_prefetch(A, j);
        Grad14 o;
        project_adjoint_one(g, cam, W, conic, g2, stride, j, o, pose);
        adam_gaussian(A, j, o, ibc1, ibc2);
      }
    }
    if (!last) {  // carry the partial run of fewer than 32 to the front
      const int done = qn & ~31;
      __syncwarp();
      if (lane < qn - done) queue[warp][lane] = queue[warp][done + lane];
      qn -= done;
    }
    __syncwarp();
  }
  if (d_pose) add_pose(pose, d_pose);
  if (P.w2c) {  // the pose's Adam step, by the last kept CTA: every kept CTA has read w2c and added its gradient
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(P.counter, 1u) == (unsigned)kept_blocks - 1u;
    __syncthreads();
    if (s_last && warp == 0) {  // one warp, all loads issued together
      __threadfence();
      const float gk = lane < 6 ? __ldcg(d_pose + lane) : 0.0f;
      const float mk = lane < 6 ? P.m[lane] : 0.0f, vk = lane < 6 ? P.v[lane] : 0.0f;
      float Wp[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) Wp[k] = P.w2c[k];
      const float bc1 = bias_correction(P.b1, P.step), bc2 = bias_correction(P.b2, P.step);
      __syncwarp();  // every lane has read the pose before lanes 0-11 overwrite it
      pose_adam_warp(P.w2c, Wp, gk, mk, vk, P.m, P.v, P.lr_t, P.lr_r, P.b1, P.b2, bc1, bc2, P.eps);
      if (lane == 0) *P.counter = 0u;
    }
  }
}

int launch_project_fwd(const GaussiansK& g, const CamK& cam, const float* w2c, const ProjectedK& out,
                       cudaStream_t s) {
  if (g.n == 0) return SPLAT_OK;
  SPLAT_LAUNCH("project_fwd_kernel", s, project_fwd_kernel<<<ceil_div(g.n, 256), 256, 0, s>>>(g, cam, w2c, out));
  return check_launch("project_fwd_kernel");
}

// The culled Gaussians' zero-gradient step alone (its own launch).
__global__ void __launch_bounds__(kPbThreads) adam_culled_kernel(int64_t n, const int32_t* __restrict__ radius,
                                                                 AdamMapK A) {
  const float ibc1 = 1.0f / bias_correction(A.b1, A.step);
  const float ibc2 = 1.0f / bias_correction(A.b2, A.step);
  const int64_t first = (int64_t)blockIdx.x * kPbThreads + threadIdx.x, stride = (int64_t)gridDim.x * kPbThreads;
  if (A.seen)
    culled_seen(A, radius, n, first, stride, ibc1, ibc2);
  else
    culled_units(A, radius, n, first, stride, ibc1, ibc2);
}

int launch_adam_culled(int64_t n, const int32_t* radius, const AdamMapK& adam, cudaStream_t s) {
  if (n == 0) return SPLAT_OK;
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t units = (14 * n + 3) / 4;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(units, kPbThreads * kCulledUnroll), 4 * sms));
  SPLAT_LAUNCH("adam_culled_kernel", s, adam_culled_kernel<<<grid, kPbThreads, 0, s>>>(n, radius, adam));
  return check_launch("adam_culled_kernel");
}

int launch_project_bwd_adam(const GaussiansK& g, const CamK& cam, const float* w2c, const float* conic,
                            const int32_t* radius, const float* g2, int stride, const AdamMapK& adam, float* d_pose,
                            const PoseAdamK& pose, bool culled, cudaStream_t s) {
  if (g.n == 0) return SPLAT_OK;
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // both parts resident at once (two CTAs per SM): one for the kept Gaussians' adjoint, one for the culled
  const int kept_blocks = (int)std::min<int64_t>(ceil_div(g.n, kPbThreads), culled ? sms : 2 * sms);
  const int grid = kept_blocks + (culled ? sms : 0);
  SPLAT_LAUNCH("project_bwd_adam_kernel", s,
               project_bwd_adam_kernel<<<grid, kPbThreads, 0, s>>>(g, cam, w2c, conic, radius, g2, stride, adam,
                                                                   d_pose, pose, kept_blocks));
  return check_launch("project_bwd_adam_kernel");
}

int launch_project_bwd(const GaussiansK& g, const CamK& cam, const float* w2c, const float* conic,
                       const int32_t* radius, const float* g2, int stride, const GradK& out, float* d_pose,
                       float* d2d_out, cudaStream_t s) {
  if (g.n == 0) return SPLAT_OK;
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<int64_t>(ceil_div(g.n, kPbThreads), 2 * (int64_t)sms);
  SPLAT_LAUNCH("project_bwd_kernel", s,
               project_bwd_kernel<<<grid, kPbThreads, 0, s>>>(g, cam, w2c, conic, radius, g2, stride, out, d_pose,
                                                             d2d_out));
  return check_launch("project_bwd_kernel");
}

}  // namespace splat
