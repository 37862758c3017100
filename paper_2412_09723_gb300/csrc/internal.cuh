// internal.cuh -- kernel-side views of the ABI structs and launcher
// declarations shared between the translation units of the library.
#pragma once

#include "common.cuh"

namespace splat {

struct CamK {
  int width, height, tiles_x, tiles_y;
  float fx, fy, cx, cy, znear;
  float maxd2;  // squared distance limit, 0 = none
};

struct GaussiansK {
  const float* mean;
  const float* log_scale;
  const float* quat;
  const float* opacity_logit;
  const float* rgb;
  int64_t n;
};

struct ProjectedK {
  float* xyzo;
  float* conic;
  int32_t* radius;
  int32_t* rect;
  int32_t* tiles_touched;
};

struct GradK {
  float* mean;
  float* log_scale;
  float* quat;
  float* opacity_logit;
  float* rgb;
};

// Adam (bias-corrected; one update of one element).  1 - beta^t in float from
// a device-resident step count; the bias corrections enter as reciprocals and
// the step's division is the fast one: the update differs from the textbook
// expression by a few ulp of the step, not of the parameter.  An element whose
// gradient and moments are all +0 is left exactly as it is (m, v stay +0,
// p - 0 = p), so skipping it changes nothing.
__device__ __forceinline__ float bias_correction(float beta, const int32_t* step) {
  return 1.0f - powf(beta, (float)(*step));
}

__device__ __forceinline__ void adam_update(float& p, float g, float& m, float& v, float lr, float b1, float b2,
                                            float ibc1, float ibc2, float eps) {
  m = b1 * m + (1.0f - b1) * g;
  v = b2 * v + (1.0f - b2) * g * g;
  p = p - __fdividef(lr * (m * ibc1), sqrtf(v * ibc2) + eps);
}

// Adam on the 6-vector pose gradient, then w2c <- exp(delta^) w2c, by one
// warp: lane k < 6 updates moment k and forms step k (gk, mk, vk: its
// gradient and moments, read by the caller; ignored in lanes >= 6); every
// lane then forms exp(delta^) from the six steps with the same operations,
// and lane i < 12 writes entry i (row-major) of the new w2c.  W: the current
// w2c in every lane; bc1, bc2: the bias corrections 1 - beta^t.  All reads
// precede the call, so the step costs one round of loads, not one per element.
__device__ __forceinline__ void pose_adam_warp(float* __restrict__ w2c, const float (&W)[12], float gk, float mk,
                                               float vk, float* __restrict__ m, float* __restrict__ v, float lr_t,
                                               float lr_r, float b1, float b2, float bc1, float bc2, float eps) {
  const int lane = threadIdx.x & 31;
  const float mi = b1 * mk + (1.0f - b1) * gk;
  const float vi = b2 * vk + (1.0f - b2) * gk * gk;
  if (lane < 6) {
    m[lane] = mi;
    v[lane] = vi;
  }
  const float dk = -(lane < 3 ? lr_t : lr_r) * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  float d[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) d[k] = __shfl_sync(0xffffffffu, dk, k);
  // exp of (rho, phi): R by Rodrigues, t = V rho
  const float px = d[3], py = d[4], pz = d[5];
  const float th2 = px * px + py * py + pz * pz;
  const float th = sqrtf(th2);
  float A, Bc, Cc;  // sin(th)/th, (1-cos)/th^2, (th - sin)/th^3
  if (th < 1e-4f) {
    A = 1.0f - th2 / 6.0f;
    Bc = 0.5f - th2 / 24.0f;
    Cc = 1.0f / 6.0f - th2 / 120.0f;
  } else {
    A = sinf(th) / th;
    Bc = (1.0f - cosf(th)) / th2;
    Cc = (th - sinf(th)) / (th2 * th);
  }
  const float K[9] = {0.f, -pz, py, pz, 0.f, -px, -py, px, 0.f};
  float K2[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
  float R[9], V[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float I = (k % 4 == 0) ? 1.0f : 0.0f;
    R[k] = I + A * K[k] + Bc * K2[k];
    V[k] = I + Bc * K[k] + Cc * K2[k];
  }
  float t[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) t[i] = V[3 * i] * d[0] + V[3 * i + 1] * d[1] + V[3 * i + 2] * d[2];
  float o = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float e = R[3 * i] * W[j] + R[3 * i + 1] * W[4 + j] + R[3 * i + 2] * W[8 + j];
      if (j == 3) e += t[i];
      o = lane == 4 * i + j ? e : o;
    }
  }
  if (lane < 12) w2c[lane] = o;
}

// The pose's Adam step taken by the last CTA of the fused projection adjoint
// (w2c null: none).
struct PoseAdamK {
  float* w2c;
  float* m;
  float* v;
  const int32_t* step;
  float lr_t, lr_r, b1, b2, eps;
  unsigned* counter;  // zero on entry, left zero
};

// The map's Adam state for the fused projection adjoint + update.
struct AdamMapK {
  float* p[5];  // parameters (mean, log_scale, quat, opacity_logit, rgb), updated in place
  float* m[5];
  float* v[5];
  float lr[5];
  int vec[5];   // p, m, v of the group 16-byte aligned
  float b1, b2, eps;
  const int32_t* step;
  uint32_t* seen;  // bit i: Gaussian i's moments may be nonzero (0 promises m = v = 0), or null
};

inline CamK make_camk(const splat_camera& c) {
  CamK k;
  k.width = c.width;
  k.height = c.height;
  k.tiles_x = (c.width + kTile - 1) / kTile;
  k.tiles_y = (c.height + kTile - 1) / kTile;
  k.fx = c.fx; k.fy = c.fy; k.cx = c.cx; k.cy = c.cy; k.znear = c.z_near;
  k.maxd2 = c.max_dist > 0.f ? c.max_dist * c.max_dist : 0.f;
  return k;
}

int launch_project_fwd(const GaussiansK& g, const CamK& cam, const float* w2c, const ProjectedK& out,
                       cudaStream_t s);
// g2: screen-space gradients, rows of `stride` floats (du, dv, d conic a, b, c,
// d opacity, d rgb[3], d depth, padding); d2d_out (optional): copy [n,10].
// radius: the forward projection's radii (0 = culled: no gradient, skipped).
int launch_project_bwd(const GaussiansK& g, const CamK& cam, const float* w2c, const float* conic,
                       const int32_t* radius, const float* g2, int stride, const GradK& out, float* d_pose,
                       float* d2d_out, cudaStream_t s);

// Projection adjoint with the map's Adam step in the same pass: every
// Gaussian's parameters move by Adam with the gradient the adjoint gives it
// (0 for a culled one); nothing is written to gradient arrays.
// culled: the same launch also takes the culled Gaussians' zero-gradient step
// (else launch_adam_culled does, e.g. on another stream).
int launch_project_bwd_adam(const GaussiansK& g, const CamK& cam, const float* w2c, const float* conic,
                            const int32_t* radius, const float* g2, int stride, const AdamMapK& adam, float* d_pose,
                            const PoseAdamK& pose, bool culled, cudaStream_t s);
int launch_adam_culled(int64_t n, const int32_t* radius, const AdamMapK& adam, cudaStream_t s);

// L1 terms: grgb = sc sign(rgb - trgb), gdepth = sd sign(depth - tdepth) (overwritten),
// loss += sc sum|rgb - trgb| + sd sum|depth - tdepth|.
int launch_loss_l1(const float* rgb, const float* depth, const float* trgb, const float* tdepth, int64_t npix,
                   float sc, float sd, float* grgb, float* gdepth, float* loss, cudaStream_t s);

}  // namespace splat
