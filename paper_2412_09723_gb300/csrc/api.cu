// api.cu -- error plumbing, the projection entry point, and the small
// per-element kernels of the hot path: L1 loss (L1 terms of Eq. optim,
// Sec. 3.5), Adam on resident parameters (map optimisation, Sec. 3.4 step 4),
// the pose step (Adam + SE(3) retraction for render-driven tracking and the
// inter-agent relative transform) and the exponential.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "internal.cuh"

namespace splat {

static thread_local char g_last_error[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return code;
}

int check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SPLAT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return SPLAT_OK;
}

// ----------------------------------------------------------------------------
// L1 loss
// ----------------------------------------------------------------------------
__device__ __forceinline__ float l1_term(float x, float t, float sc, float& g) {
  const float e = x - t;
  g = e > 0.f ? sc : (e < 0.f ? -sc : 0.f);
  return fabsf(e);
}

// Four pixels per thread: with 16-byte aligned images, three float4 of colour
// and one of depth per image (a group of four pixels starts on a 48- / 16-byte
// boundary); the last npix % 4 pixels, or every pixel of unaligned images, one
// at a time.
__global__ void __launch_bounds__(256) loss_l1_kernel(const float* __restrict__ rgb, const float* __restrict__ depth,
                                                      const float* __restrict__ trgb, const float* __restrict__ tdepth,
                                                      int64_t npix, float sc, float sd, float* __restrict__ grgb,
                                                      float* __restrict__ gdepth, float* __restrict__ loss, bool vec) {
  float acc_c = 0.f, acc_d = 0.f;
  const int64_t n4 = vec ? npix / 4 : 0;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = tid; q < n4; q += nth) {
    const float4* x4 = reinterpret_cast<const float4*>(rgb) + 3 * q;
    const float4* t4 = reinterpret_cast<const float4*>(trgb) + 3 * q;
    float4* g4 = reinterpret_cast<float4*>(grgb) + 3 * q;
#pragma unroll
    for (int h = 0; h < 3; ++h) {
      const float4 x = x4[h], t = t4[h];
      float4 g;
      acc_c += l1_term(x.x, t.x, sc, g.x) + l1_term(x.y, t.y, sc, g.y) + l1_term(x.z, t.z, sc, g.z) +
               l1_term(x.w, t.w, sc, g.w);
      g4[h] = g;
    }
    const float4 d = reinterpret_cast<const float4*>(depth)[q], td = reinterpret_cast<const float4*>(tdepth)[q];
    float4 gd;
    acc_d += l1_term(d.x, td.x, sd, gd.x) + l1_term(d.y, td.y, sd, gd.y) + l1_term(d.z, td.z, sd, gd.z) +
             l1_term(d.w, td.w, sd, gd.w);
    reinterpret_cast<float4*>(gdepth)[q] = gd;
  }
  for (int64_t p = 4 * n4 + tid; p < npix; p += nth) {
#pragma unroll
    for (int k = 0; k < 3; ++k) acc_c += l1_term(rgb[3 * p + k], trgb[3 * p + k], sc, grgb[3 * p + k]);
    acc_d += l1_term(depth[p], tdepth[p], sd, gdepth[p]);
  }
  float acc = sc * acc_c + sd * acc_d;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (threadIdx.x == 0 && loss) atomicAdd(loss, x);
  }
}

int launch_loss_l1(const float* rgb, const float* depth, const float* trgb, const float* tdepth, int64_t npix,
                   float sc, float sd, float* grgb, float* gdepth, float* loss, cudaStream_t s) {
  if (npix == 0) return SPLAT_OK;
  const bool vec = aligned16(rgb) && aligned16(depth) && aligned16(trgb) && aligned16(tdepth) && aligned16(grgb) &&
                   aligned16(gdepth);
  const int grid = (int)std::min<int64_t>((npix / 4 + 255) / 256 + 1, 152 * 4);
  SPLAT_LAUNCH("loss_l1_kernel", s,
               loss_l1_kernel<<<grid, 256, 0, s>>>(rgb, depth, trgb, tdepth, npix, sc, sd, grgb, gdepth, loss, vec));
  return check_launch("loss_l1_kernel");
}

// ----------------------------------------------------------------------------
// Adam
// ----------------------------------------------------------------------------
// bias_correction and adam_update: internal.cuh.

__global__ void __launch_bounds__(256) adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                                                   float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                                                   float b1, float b2, const int32_t* __restrict__ step, float eps) {
  const float ibc1 = 1.0f / bias_correction(b1, step);
  const float ibc2 = 1.0f / bias_correction(b2, step);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float pi = p[i], mi = m[i], vi = v[i];
    adam_update(pi, g[i], mi, vi, lr, b1, b2, ibc1, ibc2, eps);
    m[i] = mi;
    v[i] = vi;
    p[i] = pi;
  }
}

struct AdamGroups {
  float* p[8];
  float* g[8];
  float* m[8];
  float* v[8];
  int64_t size[8];
  int64_t end[8];  // inclusive prefix of the group sizes in units of 4 elements
  float lr[8];
  int vec[8];      // all four arrays 16-byte aligned
  int n;
};

__device__ __forceinline__ void adam_one(float& p, float& g, float& m, float& v, float lr, float b1, float b2,
                                         float ibc1, float ibc2, float eps, int zero_grad) {
  adam_update(p, g, m, v, lr, b1, b2, ibc1, ibc2, eps);
  if (zero_grad) g = 0.0f;
}

// Grid-stride over the concatenation of the groups in units of 4 elements
// (float4 loads where the 4 elements lie inside one 16-byte-aligned group).
__global__ void __launch_bounds__(256) adam_groups_kernel(AdamGroups G, int64_t total4, float b1, float b2,
                                                          const int32_t* __restrict__ step, float eps, int zero_grad) {
  const float bc1 = 1.0f / bias_correction(b1, step);  // reciprocals
  const float bc2 = 1.0f / bias_correction(b2, step);
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < total4; u += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < G.n && u >= G.end[k]) ++k;
    const int64_t j = 4 * (u - (k ? G.end[k - 1] : 0));
    const int64_t size = G.size[k];
    float* P = G.p[k] + j;
    float* Gr = G.g[k] + j;
    float* M = G.m[k] + j;
    float* V = G.v[k] + j;
    const float lr = G.lr[k];
    if (j + 4 <= size && G.vec[k]) {
      float4 g4 = *reinterpret_cast<float4*>(Gr);
      float4 m4 = *reinterpret_cast<float4*>(M), v4 = *reinterpret_cast<float4*>(V);
      // Elements whose gradient and moments are all +0 (a Gaussian never seen
      // since its moments were last zero) have an update of exactly 0: m and v
      // stay +0, p - 0 = p; their parameters are neither read nor written.
      const uint32_t any_bits = __float_as_uint(g4.x) | __float_as_uint(g4.y) | __float_as_uint(g4.z) |
                                __float_as_uint(g4.w) | __float_as_uint(m4.x) | __float_as_uint(m4.y) |
                                __float_as_uint(m4.z) | __float_as_uint(m4.w) | __float_as_uint(v4.x) |
                                __float_as_uint(v4.y) | __float_as_uint(v4.z) | __float_as_uint(v4.w);
      if (any_bits == 0u) continue;
      float4 p4 = *reinterpret_cast<float4*>(P);
      adam_one(p4.x, g4.x, m4.x, v4.x, lr, b1, b2, bc1, bc2, eps, zero_grad);
      adam_one(p4.y, g4.y, m4.y, v4.y, lr, b1, b2, bc1, bc2, eps, zero_grad);
      adam_one(p4.z, g4.z, m4.z, v4.z, lr, b1, b2, bc1, bc2, eps, zero_grad);
      adam_one(p4.w, g4.w, m4.w, v4.w, lr, b1, b2, bc1, bc2, eps, zero_grad);
      *reinterpret_cast<float4*>(P) = p4;
      *reinterpret_cast<float4*>(M) = m4;
      *reinterpret_cast<float4*>(V) = v4;
      if (zero_grad) *reinterpret_cast<float4*>(Gr) = g4;
    } else {
      for (int e = 0; e < 4 && j + e < size; ++e)
        adam_one(P[e], Gr[e], M[e], V[e], lr, b1, b2, bc1, bc2, eps, zero_grad);
    }
  }
}

// Adam on the 6-vector pose gradient, then w2c <- exp(delta^) w2c.
__global__ void pose_step_kernel(float* __restrict__ w2c, const float* __restrict__ g, float* __restrict__ m,
                                 float* __restrict__ v, float lr_t, float lr_r, float b1, float b2,
                                 const int32_t* __restrict__ step, float eps) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  float W[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) W[k] = w2c[k];
  const float gk = lane < 6 ? g[lane] : 0.0f, mk = lane < 6 ? m[lane] : 0.0f, vk = lane < 6 ? v[lane] : 0.0f;
  const float bc1 = bias_correction(b1, step), bc2 = bias_correction(b2, step);
  __syncwarp();  // every lane has read the pose before lanes 0-11 overwrite it
  pose_adam_warp(w2c, W, gk, mk, vk, m, v, lr_t, lr_r, b1, b2, bc1, bc2, eps);
}

__global__ void pose_compose_kernel(int n, const float* __restrict__ a, const float* __restrict__ b,
                                    float* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float* A = a + 16 * k;
  float* O = out + 16 * k;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      O[4 * i + j] = A[4 * i] * b[j] + A[4 * i + 1] * b[4 + j] + A[4 * i + 2] * b[8 + j] + A[4 * i + 3] * b[12 + j];
}

__global__ void pose_rel_grad_kernel(int n, const float* __restrict__ w2c, const float* __restrict__ d_cam,
                                     float* __restrict__ d_rel) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < n; ++k) {
    const float* T = w2c + 16 * k;
    const float* g = d_cam + 6 * k;
    const float t0 = T[3], t1 = T[7], t2 = T[11];
    // h = g_phi - t x g_rho
    const float h0 = g[3] - (t1 * g[2] - t2 * g[1]);
    const float h1 = g[4] - (t2 * g[0] - t0 * g[2]);
    const float h2 = g[5] - (t0 * g[1] - t1 * g[0]);
    for (int j = 0; j < 3; ++j) {  // R^T v: column j of R dotted with v
      acc[j] += T[j] * g[0] + T[4 + j] * g[1] + T[8 + j] * g[2];
      acc[3 + j] += T[j] * h0 + T[4 + j] * h1 + T[8 + j] * h2;
    }
  }
  for (int j = 0; j < 6; ++j) d_rel[j] = acc[j];
}

__global__ void exp_kernel(const float* __restrict__ x, float* __restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = exp_full(x[i]);
}

}  // namespace splat

using namespace splat;

extern "C" int32_t splat_abi_version(void) { return 3; }

extern "C" const char* splat_last_error(void) { return g_last_error; }

extern "C" int splat_project(const splat_gaussians* g, const splat_camera* cam, const float* w2c,
                             const splat_projected* out, splat_stream_t stream) {
  if (!g || !cam || !w2c || !out) return fail(SPLAT_EINVAL, "splat_project: null argument");
  if (g->n < 0 || cam->width <= 0 || cam->height <= 0) return fail(SPLAT_EINVAL, "splat_project: bad sizes");
  if (g->n > 0 && (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !out->xyzo || !out->conic ||
                   !out->radius || !out->rect || !out->tiles_touched))
    return fail(SPLAT_EINVAL, "splat_project: null array");
  if (!aligned16(g->quat) || !aligned16(out->xyzo) || !aligned16(out->conic) || !aligned16(out->rect))
    return fail(SPLAT_EINVAL, "splat_project: quat/xyzo/conic/rect must be 16-byte aligned");
  GaussiansK gk{g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, g->n};
  ProjectedK pk{out->xyzo, out->conic, out->radius, out->rect, out->tiles_touched};
  return launch_project_fwd(gk, make_camk(*cam), w2c, pk, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int splat_loss_l1(const float* rgb, const float* depth, const float* target_rgb, const float* target_depth,
                             int64_t npix, float w_rgb, float w_depth, float* d_rgb, float* d_depth, float* loss,
                             splat_stream_t stream) {
  if (!rgb || !depth || !target_rgb || !target_depth || !d_rgb || !d_depth || npix < 0)
    return fail(SPLAT_EINVAL, "splat_loss_l1: bad argument");
  if (npix == 0) return SPLAT_OK;
  return launch_loss_l1(rgb, depth, target_rgb, target_depth, npix, w_rgb / (float)(3 * npix), w_depth / (float)npix,
                        d_rgb, d_depth, loss, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int splat_adam(float* param, const float* grad, float* m, float* v, int64_t n, const int32_t* step,
                          float lr, float beta1, float beta2, float eps, splat_stream_t stream) {
  if (!param || !grad || !m || !v || !step || n < 0) return fail(SPLAT_EINVAL, "splat_adam: bad argument");
  if (n == 0) return SPLAT_OK;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  SPLAT_LAUNCH("adam_kernel", reinterpret_cast<cudaStream_t>(stream), adam_kernel<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(param, grad, m, v, n, lr, beta1, beta2, step,
                                                                           eps));
  return check_launch("adam_kernel");
}

extern "C" int splat_adam_groups(int32_t n_groups, float* const* params, float* const* grads, float* const* m,
                                 float* const* v, const int64_t* sizes, const float* lr, const int32_t* step,
                                 float beta1, float beta2, float eps, int32_t zero_grad, splat_stream_t stream) {
  if (n_groups < 1 || n_groups > 8 || !params || !grads || !m || !v || !sizes || !lr || !step)
    return fail(SPLAT_EINVAL, "splat_adam_groups: bad argument");
  AdamGroups G;
  int64_t total4 = 0;
  for (int k = 0; k < n_groups; ++k) {
    if (sizes[k] < 0 || (sizes[k] > 0 && (!params[k] || !grads[k] || !m[k] || !v[k])))
      return fail(SPLAT_EINVAL, "splat_adam_groups: bad group %d", k);
    G.p[k] = params[k];
    G.g[k] = grads[k];
    G.m[k] = m[k];
    G.v[k] = v[k];
    G.lr[k] = lr[k];
    G.size[k] = sizes[k];
    G.vec[k] = aligned16(params[k]) && aligned16(grads[k]) && aligned16(m[k]) && aligned16(v[k]);
    total4 += (sizes[k] + 3) / 4;
    G.end[k] = total4;
  }
  G.n = n_groups;
  if (total4 == 0) return SPLAT_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one resident wave (6 CTAs of 256 threads per SM at this kernel's registers), grid-stride beyond
  const int blocks = (int)std::min<int64_t>((total4 + 255) / 256, 6 * (int64_t)sms);
  SPLAT_LAUNCH("adam_groups_kernel", s,
               adam_groups_kernel<<<blocks, 256, 0, s>>>(G, total4, beta1, beta2, step, eps, zero_grad));
  return check_launch("adam_groups_kernel");
}

extern "C" int splat_pose_step(float* w2c, const float* d_pose, float* m, float* v, const int32_t* step, float lr_t,
                               float lr_r, float beta1, float beta2, float eps, splat_stream_t stream) {
  if (!w2c || !d_pose || !m || !v || !step) return fail(SPLAT_EINVAL, "splat_pose_step: bad argument");
  SPLAT_LAUNCH("pose_step_kernel", reinterpret_cast<cudaStream_t>(stream), pose_step_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(w2c, d_pose, m, v, lr_t, lr_r, beta1, beta2,
                                                                          step, eps));
  return check_launch("pose_step_kernel");
}

extern "C" int splat_pose_compose(int32_t n, const float* a, const float* b, float* out, splat_stream_t stream) {
  if (n < 0 || (n > 0 && (!a || !b || !out))) return fail(SPLAT_EINVAL, "splat_pose_compose: bad argument");
  if (n == 0) return SPLAT_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SPLAT_LAUNCH("pose_compose_kernel", s, pose_compose_kernel<<<ceil_div(n, 64), 64, 0, s>>>(n, a, b, out));
  return check_launch("pose_compose_kernel");
}

extern "C" int splat_pose_rel_grad(int32_t n, const float* w2c, const float* d_cam, float* d_rel,
                                   splat_stream_t stream) {
  if (n < 0 || !d_rel || (n > 0 && (!w2c || !d_cam))) return fail(SPLAT_EINVAL, "splat_pose_rel_grad: bad argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SPLAT_LAUNCH("pose_rel_grad_kernel", s, pose_rel_grad_kernel<<<1, 32, 0, s>>>(n, w2c, d_cam, d_rel));
  return check_launch("pose_rel_grad_kernel");
}

extern "C" int splat_exp_f32(const float* x, float* y, int64_t n, splat_stream_t stream) {
  if (!x || !y || n < 0) return fail(SPLAT_EINVAL, "splat_exp_f32: bad argument");
  if (n == 0) return SPLAT_OK;
  SPLAT_LAUNCH("exp_kernel", reinterpret_cast<cudaStream_t>(stream), exp_kernel<<<ceil_div(n, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(x, y, n));
  return check_launch("exp_kernel");
}
