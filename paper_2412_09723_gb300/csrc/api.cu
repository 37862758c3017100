// api.cu -- error plumbing, the projection entry point, and the small
// per-element kernels of the hot path: L1 loss (L1 terms of Eq. optim,
// Sec. 3.5), Adam on resident parameters (map optimisation, Sec. 3.4 step 4),
// the pose step (Adam + SE(3) retraction for render-driven tracking and the
// inter-agent relative transform), render-based association (Sec. 3.5 step 2)
// and the exponential.
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
__global__ void __launch_bounds__(256) loss_l1_kernel(const float* __restrict__ rgb, const float* __restrict__ depth,
                                                      const float* __restrict__ trgb, const float* __restrict__ tdepth,
                                                      int64_t npix, float sc, float sd, float* __restrict__ grgb,
                                                      float* __restrict__ gdepth, float* __restrict__ loss) {
  float acc = 0.f;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
    float ac = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float e = rgb[3 * p + k] - trgb[3 * p + k];
      ac += fabsf(e);
      grgb[3 * p + k] = e > 0.f ? sc : (e < 0.f ? -sc : 0.f);
    }
    const float e = depth[p] - tdepth[p];
    gdepth[p] = e > 0.f ? sd : (e < 0.f ? -sd : 0.f);
    acc += sc * ac + sd * fabsf(e);
  }
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

// ----------------------------------------------------------------------------
// Adam
// ----------------------------------------------------------------------------
// 1 - beta^t in float, from a device-resident step count.
__device__ __forceinline__ float bias_correction(float beta, const int32_t* step) {
  return 1.0f - powf(beta, (float)(*step));
}

__global__ void __launch_bounds__(256) adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                                                   float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                                                   float b1, float b2, const int32_t* __restrict__ step, float eps) {
  const float bc1 = bias_correction(b1, step);
  const float bc2 = bias_correction(b2, step);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / bc1;
    const float vh = vi / bc2;
    p[i] = p[i] - lr * mh / (sqrtf(vh) + eps);
  }
}

// Adam on the 6-vector pose gradient, then w2c <- exp(delta^) w2c.
__global__ void pose_step_kernel(float* __restrict__ w2c, const float* __restrict__ g, float* __restrict__ m,
                                 float* __restrict__ v, float lr_t, float lr_r, float b1, float b2,
                                 const int32_t* __restrict__ step, float eps) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const float bc1 = bias_correction(b1, step);
  const float bc2 = bias_correction(b2, step);
  float d[6];
  for (int k = 0; k < 6; ++k) {
    const float mi = b1 * m[k] + (1.0f - b1) * g[k];
    const float vi = b2 * v[k] + (1.0f - b2) * g[k] * g[k];
    m[k] = mi;
    v[k] = vi;
    d[k] = -(k < 3 ? lr_t : lr_r) * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
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
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
  float R[9], V[9];
  for (int k = 0; k < 9; ++k) {
    const float I = (k % 4 == 0) ? 1.0f : 0.0f;
    R[k] = I + A * K[k] + Bc * K2[k];
    V[k] = I + Bc * K[k] + Cc * K2[k];
  }
  float t[3];
  for (int i = 0; i < 3; ++i) t[i] = V[3 * i] * d[0] + V[3 * i + 1] * d[1] + V[3 * i + 2] * d[2];
  float out[12];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 4; ++j)
      out[4 * i + j] = R[3 * i] * w2c[j] + R[3 * i + 1] * w2c[4 + j] + R[3 * i + 2] * w2c[8 + j];
    out[4 * i + 3] += t[i];
  }
  for (int k = 0; k < 12; ++k) w2c[k] = out[k];
}

// ----------------------------------------------------------------------------
// Association
// ----------------------------------------------------------------------------
__global__ void assoc_flag_kernel(const int32_t* __restrict__ ia, const float* __restrict__ ta,
                                  const int32_t* __restrict__ ib, const float* __restrict__ tb, int64_t npix,
                                  float tmax, uint32_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  flag[i] = (ia[i] >= 0 && ib[i] >= 0 && ta[i] <= tmax && tb[i] <= tmax) ? 1u : 0u;
}

__global__ void assoc_compact_kernel(const int32_t* __restrict__ ia, const int32_t* __restrict__ ib,
                                     const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                                     int64_t npix, int bits_b, uint64_t* __restrict__ keys,
                                     int64_t* __restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  if (flag[i]) keys[pos[i]] = ((uint64_t)(uint32_t)ia[i] << bits_b) | (uint64_t)(uint32_t)ib[i];
  if (i == npix - 1) *count = (int64_t)pos[i] + flag[i];
}

__global__ void assoc_head_kernel(const uint64_t* __restrict__ keys, const int64_t* __restrict__ count, int64_t npix,
                                  uint32_t* __restrict__ head) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  const int64_t c = *count;
  head[i] = (i < c && (i == 0 || keys[i] != keys[i - 1])) ? 1u : 0u;
}

__global__ void assoc_starts_kernel(const uint32_t* __restrict__ head, const uint32_t* __restrict__ uidx,
                                    const int64_t* __restrict__ count, int64_t npix, int64_t capacity,
                                    uint32_t* __restrict__ starts, int64_t* __restrict__ m_dev,
                                    int32_t* __restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  const int64_t c = *count;
  if (head[i]) starts[uidx[i]] = (uint32_t)i;
  if (i == npix - 1) {
    const int64_t m = (int64_t)uidx[i] + head[i];
    *m_dev = m;
    starts[m] = (uint32_t)c;
    if (m > capacity) raise_status(status, SPLAT_ECAPACITY);
  }
}

__global__ void assoc_write_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ starts,
                                   const int64_t* __restrict__ m_dev, int64_t capacity, int bits_b,
                                   int32_t* __restrict__ pairs, int32_t* __restrict__ counts) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t m = *m_dev;
  if (u >= m || u >= capacity) return;
  const uint64_t k = keys[starts[u]];
  pairs[2 * u] = (int32_t)(k >> bits_b);
  pairs[2 * u + 1] = (int32_t)(k & ((1ull << bits_b) - 1ull));
  counts[u] = (int32_t)(starts[u + 1] - starts[u]);
}

struct AssocWs {
  uint32_t *flag, *pos, *head, *uidx, *starts;
  uint64_t *k0, *k1;
  int64_t* count;
  void* scan;
  void* radix;
};

static size_t carve_assoc(int64_t npix, char* base, AssocWs* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  const size_t n = (size_t)(npix > 0 ? npix : 1);
  AssocWs t;
  t.flag = (uint32_t*)take(4 * n);
  t.pos = (uint32_t*)take(4 * n);
  t.head = (uint32_t*)take(4 * n);
  t.uidx = (uint32_t*)take(4 * n);
  t.starts = (uint32_t*)take(4 * (n + 1));
  t.k0 = (uint64_t*)take(8 * n);
  t.k1 = (uint64_t*)take(8 * n);
  t.count = (int64_t*)take(8);
  t.scan = take(scan_workspace_size((int64_t)n));
  t.radix = take(radix_workspace_size((int64_t)n));
  if (w) *w = t;
  return off;
}

static int bits_for(int64_t n) {
  int b = 1;
  while (b < 31 && ((int64_t)1 << b) < n) ++b;
  return b;
}

__global__ void exp_kernel(const float* __restrict__ x, float* __restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = exp_full(x[i]);
}

}  // namespace splat

using namespace splat;

extern "C" int32_t splat_abi_version(void) { return 1; }

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
  const float sc = w_rgb / (float)(3 * npix);
  const float sd = w_depth / (float)npix;
  const int blocks = (int)std::min<int64_t>((npix + 255) / 256, 152 * 8);
  SPLAT_LAUNCH("loss_l1_kernel", reinterpret_cast<cudaStream_t>(stream), loss_l1_kernel<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(rgb, depth, target_rgb, target_depth,
                                                                              npix, sc, sd, d_rgb, d_depth, loss));
  return check_launch("loss_l1_kernel");
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

extern "C" int splat_pose_step(float* w2c, const float* d_pose, float* m, float* v, const int32_t* step, float lr_t,
                               float lr_r, float beta1, float beta2, float eps, splat_stream_t stream) {
  if (!w2c || !d_pose || !m || !v || !step) return fail(SPLAT_EINVAL, "splat_pose_step: bad argument");
  SPLAT_LAUNCH("pose_step_kernel", reinterpret_cast<cudaStream_t>(stream), pose_step_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(w2c, d_pose, m, v, lr_t, lr_r, beta1, beta2,
                                                                          step, eps));
  return check_launch("pose_step_kernel");
}

extern "C" size_t splat_assoc_workspace_size(int64_t npix) { return npix < 0 ? 0 : carve_assoc(npix, nullptr, nullptr); }

extern "C" int splat_assoc(const int32_t* id_a, const float* t_a, const int32_t* id_b, const float* t_b, int64_t npix,
                           int64_t n_a, int64_t n_b, float t_max, int32_t* pairs, int32_t* counts, int64_t capacity,
                           int64_t* m_dev, int32_t* status, void* ws, size_t ws_bytes, splat_stream_t stream) {
  if (!id_a || !t_a || !id_b || !t_b || !m_dev || !status || !ws || npix < 0 || capacity < 0 || n_a < 1 || n_b < 1 ||
      n_a > 0x7fffffff || n_b > 0x7fffffff || npix > 0x7fffffff)
    return fail(SPLAT_EINVAL, "splat_assoc: bad argument");
  if (capacity > 0 && (!pairs || !counts)) return fail(SPLAT_EINVAL, "splat_assoc: null output");
  if (ws_bytes < carve_assoc(npix, nullptr, nullptr)) return fail(SPLAT_EINVAL, "splat_assoc: workspace too small");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (npix == 0) {
    if (cudaMemsetAsync(m_dev, 0, sizeof(int64_t), s) != cudaSuccess) return fail(SPLAT_ECUDA, "splat_assoc: memset");
    return SPLAT_OK;
  }
  AssocWs w;
  carve_assoc(npix, static_cast<char*>(ws), &w);
  const int ba = bits_for(n_a), bb = bits_for(n_b);
  const int nb = ceil_div(npix, 256);
  SPLAT_LAUNCH("assoc_flag_kernel", s, assoc_flag_kernel<<<nb, 256, 0, s>>>(id_a, t_a, id_b, t_b, npix, t_max, w.flag));
  int rc = exclusive_scan_u32(w.flag, w.pos, npix, w.scan, s);
  if (rc) return rc;
  SPLAT_LAUNCH("assoc_compact_kernel", s, assoc_compact_kernel<<<nb, 256, 0, s>>>(id_a, id_b, w.flag, w.pos, npix, bb, w.k0, w.count));
  if ((rc = check_launch("assoc_compact_kernel"))) return rc;
  int which = 0;
  if ((rc = radix_sort<uint64_t>(w.k0, nullptr, w.k1, nullptr, npix, w.count, 0, ba + bb, w.radix, s, &which)))
    return rc;
  const uint64_t* keys = which ? w.k1 : w.k0;
  SPLAT_LAUNCH("assoc_head_kernel", s, assoc_head_kernel<<<nb, 256, 0, s>>>(keys, w.count, npix, w.head));
  if ((rc = exclusive_scan_u32(w.head, w.uidx, npix, w.scan, s))) return rc;
  SPLAT_LAUNCH("assoc_starts_kernel", s, assoc_starts_kernel<<<nb, 256, 0, s>>>(w.head, w.uidx, w.count, npix, capacity, w.starts, m_dev, status));
  if ((rc = check_launch("assoc_starts_kernel"))) return rc;
  if (capacity == 0) return SPLAT_OK;
  SPLAT_LAUNCH("assoc_write_kernel", s, assoc_write_kernel<<<nb, 256, 0, s>>>(keys, w.starts, m_dev, capacity, bb, pairs, counts));
  return check_launch("assoc_write_kernel");
}

extern "C" int splat_exp_f32(const float* x, float* y, int64_t n, splat_stream_t stream) {
  if (!x || !y || n < 0) return fail(SPLAT_EINVAL, "splat_exp_f32: bad argument");
  if (n == 0) return SPLAT_OK;
  SPLAT_LAUNCH("exp_kernel", reinterpret_cast<cudaStream_t>(stream), exp_kernel<<<ceil_div(n, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(x, y, n));
  return check_launch("exp_kernel");
}
