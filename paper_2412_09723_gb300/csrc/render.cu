// render.cu -- per-tile front-to-back compositing of colour, depth and
// silhouette (rendering equation of Sec. 3.3; rendered depth of Sec. 3.5) and
// its back-to-front adjoint.
//
// Forward: one CTA per 16x16 tile, one thread per pixel.  The tile's list is
// staged through shared memory in batches of 256 Gaussians (16 B position /
// depth / opacity, 16 B conic + exponent cut, 12 B colour, 4 B id each) and
// every thread walks the batch in order.  A pair whose exponent lies below the
// Gaussian's cut (precomputed by the projection so that opacity * exp(power) <
// 1/255 is certain) is skipped before the exponential is evaluated; this
// changes no result.  Blocks leave as soon as every pixel has reached the
// transmittance stop.  No atomics: the output is deterministic.
//
// Backward: same tiling, 128 threads with 2 pixels each ((x, y) and
// (x, y + 2); a warp covers 16 x 4 pixels).  Every pixel starts from its final
// transmittance and last contributor, walks the list back to front, recovers
// T_i = T_{i+1} / (1 - alpha_i), and keeps the suffix sums
// R_X <- X_i alpha_i + (1 - alpha_i) R_X of colour, depth and silhouette, so
// dL/dalpha_i = T_i [gC.(c_i - R_C) + gD (z_i - R_D) + gS (1 - R_S)]
//             - (gC.bg) T_final / (1 - alpha_i).
// Per Gaussian and warp, ten sums are reduced with a recursive-halving
// reduce-scatter (five moments of dL/dpower -- sum dp dx, dp dy, dp dx^2,
// dp dx dy, dp dy^2 -- whose conic terms are applied once per Gaussian, plus
// d opacity, d rgb, d depth), collected per CTA in shared memory and added to
// global memory with three float4 atomics per Gaussian per CTA.
#include <algorithm>

#include "common.cuh"
#include "internal.cuh"

namespace splat {

constexpr int kBatch = 256;
constexpr int kThreads = 128;  // backward: 2 pixels per thread, (x, y) and (x, y + 2)
constexpr int kGradStride = 12;  // internal screen-space gradient row (3 float4)
constexpr int kAccStride = 11;   // shared accumulator row (10 sums, padded against bank conflicts)

struct ImageK {
  float* rgb;
  float* depth;
  float* sil;
  float* t_final;
  int32_t* n_contrib;
  int32_t* max_id;
  int32_t* n_used;
};

// Pixel coordinates of thread t's two pixels: warp w covers rows 4w .. 4w+3.
__device__ __forceinline__ void pixel_of(int t, int p, int& lx, int& ly) {
  const int lane = t & 31, warp = t >> 5;
  lx = lane & 15;
  ly = 4 * warp + (lane >> 4) + 2 * p;
}

struct FwdPix {
  float T, C0, C1, C2, D, S, wmax;
  int32_t id, last, used;
  bool done;
};

// One front-to-back compositing step of one pixel (the specified order).
__device__ __forceinline__ void composite_step(FwdPix& q, const float4 xo, const float4 co, float fx, float fy,
                                               const float* c, int32_t gid, int32_t pos) {
  const float dx = xo.x - fx;
  const float dy = xo.y - fy;
  const float A = -0.5f * co.x;
  const float B = -co.y;
  const float Cc = -0.5f * co.z;
  const float power = __fmaf_rn(Cc * dy, dy, dx * __fmaf_rn(A, dx, B * dy));
  if (power > 0.0f || power < co.w) return;
  const float G = exp_core(power);
  const float alpha = fminf(kAlphaCap, xo.w * G);
  if (alpha < kAlphaMin) return;
  const float test_T = q.T * (1.0f - alpha);
  if (test_T < kTStop) {
    q.done = true;
    return;
  }
  const float w = alpha * q.T;
  q.C0 = __fmaf_rn(c[0], w, q.C0);
  q.C1 = __fmaf_rn(c[1], w, q.C1);
  q.C2 = __fmaf_rn(c[2], w, q.C2);
  q.D = __fmaf_rn(xo.z, w, q.D);
  q.S = q.S + w;
  if (w > q.wmax) {
    q.wmax = w;
    q.id = gid;
  }
  q.T = test_T;
  q.last = pos + 1;
  ++q.used;
}

__global__ void __launch_bounds__(kTilePixels) render_fwd_kernel(const float4* __restrict__ xyzo,
                                                                 const float4* __restrict__ conic,
                                                                 const float* __restrict__ rgb,
                                                                 const uint32_t* __restrict__ vals,
                                                                 const uint2* __restrict__ ranges, CamK cam,
                                                                 float bg0, float bg1, float bg2, ImageK out) {
  __shared__ float4 s_xyzo[kBatch];
  __shared__ float4 s_con[kBatch];
  __shared__ float s_rgb[3 * kBatch];
  __shared__ int32_t s_id[kBatch];
  const int tile = blockIdx.x;
  const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x >> 4);
  const bool inside = px < cam.width && py < cam.height;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  FwdPix q{1.0f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1, 0, 0, !inside};
  const uint2 rg = ranges[tile];
  for (uint32_t start = rg.x; start < rg.y; start += kBatch) {
    if (__syncthreads_count(q.done) == kTilePixels) break;
    const uint32_t idx = start + threadIdx.x;
    if (idx < rg.y) {
      const uint32_t g = vals[idx];
      s_id[threadIdx.x] = (int32_t)g;
      s_xyzo[threadIdx.x] = xyzo[g];
      s_con[threadIdx.x] = conic[g];
      s_rgb[3 * threadIdx.x + 0] = rgb[3 * (size_t)g + 0];
      s_rgb[3 * threadIdx.x + 1] = rgb[3 * (size_t)g + 1];
      s_rgb[3 * threadIdx.x + 2] = rgb[3 * (size_t)g + 2];
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kBatch, rg.y - start);
    const int32_t base = (int32_t)(start - rg.x);
    for (int j = 0; j < cnt && !q.done; ++j)
      composite_step(q, s_xyzo[j], s_con[j], fx, fy, &s_rgb[3 * j], s_id[j], base + j);
  }
  if (!inside) return;
  const size_t i = (size_t)py * cam.width + px;
  out.rgb[3 * i + 0] = __fmaf_rn(q.T, bg0, q.C0);
  out.rgb[3 * i + 1] = __fmaf_rn(q.T, bg1, q.C1);
  out.rgb[3 * i + 2] = __fmaf_rn(q.T, bg2, q.C2);
  out.depth[i] = q.D;
  out.sil[i] = q.S;
  out.t_final[i] = q.T;
  out.n_contrib[i] = q.last;
  out.max_id[i] = q.id;
  if (out.n_used) out.n_used[i] = q.used;
}

// ----------------------------------------------------------------------------
// Backward
// ----------------------------------------------------------------------------
// Sums v[0..9] over the 32 lanes of a warp by recursive halving: at each of
// the first four levels a lane keeps half of its values and sends the other
// half to its partner, so every lane ends up with one total.  Returns the
// index of the value whose warp total `out` holds, or -1 for lanes that hold
// a duplicate or a padding slot.
__device__ __forceinline__ int warp_reduce_scatter10(const float (&v)[10], float& out) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float w[6];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float send = b4 ? v[k] : v[5 + k];
    const float keep = b4 ? v[5 + k] : v[k];
    w[k] = keep + __shfl_xor_sync(full, send, 16);
  }
  w[5] = 0.f;
  float x[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float send = b3 ? w[k] : w[3 + k];
    const float keep = b3 ? w[3 + k] : w[k];
    x[k] = keep + __shfl_xor_sync(full, send, 8);
  }
  x[3] = 0.f;
  float y[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = b2 ? x[k] : x[2 + k];
    const float keep = b2 ? x[2 + k] : x[k];
    y[k] = keep + __shfl_xor_sync(full, send, 4);
  }
  float z = (b1 ? y[1] : y[0]) + __shfl_xor_sync(full, b1 ? y[0] : y[1], 2);
  z += __shfl_xor_sync(full, z, 1);
  out = z;
  const int i2 = (b2 ? 2 : 0) + (b1 ? 1 : 0);
  const int i1 = (b3 ? 3 : 0) + i2;
  return (!(lane & 1) && i2 < 3 && i1 < 5) ? (b4 ? 5 : 0) + i1 : -1;
}

struct BwdPix {
  float fx, fy, T, Tfin, gC0, gC1, gC2, gD, gS, gbgT, R0, R1, R2, RD, RS;
  int last;
};

// Per-pixel adjoint of one list position (back to front).  Accumulates the
// pixel's share of (sum dp dx, sum dp dy, sum dp dx^2, sum dp dx dy, sum dp
// dy^2, d opacity, d rgb[3], d depth) into v, dp = dL/d(power).
__device__ __forceinline__ bool adjoint_step(BwdPix& q, const float4 xo, const float4 co, float c0, float c1,
                                             float c2, float (&v)[10]) {
  const float dx = xo.x - q.fx;
  const float dy = xo.y - q.fy;
  const float A = -0.5f * co.x;
  const float B = -co.y;
  const float Cc = -0.5f * co.z;
  const float power = __fmaf_rn(Cc * dy, dy, dx * __fmaf_rn(A, dx, B * dy));
  if (power > 0.0f || power < co.w) return false;
  const float G = exp_core(power);
  const float raw = xo.w * G;
  const float alpha = fminf(kAlphaCap, raw);
  if (alpha < kAlphaMin) return false;
  const float om = 1.0f - alpha;
  const float r = __frcp_rn(om);
  q.T = q.T * r;  // T_i
  const float w = alpha * q.T;
  v[6] = __fmaf_rn(q.gC0, w, v[6]);
  v[7] = __fmaf_rn(q.gC1, w, v[7]);
  v[8] = __fmaf_rn(q.gC2, w, v[8]);
  v[9] = __fmaf_rn(q.gD, w, v[9]);
  float dA = q.gC0 * (c0 - q.R0);
  dA = __fmaf_rn(q.gC1, c1 - q.R1, dA);
  dA = __fmaf_rn(q.gC2, c2 - q.R2, dA);
  dA = __fmaf_rn(q.gD, xo.z - q.RD, dA);
  dA = __fmaf_rn(q.gS, 1.0f - q.RS, dA);
  dA = __fmaf_rn(dA, q.T, -q.gbgT * r);
  q.R0 = __fmaf_rn(c0, alpha, om * q.R0);
  q.R1 = __fmaf_rn(c1, alpha, om * q.R1);
  q.R2 = __fmaf_rn(c2, alpha, om * q.R2);
  q.RD = __fmaf_rn(xo.z, alpha, om * q.RD);
  q.RS = __fmaf_rn(1.0f, alpha, om * q.RS);
  if (!(raw > kAlphaCap)) {
    v[5] = __fmaf_rn(G, dA, v[5]);
    const float dp = raw * dA;
    const float m1 = dp * dx, m2 = dp * dy;
    v[0] += m1;
    v[1] += m2;
    v[2] = __fmaf_rn(m1, dx, v[2]);
    v[3] = __fmaf_rn(m1, dy, v[3]);
    v[4] = __fmaf_rn(m2, dy, v[4]);
  }
  return true;
}

__global__ void __launch_bounds__(kThreads) render_bwd_kernel(
    const float4* __restrict__ xyzo, const float4* __restrict__ conic, const float* __restrict__ rgb,
    const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges, CamK cam, float bg0, float bg1, float bg2,
    const float* __restrict__ t_final, const int32_t* __restrict__ n_contrib, const float* __restrict__ d_rgb,
    const float* __restrict__ d_depth, const float* __restrict__ d_sil, float* __restrict__ g2) {
  __shared__ float4 s_xyzo[kBatch];
  __shared__ float4 s_con[kBatch];
  __shared__ float s_rgb[3 * kBatch];
  __shared__ int32_t s_id[kBatch];
  __shared__ float s_acc[kBatch * kAccStride];
  __shared__ int s_maxlast;
  const int tile = blockIdx.x;
  const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
  const uint2 rg = ranges[tile];
  BwdPix q[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    int lx, ly;
    pixel_of(threadIdx.x, p, lx, ly);
    const int x = tx * kTile + lx, y = ty * kTile + ly;
    const bool inside = x < cam.width && y < cam.height;
    const size_t i = inside ? (size_t)y * cam.width + x : 0;
    BwdPix& b = q[p];
    b.fx = (float)x + 0.5f;
    b.fy = (float)y + 0.5f;
    b.Tfin = inside ? t_final[i] : 1.0f;
    b.T = b.Tfin;
    b.last = inside ? n_contrib[i] : 0;
    b.gC0 = inside ? d_rgb[3 * i + 0] : 0.f;
    b.gC1 = inside ? d_rgb[3 * i + 1] : 0.f;
    b.gC2 = inside ? d_rgb[3 * i + 2] : 0.f;
    b.gD = (inside && d_depth) ? d_depth[i] : 0.f;
    b.gS = (inside && d_sil) ? d_sil[i] : 0.f;
    b.gbgT = (b.gC0 * bg0 + b.gC1 * bg1 + b.gC2 * bg2) * b.Tfin;
    b.R0 = b.R1 = b.R2 = b.RD = b.RS = 0.f;
  }
  const int lane = threadIdx.x & 31;
  const int wlast = (int)__reduce_max_sync(0xffffffffu, (unsigned)max(q[0].last, q[1].last));
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  if (lane == 0 && wlast > 0) atomicMax(&s_maxlast, wlast);
  __syncthreads();
  const int maxlast = s_maxlast;
  for (int end = maxlast; end > 0; end -= kBatch) {
    const int start = max(0, end - kBatch);
    const int cnt = end - start;
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kThreads) {
      const uint32_t g = vals[rg.x + start + i];
      s_id[i] = (int32_t)g;
      s_xyzo[i] = xyzo[g];
      s_con[i] = conic[g];
      s_rgb[3 * i + 0] = rgb[3 * (size_t)g + 0];
      s_rgb[3 * i + 1] = rgb[3 * (size_t)g + 1];
      s_rgb[3 * i + 2] = rgb[3 * (size_t)g + 2];
    }
    for (int i = threadIdx.x; i < kBatch * kAccStride; i += kThreads) s_acc[i] = 0.f;
    __syncthreads();
    for (int j = cnt - 1; j >= 0; --j) {
      const int pos = start + j;
      if (pos >= wlast) continue;  // warp-uniform: no pixel of this warp reaches pos
      const float4 xo = s_xyzo[j];
      const float4 co = s_con[j];
      const float c0 = s_rgb[3 * j + 0], c1 = s_rgb[3 * j + 1], c2 = s_rgb[3 * j + 2];
      float v[10];
#pragma unroll
      for (int k = 0; k < 10; ++k) v[k] = 0.f;
      bool any = false;
#pragma unroll
      for (int p = 0; p < 2; ++p)
        if (pos < q[p].last) any |= adjoint_step(q[p], xo, co, c0, c1, c2, v);
      if (__any_sync(0xffffffffu, any)) {
        float tot;
        const int k = warp_reduce_scatter10(v, tot);
        if (k >= 0 && tot != 0.f) atomicAdd(&s_acc[j * kAccStride + k], tot);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kThreads) {
      const float* a = &s_acc[i * kAccStride];
      const float4 co = s_con[i];
      const float4 u0 = make_float4(-(co.x * a[0] + co.y * a[1]), -(co.y * a[0] + co.z * a[1]), -0.5f * a[2], -a[3]);
      const float4 u1 = make_float4(-0.5f * a[4], a[5], a[6], a[7]);
      const float4 u2 = make_float4(a[8], a[9], 0.f, 0.f);
      float4* dst = reinterpret_cast<float4*>(g2 + kGradStride * (size_t)s_id[i]);
      if (u0.x != 0.f || u0.y != 0.f || u0.z != 0.f || u0.w != 0.f) atomicAdd(dst, u0);
      if (u1.x != 0.f || u1.y != 0.f || u1.z != 0.f || u1.w != 0.f) atomicAdd(dst + 1, u1);
      if (u2.x != 0.f || u2.y != 0.f) atomicAdd(dst + 2, u2);
    }
  }
}

}  // namespace splat

using namespace splat;

static int check_proj(const splat_projected* proj, int64_t n, const char* who) {
  if (!proj || (n > 0 && (!proj->xyzo || !proj->conic)) || !aligned16(proj->xyzo) || !aligned16(proj->conic))
    return fail(SPLAT_EINVAL, "%s: projected arrays null or not 16-byte aligned", who);
  return SPLAT_OK;
}

extern "C" int splat_render_fwd(const splat_projected* proj, const float* rgb, int64_t n, const uint32_t* vals,
                                const uint32_t* ranges, const splat_camera* cam, const float* bg,
                                const splat_image* out, splat_stream_t stream) {
  int rc = check_proj(proj, n, "splat_render_fwd");
  if (rc) return rc;
  if ((n > 0 && !rgb) || !vals || !ranges || !cam || !bg || !out || !out->rgb || !out->depth || !out->sil || !out->t_final ||
      !out->n_contrib || !out->max_id)
    return fail(SPLAT_EINVAL, "splat_render_fwd: null argument");
  if (n < 0 || cam->width <= 0 || cam->height <= 0) return fail(SPLAT_EINVAL, "splat_render_fwd: bad sizes");
  const CamK ck = make_camk(*cam);
  ImageK im{out->rgb, out->depth, out->sil, out->t_final, out->n_contrib, out->max_id, out->n_used};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SPLAT_LAUNCH("render_fwd_kernel", s, render_fwd_kernel<<<ck.tiles_x * ck.tiles_y, kTilePixels, 0, s>>>(
      reinterpret_cast<const float4*>(proj->xyzo), reinterpret_cast<const float4*>(proj->conic), rgb, vals,
      reinterpret_cast<const uint2*>(ranges), ck, bg[0], bg[1], bg[2], im));
  return check_launch("render_fwd_kernel");
}

extern "C" size_t splat_render_bwd_workspace_size(int64_t n) {
  return n < 0 ? 0 : align_up(sizeof(float) * kGradStride * (size_t)std::max<int64_t>(n, 1));
}

extern "C" int splat_render_bwd(const splat_gaussians* g, const splat_projected* proj, const splat_camera* cam,
                                const float* w2c, const uint32_t* vals, const uint32_t* ranges,
                                const splat_image* fwd, const float* bg, const float* d_rgb, const float* d_depth,
                                const float* d_sil, const splat_gaussians_grad* out, float* d_pose, float* d2d,
                                void* ws, size_t ws_bytes, splat_stream_t stream) {
  if (!g) return fail(SPLAT_EINVAL, "splat_render_bwd: null argument");
  int rc = check_proj(proj, g->n, "splat_render_bwd");
  if (rc) return rc;
  if (!cam || !w2c || !vals || !ranges || !fwd || !fwd->t_final || !fwd->n_contrib || !bg || !d_rgb || !out ||
      (g->n > 0 && (!out->mean || !out->log_scale || !out->quat || !out->opacity_logit || !out->rgb)))
    return fail(SPLAT_EINVAL, "splat_render_bwd: null argument");
  if ((g->n > 0 && (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->rgb)) || !aligned16(g->quat))
    return fail(SPLAT_EINVAL, "splat_render_bwd: gaussian arrays null or quat not 16-byte aligned");
  if (g->n < 0 || cam->width <= 0 || cam->height <= 0) return fail(SPLAT_EINVAL, "splat_render_bwd: bad sizes");
  if (!ws || !aligned16(ws) || ws_bytes < splat_render_bwd_workspace_size(g->n))
    return fail(SPLAT_EINVAL, "splat_render_bwd: workspace missing, too small or not 16-byte aligned");
  float* g2 = static_cast<float*>(ws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (g->n > 0 && cudaMemsetAsync(g2, 0, sizeof(float) * kGradStride * (size_t)g->n, s) != cudaSuccess)
    return fail(SPLAT_ECUDA, "splat_render_bwd: memset failed");
  const CamK ck = make_camk(*cam);
  SPLAT_LAUNCH("render_bwd_kernel", s, render_bwd_kernel<<<ck.tiles_x * ck.tiles_y, kThreads, 0, s>>>(
      reinterpret_cast<const float4*>(proj->xyzo), reinterpret_cast<const float4*>(proj->conic), g->rgb, vals,
      reinterpret_cast<const uint2*>(ranges), ck, bg[0], bg[1], bg[2], fwd->t_final, fwd->n_contrib, d_rgb, d_depth,
      d_sil, g2));
  if ((rc = check_launch("render_bwd_kernel"))) return rc;
  GaussiansK gk{g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, g->n};
  GradK gr{out->mean, out->log_scale, out->quat, out->opacity_logit, out->rgb};
  return launch_project_bwd(gk, ck, w2c, proj->conic, g2, kGradStride, gr, d_pose, d2d, s);
}
