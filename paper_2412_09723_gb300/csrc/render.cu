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
// Backward: same tiling; every thread starts from its pixel's final
// transmittance and last contributor, walks the list back to front, recovers
// T_i = T_{i+1} / (1 - alpha_i), and keeps the suffix sums
// R_X <- X_i alpha_i + (1 - alpha_i) R_X of colour, depth and silhouette so that
// dL/dalpha_i = T_i [gC.(c_i - R_C) + gD (z_i - R_D) + gS (1 - R_S)]
//             - (gC.bg) T_final / (1 - alpha_i).
// The 10 screen-space gradients of a Gaussian are summed over the 32 pixels of
// a warp with shuffles, over the warps of the CTA in shared memory, and added
// to global memory with one atomic per value per CTA.
#include <algorithm>

#include "common.cuh"
#include "internal.cuh"

namespace splat {

constexpr int kBatch = 256;

struct ImageK {
  float* rgb;
  float* depth;
  float* sil;
  float* t_final;
  int32_t* n_contrib;
  int32_t* max_id;
  int32_t* n_used;
};

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
  const uint2 rg = ranges[tile];
  float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, S = 0.f, wmax = 0.f;
  int32_t id = -1, last = 0, used = 0;
  bool done = !inside;
  for (uint32_t start = rg.x; start < rg.y; start += kBatch) {
    if (__syncthreads_count(done) == kTilePixels) break;
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
    if (!done) {
      for (int j = 0; j < cnt; ++j) {
        const float4 xo = s_xyzo[j];
        const float4 co = s_con[j];
        const float dx = xo.x - fx;
        const float dy = xo.y - fy;
        const float A = -0.5f * co.x;
        const float B = -co.y;
        const float Cc = -0.5f * co.z;
        const float power = __fmaf_rn(Cc * dy, dy, dx * __fmaf_rn(A, dx, B * dy));
        if (power > 0.0f || power < co.w) continue;
        const float G = exp_core(power);
        const float alpha = fminf(kAlphaCap, xo.w * G);
        if (alpha < kAlphaMin) continue;
        const float test_T = T * (1.0f - alpha);
        if (test_T < kTStop) {
          done = true;
          break;
        }
        const float w = alpha * T;
        C0 = __fmaf_rn(s_rgb[3 * j + 0], w, C0);
        C1 = __fmaf_rn(s_rgb[3 * j + 1], w, C1);
        C2 = __fmaf_rn(s_rgb[3 * j + 2], w, C2);
        D = __fmaf_rn(xo.z, w, D);
        S = S + w;
        if (w > wmax) {
          wmax = w;
          id = s_id[j];
        }
        T = test_T;
        last = (int32_t)(start - rg.x) + j + 1;
        ++used;
      }
    }
  }
  if (!inside) return;
  const size_t p = (size_t)py * cam.width + px;
  out.rgb[3 * p + 0] = __fmaf_rn(T, bg0, C0);
  out.rgb[3 * p + 1] = __fmaf_rn(T, bg1, C1);
  out.rgb[3 * p + 2] = __fmaf_rn(T, bg2, C2);
  out.depth[p] = D;
  out.sil[p] = S;
  out.t_final[p] = T;
  out.n_contrib[p] = last;
  out.max_id[p] = id;
  if (out.n_used) out.n_used[p] = used;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__global__ void __launch_bounds__(kTilePixels) render_bwd_kernel(
    const float4* __restrict__ xyzo, const float4* __restrict__ conic, const float* __restrict__ rgb,
    const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges, CamK cam, float bg0, float bg1, float bg2,
    const float* __restrict__ t_final, const int32_t* __restrict__ n_contrib, const float* __restrict__ d_rgb,
    const float* __restrict__ d_depth, const float* __restrict__ d_sil, float* __restrict__ d2d) {
  __shared__ float4 s_xyzo[kBatch];
  __shared__ float4 s_con[kBatch];
  __shared__ float s_rgb[3 * kBatch];
  __shared__ int32_t s_id[kBatch];
  __shared__ float s_grad[10][kBatch];
  __shared__ int s_maxlast;
  const int tile = blockIdx.x;
  const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x >> 4);
  const bool inside = px < cam.width && py < cam.height;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const uint2 rg = ranges[tile];
  const size_t p = inside ? (size_t)py * cam.width + px : 0;
  const float Tfin = inside ? t_final[p] : 1.0f;
  const int last = inside ? n_contrib[p] : 0;
  const float gC0 = inside ? d_rgb[3 * p + 0] : 0.f;
  const float gC1 = inside ? d_rgb[3 * p + 1] : 0.f;
  const float gC2 = inside ? d_rgb[3 * p + 2] : 0.f;
  const float gD = (inside && d_depth) ? d_depth[p] : 0.f;
  const float gS = (inside && d_sil) ? d_sil[p] : 0.f;
  const float gbg = gC0 * bg0 + gC1 * bg1 + gC2 * bg2;
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  if (last > 0) atomicMax(&s_maxlast, last);
  __syncthreads();
  const int maxlast = s_maxlast;
  float T = Tfin;
  float R0 = 0.f, R1 = 0.f, R2 = 0.f, RD = 0.f, RS = 0.f;
  const int lane = threadIdx.x & 31;
  for (int end = maxlast; end > 0; end -= kBatch) {
    const int start = max(0, end - kBatch);
    const int cnt = end - start;
    __syncthreads();
    if (threadIdx.x < cnt) {
      const uint32_t g = vals[rg.x + start + threadIdx.x];
      s_id[threadIdx.x] = (int32_t)g;
      s_xyzo[threadIdx.x] = xyzo[g];
      s_con[threadIdx.x] = conic[g];
      s_rgb[3 * threadIdx.x + 0] = rgb[3 * (size_t)g + 0];
      s_rgb[3 * threadIdx.x + 1] = rgb[3 * (size_t)g + 1];
      s_rgb[3 * threadIdx.x + 2] = rgb[3 * (size_t)g + 2];
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) s_grad[k][threadIdx.x] = 0.f;
    __syncthreads();
    for (int j = cnt - 1; j >= 0; --j) {
      float v[10];
#pragma unroll
      for (int k = 0; k < 10; ++k) v[k] = 0.f;
      bool act = start + j < last;
      if (act) {
        const float4 xo = s_xyzo[j];
        const float4 co = s_con[j];
        const float dx = xo.x - fx;
        const float dy = xo.y - fy;
        const float A = -0.5f * co.x;
        const float B = -co.y;
        const float Cc = -0.5f * co.z;
        const float power = __fmaf_rn(Cc * dy, dy, dx * __fmaf_rn(A, dx, B * dy));
        act = !(power > 0.0f || power < co.w);
        if (act) {
          const float G = exp_core(power);
          const float raw = xo.w * G;
          const float alpha = fminf(kAlphaCap, raw);
          act = !(alpha < kAlphaMin);
          if (act) {
            const float om = 1.0f - alpha;
            T = T / om;  // T_i
            const float w = alpha * T;
            const float c0 = s_rgb[3 * j + 0], c1 = s_rgb[3 * j + 1], c2 = s_rgb[3 * j + 2];
            v[6] = gC0 * w;
            v[7] = gC1 * w;
            v[8] = gC2 * w;
            v[9] = gD * w;
            float dA = (gC0 * (c0 - R0) + gC1 * (c1 - R1) + gC2 * (c2 - R2)) + gD * (xo.z - RD) + gS * (1.0f - RS);
            dA = dA * T - gbg * Tfin / om;
            R0 = c0 * alpha + om * R0;
            R1 = c1 * alpha + om * R1;
            R2 = c2 * alpha + om * R2;
            RD = xo.z * alpha + om * RD;
            RS = alpha + om * RS;
            if (!(raw > kAlphaCap)) {
              v[5] = G * dA;
              const float dp = raw * dA;
              v[0] = -dp * (co.x * dx + co.y * dy);
              v[1] = -dp * (co.y * dx + co.z * dy);
              v[2] = -0.5f * dp * dx * dx;
              v[3] = -dp * dx * dy;
              v[4] = -0.5f * dp * dy * dy;
            }
          }
        }
      }
      if (__any_sync(0xffffffffu, act)) {
#pragma unroll
        for (int k = 0; k < 10; ++k) v[k] = warp_sum(v[k]);
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < 10; ++k)
            if (v[k] != 0.f) atomicAdd(&s_grad[k][j], v[k]);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      float* dst = d2d + 10 * (size_t)s_id[threadIdx.x];
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        const float x = s_grad[k][threadIdx.x];
        if (x != 0.f) atomicAdd(dst + k, x);
      }
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
  return n < 0 ? 0 : align_up(sizeof(float) * 10 * (size_t)std::max<int64_t>(n, 1));
}

extern "C" int splat_render_bwd(const splat_gaussians* g, const splat_projected* proj, const splat_camera* cam,
                                const float* w2c, const uint32_t* vals, const uint32_t* ranges,
                                const splat_image* fwd, const float* bg, const float* d_rgb, const float* d_depth,
                                const float* d_sil, const splat_gaussians_grad* out, float* d_pose, float* d2d,
                                void* ws, size_t ws_bytes, splat_stream_t stream) {
  if (!g) return fail(SPLAT_EINVAL, "splat_render_bwd: null argument");
  int rc = check_proj(proj, g->n, "splat_render_bwd");
  if (rc) return rc;
  if (!g || !cam || !w2c || !vals || !ranges || !fwd || !fwd->t_final || !fwd->n_contrib || !bg || !d_rgb || !out ||
      (g->n > 0 && (!out->mean || !out->log_scale || !out->quat || !out->opacity_logit || !out->rgb)))
    return fail(SPLAT_EINVAL, "splat_render_bwd: null argument");
  if ((g->n > 0 && (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->rgb)) || !aligned16(g->quat))
    return fail(SPLAT_EINVAL, "splat_render_bwd: gaussian arrays null or quat not 16-byte aligned");
  if (g->n < 0 || cam->width <= 0 || cam->height <= 0) return fail(SPLAT_EINVAL, "splat_render_bwd: bad sizes");
  float* grad2d = d2d;
  if (!grad2d) {
    if (!ws || ws_bytes < splat_render_bwd_workspace_size(g->n))
      return fail(SPLAT_EINVAL, "splat_render_bwd: workspace too small");
    grad2d = static_cast<float*>(ws);
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (g->n > 0 && cudaMemsetAsync(grad2d, 0, sizeof(float) * 10 * (size_t)g->n, s) != cudaSuccess)
    return fail(SPLAT_ECUDA, "splat_render_bwd: memset failed");
  const CamK ck = make_camk(*cam);
  SPLAT_LAUNCH("render_bwd_kernel", s, render_bwd_kernel<<<ck.tiles_x * ck.tiles_y, kTilePixels, 0, s>>>(
      reinterpret_cast<const float4*>(proj->xyzo), reinterpret_cast<const float4*>(proj->conic), g->rgb, vals,
      reinterpret_cast<const uint2*>(ranges), ck, bg[0], bg[1], bg[2], fwd->t_final, fwd->n_contrib, d_rgb, d_depth,
      d_sil, grad2d));
  if ((rc = check_launch("render_bwd_kernel"))) return rc;
  GaussiansK gk{g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, g->n};
  GradK gr{out->mean, out->log_scale, out->quat, out->opacity_logit, out->rgb};
  return launch_project_bwd(gk, ck, w2c, proj->conic, grad2d, gr, d_pose, s);
}
