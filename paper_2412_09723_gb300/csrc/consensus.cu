// consensus.cu -- the inter-agent consensus terms and map pruning.
//
// * Loss of Eq. (optim) (Sec. 3.5 step 4): L1 colour, SSIM and L1 depth
//   terms with their image gradients, in two passes (the L1 terms ride on
//   the first, which has each pixel's colours staged).  SSIM uses an 11 x 11 Gaussian window
//   (sigma 1.5) over a zero-padded image; a CTA computes 32 x 16 blocks of
//   all three channels: the 42 x 26 patch of both images is staged in shared
//   memory (the statistics kernel is persistent and stages its next block's
//   patch with asynchronous copies while it computes the current one), the
//   window is applied separably (rows, then columns) to the five
//   products x, y, x^2, y^2, xy, and each pixel's SSIM and its partial derivatives with
//   respect to the three window sums that involve x (A = dS/dmu_x,
//   B = dS/dE[x^2], C = dS/dE[xy]) are written out.  A second kernel applies
//   the same window to A, B, C and forms
//   dS/dx(q) = (W*A)(q) + 2 x(q) (W*B)(q) + y(q) (W*C)(q).
// * Mahalanobis alignment (Sec. 3.5 step 3): one thread per associated pair
//   gathers both Gaussians' records in one round and builds its Gauss-Newton
//   contribution (21 + 6 + 1 numbers) in float, summed in float per thread,
//   warp and CTA (a few pairs, 32 and 8 partial sums: double-precision
//   arithmetic is slow on this part), then into the system with one double
//   atomic per number and CTA; one thread solves the 6 x 6 system by
//   Cholesky (scaled to unit diagonal, in float) and retracts T.
// * Pruning (Algorithm 1): a flag kernel (the three criteria, block counts),
//   a one-CTA scan of the block counts, and a scatter kernel that re-ranks
//   the kept Gaussians inside each block and copies every column's row.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "common.cuh"
#include "internal.cuh"
#include "segsort.cuh"

namespace splat {

// ----------------------------------------------------------------------------
// SSIM
// ----------------------------------------------------------------------------
constexpr int kSsR = 5;                   // window radius
constexpr int kSsTaps = 2 * kSsR + 1;     // 11
constexpr float kSsC1 = 0.01f * 0.01f;
constexpr float kSsC2 = 0.03f * 0.03f;

struct SsimWin {
  float w[kSsTaps];  // 1-D Gaussian taps; the 2-D window is their outer product
};

static SsimWin ssim_window() {
  double g[kSsTaps], tot = 0.0;
  for (int i = 0; i < kSsTaps; ++i) {
    const double r = i - kSsR;
    g[i] = std::exp(-r * r / (2.0 * 1.5 * 1.5));
    tot += g[i];
  }
  SsimWin w;
  for (int i = 0; i < kSsTaps; ++i) w.w[i] = (float)(g[i] / tot);
  return w;
}

__device__ __forceinline__ float block_sum_256(float v, float* red /*[8]*/) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x < 32) {
    t = threadIdx.x < 8 ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// The window sums run in two separable passes over a patch staged in shared
// memory: a horizontal pass in which a thread takes a run of kSsRun outputs of
// one patch row (each staged pixel is read once per run and added, with each
// tap weight, into the outputs it reaches), and a vertical pass in which a
// thread takes two outputs of one column.  Pairs of sums that share a weight
// ((x, y), (x^2, y^2), (A, B)) are accumulated as packed single-precision
// pairs.  One CTA covers a kSsTX x kSsTY block of all three channels.
constexpr int kSsTX = 32, kSsTY = 16;     // output block
constexpr int kSsPX = kSsTX + 2 * kSsR;   // staged patch, 42 x 26
constexpr int kSsPY = kSsTY + 2 * kSsR;
constexpr int kSsRun = 4;                 // horizontal outputs per thread
constexpr int kSsHItems = kSsPY * (kSsTX / kSsRun);  // 208 horizontal runs per channel
// Padded shared rows: the 8 runs of a patch row and the 4 rows a warp spans
// fall in distinct banks (patch rows of 43 pairs, sum rows of 33).
constexpr int kSsPXp = kSsPX + 1;
constexpr int kSsTXp = kSsTX + 1;

__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

// Asynchronous 4-byte copies global -> shared (cp.async, zero-filled when
// `in` is false: the zero padding of the window), so that a CTA stages its
// next patch while it computes the current one.
__device__ __forceinline__ void cp_async4(void* smem, const float* g, bool in) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(g), "r"(in ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Persistent CTAs: CTA b takes blocks b, b + grid, ... of the kSsTX x kSsTY
// output grid (nbx blocks per row) and double-buffers their patches.
struct SsFwdSmem {
  float2 sxy[2][3][kSsPY][kSsPXp];  // (x, y) of every channel, two patches
  float2 h1[kSsPY][kSsTXp];         // horizontal sums of (x, y)
  float2 h2[kSsPY][kSsTXp];         // ... of (x^2, y^2)
  float h3[kSsPY][kSsTXp];          // ... of x y
  float red[8];
};

// The patch of block (bx, by): a patch row is 126 consecutive floats of each image.
__device__ __forceinline__ void ssim_fwd_stage(float2 (*dst)[kSsPY][kSsPXp], const float* x, const float* y, int H,
                                               int W, int bx, int by) {
  for (int e = threadIdx.x; e < kSsPY * 3 * kSsPX; e += blockDim.x) {
    const int r = e / (3 * kSsPX), j = e - r * (3 * kSsPX);
    const int c = j / 3, ch = j - 3 * c;
    const int gx = bx - kSsR + c, gy = by - kSsR + r;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    const size_t gi = in ? ((size_t)gy * W + gx) * 3 + ch : 0;
    float2* d = &dst[ch][r][c];
    cp_async4(&d->x, x + gi, in);
    cp_async4(&d->y, y + gi, in);
  }
}

// The L1 terms of the loss ride along: each output pixel's colour residual
// x - y (already staged) and depth residual give the L1 subgradients
// (written to d_rgb / d_depth; the adjoint kernel adds the SSIM part) and
// their share of the loss.
__global__ void __launch_bounds__(256) ssim_fwd_kernel(const float* __restrict__ x, const float* __restrict__ y,
                                                       const float* __restrict__ dep, const float* __restrict__ tdep,
                                                       int H, int W, int nbx, int nblk, SsimWin win, float loss_scale,
                                                       float ssim_scale, float sc, float sd, float* __restrict__ d_rgb,
                                                       float* __restrict__ d_depth, float* __restrict__ abc,
                                                       float* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char ss_raw[];
  SsFwdSmem& sm = *reinterpret_cast<SsFwdSmem*>(ss_raw);
  const int t = threadIdx.x;
  const size_t plane = (size_t)H * W;
  float sum_1ms = 0.f, sum_s = 0.f, sum_c = 0.f, sum_d = 0.f;
  int blk = blockIdx.x, buf = 0;
  if (blk < nblk) ssim_fwd_stage(sm.sxy[0], x, y, H, W, (blk % nbx) * kSsTX, (blk / nbx) * kSsTY);
  cp_async_commit();
  for (; blk < nblk; blk += gridDim.x, buf ^= 1) {
    const int nxt = blk + gridDim.x;
    if (nxt < nblk) ssim_fwd_stage(sm.sxy[buf ^ 1], x, y, H, W, (nxt % nbx) * kSsTX, (nxt / nbx) * kSsTY);
    cp_async_commit();
    cp_async_wait<1>();  // this block's patch has landed (the next one may still be in flight)
    __syncthreads();
    float2 (*sxy)[kSsPY][kSsPXp] = sm.sxy[buf];
    const int bx = (blk % nbx) * kSsTX, by = (blk / nbx) * kSsTY;
    // depths of this thread's two outputs, requested before the window passes
    float od[2], otd[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gx = bx + (t & 31), gy = by + 2 * (t >> 5) + j;
      const bool in = gx < W && gy < H;
      const size_t pix = in ? (size_t)gy * W + gx : 0;
      od[j] = in ? dep[pix] : 0.f;
      otd[j] = in ? tdep[pix] : 0.f;
    }
    for (int ch = 0; ch < 3; ++ch) {
      if (t < kSsHItems) {
        const int r = t / (kSsTX / kSsRun), c0 = kSsRun * (t % (kSsTX / kSsRun));
        float2 a1[kSsRun], a2[kSsRun];
        float a3[kSsRun];
#pragma unroll
        for (int j = 0; j < kSsRun; ++j) {
          a1[j] = a2[j] = bc2(-0.0f);
          a3[j] = -0.0f;
        }
#pragma unroll
        for (int p = 0; p < kSsRun + 2 * kSsR; ++p) {
          const float2 v = sxy[ch][r][c0 + p];
          const float2 sq = __fmul2_rn(v, v);
          const float pr = v.x * v.y;
#pragma unroll
          for (int j = 0; j < kSsRun; ++j) {
            const int k = p - j;
            if (k >= 0 && k < kSsTaps) {
              const float2 w = bc2(win.w[k]);
              a1[j] = __ffma2_rn(w, v, a1[j]);
              a2[j] = __ffma2_rn(w, sq, a2[j]);
              a3[j] = fmaf(win.w[k], pr, a3[j]);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < kSsRun; ++j) {
          sm.h1[r][c0 + j] = a1[j];
          sm.h2[r][c0 + j] = a2[j];
          sm.h3[r][c0 + j] = a3[j];
        }
      }
      __syncthreads();
      const int tx = t & 31, ty0 = 2 * (t >> 5);
      float2 m1[2], m2[2];
      float m3[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        m1[j] = m2[j] = bc2(-0.0f);
        m3[j] = -0.0f;
      }
#pragma unroll
      for (int p = 0; p < 2 + 2 * kSsR; ++p) {
        const float2 v1 = sm.h1[ty0 + p][tx], v2 = sm.h2[ty0 + p][tx];
        const float v3 = sm.h3[ty0 + p][tx];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int k = p - j;
          if (k >= 0 && k < kSsTaps) {
            const float2 w = bc2(win.w[k]);
            m1[j] = __ffma2_rn(w, v1, m1[j]);
            m2[j] = __ffma2_rn(w, v2, m2[j]);
            m3[j] = fmaf(win.w[k], v3, m3[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int gx = bx + tx, gy = by + ty0 + j;
        if (gx >= W || gy >= H) continue;
        const float mx = m1[j].x, my = m1[j].y;
        const float vx = m2[j].x - mx * mx, vy = m2[j].y - my * my, cxy = m3[j] - mx * my;
        const float a = 2.f * mx * my + kSsC1, b = 2.f * cxy + kSsC2;
        const float c = mx * mx + my * my + kSsC1, d = vx + vy + kSsC2;
        const float rc = __frcp_rn(c), rd = __frcp_rn(d);  // two reciprocals instead of six divisions
        const float rcd = rc * rd;
        const float sv = a * b * rcd;
        const float A = 2.f * my * (b - a) * rcd - sv * (2.f * mx * rc - 2.f * mx * rd);
        const float Bm = -sv * rd;
        const float Cm = 2.f * a * rcd;
        // planar layout [map][channel][H][W], so the adjoint stages contiguous rows
        const size_t i = (size_t)ch * plane + (size_t)gy * W + gx;
        abc[i] = A;
        abc[3 * plane + i] = Bm;
        abc[6 * plane + i] = Cm;
        sum_1ms += 1.f - sv;
        sum_s += sv;
        // L1 terms (sign(0) = 0), as splat_loss_l1
        const size_t pix = (size_t)gy * W + gx;
        const float2 xy = sxy[ch][ty0 + j + kSsR][tx + kSsR];
        const float e = xy.x - xy.y;
        d_rgb[3 * pix + ch] = e > 0.f ? sc : (e < 0.f ? -sc : 0.f);
        sum_c += fabsf(e);
        if (ch == 0) {
          const float ed = od[j] - otd[j];
          d_depth[pix] = ed > 0.f ? sd : (ed < 0.f ? -sd : 0.f);
          sum_d += fabsf(ed);
        }
      }
      // the horizontal sums are rewritten for the next channel, and after the
      // last channel this patch's buffer is refilled
      __syncthreads();
    }
  }
  cp_async_wait<0>();
  const float t0 = block_sum_256(sum_1ms, sm.red);
  __syncthreads();
  const float t1 = block_sum_256(sum_s, sm.red);
  __syncthreads();
  const float t2 = block_sum_256(sc * sum_c + sd * sum_d, sm.red);
  if (t == 0) {
    atomicAdd(&loss[0], t0 * loss_scale + t2);
    atomicAdd(&loss[1], t1 * ssim_scale);
  }
}

// The adjoint: one CTA per block, the channel's (A, B), C patch staged per
// channel (high occupancy hides the staging loads; a double-buffered
// persistent form measured slower here).
__global__ void __launch_bounds__(256, 6) ssim_bwd_kernel(const float* __restrict__ x, const float* __restrict__ y,
                                                       int H, int W, SsimWin win, float grad_scale,
                                                       const float* __restrict__ abc, float* __restrict__ d_rgb) {
  __shared__ float2 sab[kSsPY][kSsPXp];  // (A, B) of the channel
  __shared__ float sc[kSsPY][kSsPXp];    // C
  __shared__ float2 hab[kSsPY][kSsTXp];
  __shared__ float hc[kSsPY][kSsTXp];
  const int t = threadIdx.x;
  const int bx = blockIdx.x * kSsTX, by = blockIdx.y * kSsTY;
  const size_t plane = (size_t)H * W;
  const int tx = t & 31, ty0 = 2 * (t >> 5);
  for (int ch = 0; ch < 3; ++ch) {
    const float* pa = abc + (size_t)ch * plane;
    // this thread's two outputs: x, y and the gradient so far, requested
    // before the window passes so that the epilogue does not wait for them
    float ox[2], oy[2], og[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gx = bx + tx, gy = by + ty0 + j;
      const bool in = gx < W && gy < H;
      const size_t i = in ? ((size_t)gy * W + gx) * 3 + ch : 0;
      ox[j] = in ? x[i] : 0.f;
      oy[j] = in ? y[i] : 0.f;
      og[j] = in ? d_rgb[i] : 0.f;
    }
    {  // six patch rows per pass, one column per thread
      const int c = t % kSsPX, r0 = t / kSsPX;
      const int gx = bx - kSsR + c;
      if (r0 < 6) {
        const bool inx = gx >= 0 && gx < W;
        for (int r = r0; r < kSsPY; r += 6) {
          const int gy = by - kSsR + r;
          const bool in = inx && gy >= 0 && gy < H;
          const size_t gi = (size_t)gy * W + gx;
          sab[r][c] = in ? make_float2(pa[gi], pa[3 * plane + gi]) : make_float2(0.f, 0.f);
          sc[r][c] = in ? pa[6 * plane + gi] : 0.f;
        }
      }
    }
    __syncthreads();
    if (t < kSsHItems) {
      const int r = t / (kSsTX / kSsRun), c0 = kSsRun * (t % (kSsTX / kSsRun));
      float2 a1[kSsRun];
      float a2[kSsRun];
#pragma unroll
      for (int j = 0; j < kSsRun; ++j) {
        a1[j] = bc2(-0.0f);
        a2[j] = -0.0f;
      }
#pragma unroll
      for (int p = 0; p < kSsRun + 2 * kSsR; ++p) {
        const float2 v = sab[r][c0 + p];
        const float vc = sc[r][c0 + p];
#pragma unroll
        for (int j = 0; j < kSsRun; ++j) {
          const int k = p - j;
          if (k >= 0 && k < kSsTaps) {
            a1[j] = __ffma2_rn(bc2(win.w[k]), v, a1[j]);
            a2[j] = fmaf(win.w[k], vc, a2[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kSsRun; ++j) {
        hab[r][c0 + j] = a1[j];
        hc[r][c0 + j] = a2[j];
      }
    }
    __syncthreads();
    float2 m1[2];
    float m2[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      m1[j] = bc2(-0.0f);
      m2[j] = -0.0f;
    }
#pragma unroll
    for (int p = 0; p < 2 + 2 * kSsR; ++p) {
      const float2 v1 = hab[ty0 + p][tx];
      const float v2 = hc[ty0 + p][tx];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int k = p - j;
        if (k >= 0 && k < kSsTaps) {
          m1[j] = __ffma2_rn(bc2(win.w[k]), v1, m1[j]);
          m2[j] = fmaf(win.w[k], v2, m2[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gx = bx + tx, gy = by + ty0 + j;
      if (gx >= W || gy >= H) continue;
      const size_t i = ((size_t)gy * W + gx) * 3 + ch;
      d_rgb[i] = fmaf(grad_scale, m1[j].x + 2.f * ox[j] * m1[j].y + oy[j] * m2[j], og[j]);
    }
    __syncthreads();  // the staged planes are rewritten for the next channel
  }
}

// ----------------------------------------------------------------------------
// Mahalanobis alignment
// ----------------------------------------------------------------------------
struct MapK {
  const float* mean;
  const float* log_scale;
  const float* quat;
};

// One Gaussian's mean, log-scale and quaternion, loaded together.
struct GaussRec {
  float3 mean, ls;
  float4 q;
};

__device__ __forceinline__ GaussRec load_rec(const MapK& g, int i) {
  GaussRec r;
  r.mean = make_float3(__ldg(g.mean + 3 * (size_t)i), __ldg(g.mean + 3 * (size_t)i + 1), __ldg(g.mean + 3 * (size_t)i + 2));
  r.ls = make_float3(__ldg(g.log_scale + 3 * (size_t)i), __ldg(g.log_scale + 3 * (size_t)i + 1),
                     __ldg(g.log_scale + 3 * (size_t)i + 2));
  r.q = __ldg(reinterpret_cast<const float4*>(g.quat) + i);
  return r;
}

// Sigma = R(q) diag(exp(2 log_scale)) R(q)^T as (xx, xy, xz, yy, yz, zz).
__device__ __forceinline__ void gaussian_cov(const GaussRec& g, float S[6]) {
  float qw = g.q.x, qx = g.q.y, qy = g.q.z, qz = g.q.w;
  const float nn = qw * qw + qx * qx + qy * qy + qz * qz;
  if (nn > 0.f) {
    const float inv = rsqrtf(nn);
    qw *= inv; qx *= inv; qy *= inv; qz *= inv;
  } else {
    qw = 1.f; qx = qy = qz = 0.f;
  }
  const float R[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                      2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                      2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
  const float s2[3] = {expf(2.f * g.ls.x), expf(2.f * g.ls.y), expf(2.f * g.ls.z)};
  int e = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b, ++e)
      S[e] = R[3 * a] * s2[0] * R[3 * b] + R[3 * a + 1] * s2[1] * R[3 * b + 1] + R[3 * a + 2] * s2[2] * R[3 * b + 2];
}

constexpr int kSysN = 28;  // 21 (H upper) + 6 (g) + 1 (cost)

__device__ void maha_solve_apply(const double* __restrict__ sys, float* __restrict__ T,
                                 double* __restrict__ delta_out, int32_t* __restrict__ status);

// With SOLVE the CTA that finishes last (a counter after the system in sys,
// taken after every CTA's atomics are fenced) solves the accumulated system,
// applies the step to T and zeroes sys and the counter for the next call; no
// CTA waits on another.  Every CTA reads T before it counts itself, so the
// update cannot reach a CTA still reading T.
template <bool SOLVE>
__global__ void __launch_bounds__(256) mahalanobis_kernel(MapK A, MapK Bm, const int32_t* __restrict__ pairs,
                                                          const int32_t* __restrict__ weights,
                                                          const int64_t* __restrict__ m_dev, int64_t capacity,
                                                          float* __restrict__ T, float max_d2,
                                                          double* __restrict__ sys, double* __restrict__ delta_out,
                                                          int32_t* __restrict__ status) {
  __shared__ float red[8][kSysN];
  const int64_t M = min(*m_dev, capacity);
  float R[9], t[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) R[3 * a + b] = T[4 * a + b];
    t[a] = T[4 * a + 3];
  }
  // per-thread and per-warp sums in float (a thread takes a few pairs, a warp
  // adds 32 partial sums); the per-CTA totals and the system in double
  float acc[kSysN];
#pragma unroll
  for (int k = 0; k < kSysN; ++k) acc[k] = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    const int2 kl = __ldg(reinterpret_cast<const int2*>(pairs) + i);
    const float w = weights ? (float)__ldg(weights + i) : 1.f;
    // both Gaussians' records are requested at once (one round of gathers)
    const GaussRec ga = load_rec(A, kl.x), gb = load_rec(Bm, kl.y);
    const float xb[3] = {gb.mean.x, gb.mean.y, gb.mean.z}, xa[3] = {ga.mean.x, ga.mean.y, ga.mean.z};
    float p[3], r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      p[a] = R[3 * a] * xb[0] + R[3 * a + 1] * xb[1] + R[3 * a + 2] * xb[2] + t[a];
      r[a] = p[a] - xa[a];
    }
    if (max_d2 > 0.f && r[0] * r[0] + r[1] * r[1] + r[2] * r[2] > max_d2) continue;
    float Sa[6], Sb[6];
    gaussian_cov(ga, Sa);
    gaussian_cov(gb, Sb);
    // R Sb R^T + Sa
    const float Sbf[9] = {Sb[0], Sb[1], Sb[2], Sb[1], Sb[3], Sb[4], Sb[2], Sb[4], Sb[5]};
    float RS[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) RS[3 * a + b] = R[3 * a] * Sbf[b] + R[3 * a + 1] * Sbf[3 + b] + R[3 * a + 2] * Sbf[6 + b];
    float S[6];
    int e = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b, ++e)
        S[e] = RS[3 * a] * R[3 * b] + RS[3 * a + 1] * R[3 * b + 1] + RS[3 * a + 2] * R[3 * b + 2] + Sa[e];
    // inverse of the symmetric S (adjugate / determinant)
    const float c00 = S[3] * S[5] - S[4] * S[4], c01 = S[2] * S[4] - S[1] * S[5], c02 = S[1] * S[4] - S[2] * S[3];
    const float c11 = S[0] * S[5] - S[2] * S[2], c12 = S[1] * S[2] - S[0] * S[4], c22 = S[0] * S[3] - S[1] * S[1];
    const float det = S[0] * c00 + S[1] * c01 + S[2] * c02;
    if (!(det > 0.f)) continue;
    const float id = 1.f / det;
    const float Mi[9] = {c00 * id, c01 * id, c02 * id, c01 * id, c11 * id, c12 * id, c02 * id, c12 * id, c22 * id};
    // J = [I | -[p]x]; columns 3..5 of J are -[p]x = [[0, p2, -p1], [-p2, 0, p0], [p1, -p0, 0]]
    float J[3][6] = {{1.f, 0.f, 0.f, 0.f, p[2], -p[1]}, {0.f, 1.f, 0.f, -p[2], 0.f, p[0]},
                     {0.f, 0.f, 1.f, p[1], -p[0], 0.f}};
    float MJ[3][6], Mr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Mr[a] = Mi[3 * a] * r[0] + Mi[3 * a + 1] * r[1] + Mi[3 * a + 2] * r[2];
#pragma unroll
      for (int c = 0; c < 6; ++c) MJ[a][c] = Mi[3 * a] * J[0][c] + Mi[3 * a + 1] * J[1][c] + Mi[3 * a + 2] * J[2][c];
    }
    const float w2 = 2.f * w;
    e = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = a; b < 6; ++b, ++e)
        acc[e] += w2 * (J[0][a] * MJ[0][b] + J[1][a] * MJ[1][b] + J[2][a] * MJ[2][b]);
#pragma unroll
    for (int a = 0; a < 6; ++a) acc[21 + a] += w2 * (J[0][a] * Mr[0] + J[1][a] * Mr[1] + J[2][a] * Mr[2]);
    acc[27] += w * (r[0] * Mr[0] + r[1] * Mr[1] + r[2] * Mr[2]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kSysN; ++k) {
    float v = acc[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kSysN) {  // the CTA's 8 warp sums in float, one double atomic per number
    float v = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
    if (v != 0.0f) atomicAdd(&sys[threadIdx.x], (double)v);
  }
  if (!SOLVE) return;
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  unsigned long long* count = reinterpret_cast<unsigned long long*>(sys + kSysN);
  if (threadIdx.x == 0) s_last = atomicAdd(count, 1ull) == (unsigned long long)gridDim.x - 1ull;
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double S[kSysN];
  for (int k = 0; k < kSysN; ++k) S[k] = __ldcg(sys + k);
  maha_solve_apply(S, T, delta_out, status);
  for (int k = 0; k < kSysN; ++k) sys[k] = 0.0;
  *count = 0ull;
}

// Solve H delta = -g and apply T <- exp(delta^) T (one thread).  The system
// is scaled to unit diagonal (H' = D H D, g' = D g, D = diag(H)^-1/2),
// factorised (Cholesky) and solved in single precision, and the step mapped
// back (delta = D delta'): double-precision arithmetic is slow on this part
// (a double Cholesky took about 30 us in one thread), and with a unit
// diagonal the single-precision solve loses only about cond(H') ulps.
__device__ void maha_solve_apply(const double* __restrict__ sys, float* __restrict__ T,
                                 double* __restrict__ delta_out, int32_t* __restrict__ status) {
  float H[6][6], L[6][6] = {}, g[6], sc[6], d[6];
  int o = 0;
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) H[a][b] = H[b][a] = (float)sys[o++];
  bool ok = true;
  for (int a = 0; a < 6; ++a) {
    ok = ok && H[a][a] > 0.0f;
    sc[a] = H[a][a] > 0.0f ? 1.0f / sqrtf(H[a][a]) : 0.0f;
    g[a] = (float)sys[21 + a] * sc[a];
  }
  for (int a = 0; a < 6 && ok; ++a)
    for (int b = 0; b < 6; ++b) H[a][b] *= sc[a] * sc[b];
  for (int j = 0; j < 6 && ok; ++j) {  // Cholesky H' = L L^T
    float s = H[j][j];
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0.0f)) {
      ok = false;
      break;
    }
    L[j][j] = sqrtf(s);
    const float r = 1.0f / L[j][j];
    for (int i = j + 1; i < 6; ++i) {
      float v = H[i][j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v * r;
    }
  }
  if (!ok) {
    raise_status(status, SPLAT_ENUMERIC);
    if (delta_out)
      for (int a = 0; a < 6; ++a) delta_out[a] = 0.0;
    return;
  }
  float z[6];
  for (int i = 0; i < 6; ++i) {  // L z = -g'
    float v = -g[i];
    for (int k = 0; k < i; ++k) v -= L[i][k] * z[k];
    z[i] = v / L[i][i];
  }
  for (int i = 5; i >= 0; --i) {  // L^T d' = z
    float v = z[i];
    for (int k = i + 1; k < 6; ++k) v -= L[k][i] * d[k];
    d[i] = v / L[i][i];
  }
  for (int a = 0; a < 6; ++a) d[a] *= sc[a];
  if (delta_out)
    for (int a = 0; a < 6; ++a) delta_out[a] = (double)d[a];
  // exp(d^): R by Rodrigues, t = V rho
  const float px = d[3], py = d[4], pz = d[5];
  const float th2 = px * px + py * py + pz * pz, th = sqrtf(th2);
  float a1, b1, c1;  // sin(th)/th, (1 - cos)/th^2, (th - sin)/th^3
  if (th < 0.1f) {  // series to th^4 (next terms below 3e-10; the closed forms cancel here)
    a1 = 1.0f - th2 * (1.0f / 6.0f) * (1.0f - th2 * (1.0f / 20.0f));
    b1 = 0.5f - th2 * (1.0f / 24.0f) * (1.0f - th2 * (1.0f / 30.0f));
    c1 = (1.0f / 6.0f) - th2 * (1.0f / 120.0f) * (1.0f - th2 * (1.0f / 42.0f));
  } else {
    float sn, cs;
    sincosf(th, &sn, &cs);
    a1 = sn / th;
    b1 = (1.0f - cs) / th2;
    c1 = (th - sn) / (th2 * th);
  }
  const float K[9] = {0.0f, -pz, py, pz, 0.0f, -px, -py, px, 0.0f};
  float K2[9], E[16];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      const float I = i == j ? 1.0f : 0.0f;
      E[4 * i + j] = I + a1 * K[3 * i + j] + b1 * K2[3 * i + j];
    }
    float tv = 0.0f;
    for (int j = 0; j < 3; ++j) {
      const float I = i == j ? 1.0f : 0.0f;
      tv += (I + b1 * K[3 * i + j] + c1 * K2[3 * i + j]) * d[j];
    }
    E[4 * i + 3] = tv;
  }
  E[12] = E[13] = E[14] = 0.0f;
  E[15] = 1.0f;
  float out[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      float v = 0.0f;
      for (int k = 0; k < 4; ++k) v += E[4 * i + k] * T[4 * k + j];
      out[4 * i + j] = v;
    }
  for (int k = 0; k < 16; ++k) T[k] = out[k];
}

__global__ void mahalanobis_step_kernel(const double* __restrict__ sys, float* __restrict__ T,
                                        double* __restrict__ delta_out, int32_t* __restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  maha_solve_apply(sys, T, delta_out, status);
}

// ----------------------------------------------------------------------------
// Pruning
// ----------------------------------------------------------------------------
constexpr int kPrThreads = 256;
constexpr int kPrMaxCols = 16;

struct PruneCols {
  const float* src[kPrMaxCols];
  float* dst[kPrMaxCols];
  int width[kPrMaxCols];
  int n;
};

__device__ __forceinline__ bool prune_decision(const float* __restrict__ logit, const float* __restrict__ ls,
                                               int64_t i, float tau_o, float tau_s, float tau_e) {
  const float lam = __fdiv_rn(1.0f, __fadd_rn(1.0f, exp_full(-logit[i])));
  bool pr = lam < tau_o;
  if (tau_s > 0.f) {
    const float s0 = exp_full(ls[3 * i]), s1 = exp_full(ls[3 * i + 1]), s2 = exp_full(ls[3 * i + 2]);
    const float largest = fmaxf(fmaxf(s0, s1), s2);
    const float total = __fadd_rn(__fadd_rn(s0, s1), s2);
    pr |= largest > tau_s;
    pr |= largest > __fmul_rn(tau_e, __fsub_rn(total, largest));
  }
  return pr;
}

__global__ void __launch_bounds__(kPrThreads) prune_flags_kernel(const float* __restrict__ logit,
                                                                 const float* __restrict__ ls, int64_t n, float tau_o,
                                                                 float tau_s, float tau_e, uint8_t* __restrict__ flag,
                                                                 uint32_t* __restrict__ block_keep) {
  const int64_t i = (int64_t)blockIdx.x * kPrThreads + threadIdx.x;
  bool keep = false;
  if (i < n) {
    const bool pr = prune_decision(logit, ls, i, tau_o, tau_s, tau_e);
    flag[i] = pr ? 1 : 0;
    keep = !pr;
  }
  const int c = __syncthreads_count(keep);
  if (threadIdx.x == 0) block_keep[blockIdx.x] = (uint32_t)c;
}

__global__ void __launch_bounds__(1024) prune_scan_kernel(const uint32_t* __restrict__ block_keep, int nb,
                                                          uint32_t* __restrict__ block_off,
                                                          int64_t* __restrict__ n_keep) {
  __shared__ uint32_t sh[33];
  uint32_t carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    const int b = base + threadIdx.x;
    const uint32_t c = b < nb ? block_keep[b] : 0u;
    uint32_t excl;
    const uint32_t tot = block_excl_scan<1024>(c, excl, sh);
    if (b < nb) block_off[b] = carry + excl;
    carry += tot;
  }
  if (threadIdx.x == 0) *n_keep = (int64_t)carry;
}

__global__ void __launch_bounds__(kPrThreads) prune_scatter_kernel(const uint8_t* __restrict__ flag, int64_t n,
                                                                   const uint32_t* __restrict__ block_off,
                                                                   PruneCols cols) {
  __shared__ uint32_t sh[33];
  const int64_t i = (int64_t)blockIdx.x * kPrThreads + threadIdx.x;
  const bool keep = i < n && flag[i] == 0;
  uint32_t excl;
  block_excl_scan<kPrThreads>(keep ? 1u : 0u, excl, sh);
  if (!keep) return;
  const int64_t dst = (int64_t)block_off[blockIdx.x] + excl;
  for (int c = 0; c < cols.n; ++c) {
    const int w = cols.width[c];
    const float* s = cols.src[c] + i * w;
    float* d = cols.dst[c] + dst * w;
    for (int k = 0; k < w; ++k) d[k] = s[k];
  }
}

struct PruneWs {
  uint8_t* flag;
  uint32_t *block_keep, *block_off;
};

static size_t carve_prune(int64_t n, char* base, PruneWs* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  const size_t nb = (nn + kPrThreads - 1) / kPrThreads;
  PruneWs t;
  t.flag = (uint8_t*)take(nn);
  t.block_keep = (uint32_t*)take(4 * nb);
  t.block_off = (uint32_t*)take(4 * nb);
  if (w) *w = t;
  return off;
}

// Persistent grid of the SSIM statistics kernel: resident CTAs per SM
// (dynamic shared memory above 48 KB is opted into once per device) x SMs,
// at most one CTA per block.
static int ssim_grid(int nblk, int* gf) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(SPLAT_ECUDA, "splat_loss_consensus: no current device");
  static std::atomic<unsigned long long> attr_done{0};
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_done.load() & bit)) {
    if (cudaFuncSetAttribute(ssim_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SsFwdSmem)) !=
        cudaSuccess)
      return fail(SPLAT_ECUDA, "splat_loss_consensus: shared memory opt-in failed");
    attr_done.fetch_or(bit);
  }
  int sms = 152, of = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&of, ssim_fwd_kernel, 256, sizeof(SsFwdSmem)) != cudaSuccess)
    return fail(SPLAT_ECUDA, "splat_loss_consensus: occupancy query failed");
  *gf = std::max(1, std::min(nblk, std::max(1, of) * sms));
  return SPLAT_OK;
}

}  // namespace splat

using namespace splat;

// ----------------------------------------------------------------------------
// Entry points
// ----------------------------------------------------------------------------
extern "C" size_t splat_loss_consensus_workspace_size(int32_t height, int32_t width) {
  if (height < 0 || width < 0) return 0;
  return align_up(sizeof(float) * 3 * 3 * (size_t)std::max(1, height) * (size_t)std::max(1, width));
}

extern "C" int splat_loss_consensus(const float* rgb, const float* depth, const float* target_rgb,
                                    const float* target_depth, int32_t height, int32_t width, float w_l1,
                                    float w_ssim, float w_geom, float* d_rgb, float* d_depth, float* loss, void* ws,
                                    size_t ws_bytes, splat_stream_t stream) {
  if (!rgb || !depth || !target_rgb || !target_depth || !d_rgb || !d_depth || !loss || height < 0 || width < 0)
    return fail(SPLAT_EINVAL, "splat_loss_consensus: bad argument");
  const int64_t npix = (int64_t)height * width;
  if (npix == 0) return SPLAT_OK;
  if (!ws || !aligned16(ws) || ws_bytes < splat_loss_consensus_workspace_size(height, width))
    return fail(SPLAT_EINVAL, "splat_loss_consensus: workspace missing, too small or misaligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const float sc = w_l1 / (float)(3 * npix), sd = w_geom / (float)npix;
  if (w_ssim == 0.f) return launch_loss_l1(rgb, depth, target_rgb, target_depth, npix, sc, sd, d_rgb, d_depth, loss, s);
  int rc;
  const SsimWin win = ssim_window();
  const int nbx = (width + kSsTX - 1) / kSsTX, nblk = nbx * ((height + kSsTY - 1) / kSsTY);
  float* abc = static_cast<float*>(ws);
  const float inv = 1.0f / (float)(3 * npix);
  int gf = 0;
  if ((rc = ssim_grid(nblk, &gf))) return rc;
  SPLAT_LAUNCH("ssim_fwd_kernel", s,
               ssim_fwd_kernel<<<gf, 256, sizeof(SsFwdSmem), s>>>(rgb, target_rgb, depth, target_depth, height, width,
                                                                  nbx, nblk, win, w_ssim * inv, inv, sc, sd, d_rgb,
                                                                  d_depth, abc, loss));
  if ((rc = check_launch("ssim_fwd_kernel"))) return rc;
  const dim3 grid2((unsigned)nbx, (unsigned)((height + kSsTY - 1) / kSsTY));
  SPLAT_LAUNCH("ssim_bwd_kernel", s,
               ssim_bwd_kernel<<<grid2, 256, 0, s>>>(rgb, target_rgb, height, width, win, -w_ssim * inv, abc, d_rgb));
  return check_launch("ssim_bwd_kernel");
}

extern "C" int splat_mahalanobis_system(const splat_gaussians* map_a, const splat_gaussians* map_b,
                                        const int32_t* pairs, const int32_t* weights, const int64_t* m_dev,
                                        int64_t capacity, const float* T, float max_dist, double* sys,
                                        splat_stream_t stream) {
  if (!map_a || !map_b || !m_dev || !T || !sys || capacity < 0 || (capacity > 0 && !pairs))
    return fail(SPLAT_EINVAL, "splat_mahalanobis_system: bad argument");
  if ((map_a->n > 0 && (!map_a->mean || !map_a->log_scale || !map_a->quat)) ||
      (map_b->n > 0 && (!map_b->mean || !map_b->log_scale || !map_b->quat)))
    return fail(SPLAT_EINVAL, "splat_mahalanobis_system: null map array");
  if (!aligned16(map_a->quat) || !aligned16(map_b->quat) || (reinterpret_cast<uintptr_t>(pairs) & 7u) != 0)
    return fail(SPLAT_EINVAL, "splat_mahalanobis_system: quaternions not 16-byte or pairs not 8-byte aligned");
  if (capacity == 0) return SPLAT_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const MapK A{map_a->mean, map_a->log_scale, map_a->quat}, Bm{map_b->mean, map_b->log_scale, map_b->quat};
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((capacity + 255) / 256, 2 * 152));
  SPLAT_LAUNCH("mahalanobis_kernel", s,
               mahalanobis_kernel<false><<<grid, 256, 0, s>>>(A, Bm, pairs, weights, m_dev, capacity,
                                                              const_cast<float*>(T),
                                                              max_dist > 0.f ? max_dist * max_dist : 0.f, sys,
                                                              nullptr, nullptr));
  return check_launch("mahalanobis_kernel");
}

extern "C" int splat_mahalanobis_system_step(const splat_gaussians* map_a, const splat_gaussians* map_b,
                                             const int32_t* pairs, const int32_t* weights, const int64_t* m_dev,
                                             int64_t capacity, float* T, float max_dist, double* sys,
                                             double* delta_out, int32_t* status, splat_stream_t stream) {
  if (!map_a || !map_b || !m_dev || !T || !sys || !status || capacity < 0 || (capacity > 0 && !pairs))
    return fail(SPLAT_EINVAL, "splat_mahalanobis_system_step: bad argument");
  if ((map_a->n > 0 && (!map_a->mean || !map_a->log_scale || !map_a->quat)) ||
      (map_b->n > 0 && (!map_b->mean || !map_b->log_scale || !map_b->quat)))
    return fail(SPLAT_EINVAL, "splat_mahalanobis_system_step: null map array");
  if (!aligned16(map_a->quat) || !aligned16(map_b->quat) || (reinterpret_cast<uintptr_t>(pairs) & 7u) != 0)
    return fail(SPLAT_EINVAL, "splat_mahalanobis_system_step: quaternions not 16-byte or pairs not 8-byte aligned");
  if ((reinterpret_cast<uintptr_t>(sys) & 7u) != 0) return fail(SPLAT_EINVAL, "splat_mahalanobis_system_step: sys");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const MapK A{map_a->mean, map_a->log_scale, map_a->quat}, Bm{map_b->mean, map_b->log_scale, map_b->quat};
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((capacity + 255) / 256, 2 * 152));
  SPLAT_LAUNCH("mahalanobis_kernel", s,
               mahalanobis_kernel<true><<<grid, 256, 0, s>>>(A, Bm, pairs, weights, m_dev, capacity, T,
                                                             max_dist > 0.f ? max_dist * max_dist : 0.f, sys,
                                                             delta_out, status));
  return check_launch("mahalanobis_kernel");
}

extern "C" int splat_mahalanobis_step(const double* sys, float* T, double* delta_out, int32_t* status,
                                      splat_stream_t stream) {
  if (!sys || !T || !status) return fail(SPLAT_EINVAL, "splat_mahalanobis_step: bad argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SPLAT_LAUNCH("mahalanobis_step_kernel", s, mahalanobis_step_kernel<<<1, 32, 0, s>>>(sys, T, delta_out, status));
  return check_launch("mahalanobis_step_kernel");
}

extern "C" size_t splat_prune_workspace_size(int64_t n) { return n < 0 ? 0 : carve_prune(n, nullptr, nullptr); }

extern "C" int splat_prune(const splat_gaussians* g, float tau_o, float tau_s, float tau_e, const splat_column* cols,
                           int32_t n_cols, uint8_t* mask, int64_t* n_keep_dev, void* ws, size_t ws_bytes,
                           splat_stream_t stream) {
  if (!g || !n_keep_dev || !ws || n_cols < 0 || n_cols > kPrMaxCols || (n_cols > 0 && !cols) || g->n < 0 ||
      g->n > 0x7fffffffLL)
    return fail(SPLAT_EINVAL, "splat_prune: bad argument");
  if (g->n > 0 && (!g->opacity_logit || !g->log_scale))
    return fail(SPLAT_EINVAL, "splat_prune: opacity_logit / log_scale missing");
  if (ws_bytes < carve_prune(g->n, nullptr, nullptr)) return fail(SPLAT_EINVAL, "splat_prune: workspace too small");
  PruneCols pc;
  pc.n = n_cols;
  for (int c = 0; c < n_cols; ++c) {
    if (!cols[c].src || !cols[c].dst || cols[c].width < 1 || cols[c].width > 16)
      return fail(SPLAT_EINVAL, "splat_prune: column %d invalid", c);
    pc.src[c] = cols[c].src;
    pc.dst[c] = cols[c].dst;
    pc.width[c] = cols[c].width;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (g->n == 0) {
    if (cudaMemsetAsync(n_keep_dev, 0, sizeof(int64_t), s) != cudaSuccess)
      return fail(SPLAT_ECUDA, "splat_prune: memset failed");
    return SPLAT_OK;
  }
  PruneWs w;
  carve_prune(g->n, static_cast<char*>(ws), &w);
  uint8_t* flag = mask ? mask : w.flag;
  const int nb = (int)((g->n + kPrThreads - 1) / kPrThreads);
  SPLAT_LAUNCH("prune_flags_kernel", s,
               prune_flags_kernel<<<nb, kPrThreads, 0, s>>>(g->opacity_logit, g->log_scale, g->n, tau_o, tau_s, tau_e,
                                                            flag, w.block_keep));
  int rc = check_launch("prune_flags_kernel");
  if (rc) return rc;
  SPLAT_LAUNCH("prune_scan_kernel", s, prune_scan_kernel<<<1, 1024, 0, s>>>(w.block_keep, nb, w.block_off, n_keep_dev));
  if ((rc = check_launch("prune_scan_kernel"))) return rc;
  if (n_cols == 0) return SPLAT_OK;
  SPLAT_LAUNCH("prune_scatter_kernel", s,
               prune_scatter_kernel<<<nb, kPrThreads, 0, s>>>(flag, g->n, w.block_off, pc));
  return check_launch("prune_scatter_kernel");
}
