// render.cu -- per-tile front-to-back compositing of colour, depth and
// silhouette (rendering equation of Sec. 3.3; rendered depth of Sec. 3.5) and
// its back-to-front adjoint, for one view per launch or for several views
// (agents of uneven map sizes, Sec. 3.6) in one persistent launch.
//
// Forward: 128 threads with 2 pixels each ((x, y) and (x, y + 4); a warp
// covers one 8 x 8 quadrant of the tile), the pair's arithmetic in packed
// single-precision pairs.  The tile's list is staged through shared memory in batches of BATCH
// Gaussians (position / depth / opacity, the quadratic form's coefficients
// A = -a/2, B = -b, C = -c/2 with the exponent cut, colour, id) and every
// thread walks the batch in order, two visits per iteration: both exponents
// and exponentials are formed first (two independent dependency chains that
// overlap; a warp alone on its scheduler late in the launch is latency-bound),
// then the two compositing steps in list order.  A pixel whose exponent lies
// below the Gaussian's cut (set by the projection so that opacity *
// exp(power) < 1/255 is certain) or above 0 skips the Gaussian; this changes
// no result.  A tile ends as soon as all of its pixels have reached the
// transmittance stop.  No atomics.
//
// Backward: the same pixels per thread and warp, again in packed pairs.  The
// list of a tile is walked in two independent parts (below): the back part
// starts from each pixel's final transmittance and last contributor, walks
// back to front and recovers T_i = T_{i+1} / (1 - alpha_i); the front part
// walks front to back from T_0 = 1.  With the pixel's upstream gradients folded
// into one scalar per Gaussian, P_i = gC.c_i + gD z_i + gS, and the weights
// w_j = alpha_j T_j, every later weight carries a factor (1 - alpha_i), so
// dL/dalpha_i = T_i P_i - [sum_{j>i} w_j P_j + (gC.bg) T_final] / (1 - alpha_i);
// the bracket is one running sum per pixel.
// Per Gaussian and warp, ten sums (five moments of dL/dpower -- sum dp dx,
// dp dy, dp dx^2, dp dx dy, dp dy^2 -- whose conic terms are applied once per
// Gaussian, plus d opacity, d rgb, d depth) are reduced through a per-warp
// shared-memory transpose: each lane writes its column for up to three
// visits, then lane r adds row r of the 30 with 16-byte loads and packed adds;
// the sums are collected per CTA in shared memory and added to global memory
// with three float4 atomics per Gaussian per CTA.  A warp skips a visit, or
// stops short in one, only when none of its lanes takes part (warp-uniform
// tests: a lane that does not take part computes with zero weights).  As in
// the forward, a warp forms the exponentials of two visits before it takes
// the two visits in walk order.
//
// Persistent launches: a grid of (CTAs per SM) x (SMs) CTAs takes (view, tile)
// work items from one atomic ticket counter until the items run out; no CTA
// ever waits on another.
#include <algorithm>

#include "common.cuh"
#include "internal.cuh"

namespace splat {

constexpr int kFwdThreads = 128;         // forward: two pixels per thread
constexpr int kBwdThreads = 128;          // backward: two pixels per thread
constexpr int kGradStride = 12;           // screen-space gradient row (3 float4)
constexpr int kAccStride = 11;            // shared accumulator row (10 sums, padded)
constexpr int kRedRow = 36;               // transposed-reduction row: 32 lanes + 4 (rows start in different banks)
constexpr int kMaxViews = SPLAT_MAX_VIEWS;
constexpr int kFwdBatch = 128;           // forward: Gaussians staged per batch (single-view calls; 128 measured
                                         // 64.9 us against 66.5 us for 256 at 300k / 640x480)
constexpr int kBwdBatch = 64;            // backward: Gaussians staged per batch (single-view calls)
constexpr int kBwdCtasPerSm = 8;          // backward: resident CTAs per SM (single-view calls)

struct ImageK {
  float* rgb;
  float* depth;
  float* sil;
  float* t_final;
  int32_t* n_contrib;
  int32_t* max_id;
  int32_t* n_used;
};

// L1 terms of the loss taken in the forward's epilogue (t_rgb == nullptr: none).
struct LossK {
  const float* t_rgb;
  const float* t_depth;
  float sc, sd;  // w_rgb / 3P, w_depth / P
  float* g_rgb;
  float* g_depth;
  float* loss;
};

struct ViewK {
  const float4* xyzo;
  const float4* conic;
  const float* rgb;
  const uint32_t* vals;
  const uint2* ranges;
  CamK cam;
  float bg0, bg1, bg2;
  ImageK img;
  const float* d_rgb;
  const float* d_depth;
  const float* d_sil;
  float* g2;
  LossK l1;
  uint32_t* sched;  // tile schedule (filled by the forward, read by the backward) or null
};

struct ViewTable {
  ViewK v[kMaxViews];
  int tile_end[kMaxViews];  // inclusive prefix of the views' tile counts
  int n;
};

// Shared-memory staging of one batch of Gaussians.
constexpr int kMaxWarps = 4;  // warps of a tile CTA (forward and backward), one per 8 x 8 quadrant
constexpr int kQuad = 8;

struct StagePtrs {
  float4* xyzo;
  float4* quad;
  float4* cid;
  uint8_t* wmask;
};

template <int BATCH>
struct Stage {
  float4 xyzo[BATCH];
  float4 quad[BATCH];  // A = -a/2, B = -b, C = -c/2, exponent cut
  float4 cid[BATCH];   // colour r, g, b and the Gaussian's id (bits of .w)
  uint8_t wmask[BATCH];              // warps whose quadrant the Gaussian can reach
  uint8_t wlist[kMaxWarps][BATCH];   // per warp: the staged positions it visits, ascending
};

// Whether the ellipse a dx^2 + 2 b dx dy + c dy^2 <= K (centred at the
// origin) meets the rectangle [dxa, dxb] x [dya, dyb]: the quadratic form is
// convex, so its minimum over the rectangle is 0 with the centre inside, else
// on an edge, where it is a 1-D quadratic minimised in closed form.
__device__ __forceinline__ bool ellipse_meets_rect(float dxa, float dxb, float dya, float dyb, float a, float b,
                                                   float c, float ba, float bc, float K) {
  if (dxa <= 0.0f && 0.0f <= dxb && dya <= 0.0f && 0.0f <= dyb) return true;
  float m = 3.0e38f;
#pragma unroll 1
  for (int e = 0; e < 2; ++e) {
    const float dy = e ? dyb : dya;  // horizontal edge, minimiser dx = -(b/a) dy
    const float dx = fminf(dxb, fmaxf(dxa, -ba * dy));
    m = fminf(m, (a * dx + 2.0f * b * dy) * dx + c * dy * dy);
    const float ex = e ? dxb : dxa;  // vertical edge, minimiser dy = -(b/c) dx
    const float ey = fminf(dyb, fmaxf(dya, -bc * ex));
    m = fminf(m, a * ex * ex + (2.0f * b * ex + c * ey) * ey);
  }
  return m <= K;
}

// Bit w set when the pixel centres of warp w (the 8 x 8 quadrant
// (8 (w & 1), 8 (w >> 1)) of the tile) can lie on the ellipse where the
// exponent reaches the Gaussian's cut (a dx^2 + 2 b dx dy + c dy^2 <= K,
// K = -2 cut): outside it every pixel skips the Gaussian, so a warp whose bit
// is clear need not look at it.  The bounding box of the ellipse (half-widths
// sqrt(K c / det), sqrt(K a / det), det = ac - b^2) gives the candidate
// columns and rows, so the candidate quadrants; with EXACT (the backward pass,
// where a visit costs most) each candidate quadrant's rectangle of pixel
// centres is then tested against the ellipse itself.  K is widened by 0.2% +
// 1e-3 and the box by 0.1% + 0.01 px, far beyond the rounding of the
// per-pixel test, so no pixel that would take the Gaussian is ever left out.
template <bool EXACT>
__device__ __forceinline__ uint8_t warp_mask(const float4 xo, const float4 co, int tx0, int ty0) {
  const float K = -2.0f * co.w;
  if (!(K > 0.0f)) return 0;  // the cut is above 1: no pixel passes
  const float a = co.x, b = co.y, c = co.z;
  const float det = a * c - b * b;
  if (!(det > 0.0f && a > 0.0f && c > 0.0f)) return 0xf;
  const float sk = K / det;
  const float ex = sqrtf(sk * c) * 1.001f + 0.01f;
  const float ey = sqrtf(sk * a) * 1.001f + 0.01f;
  if (!(ex < 1e30f && ey < 1e30f)) return 0xf;
  // pixel centres tx0 + col + 0.5 inside [x - ex, x + ex], same in y
  const float cl = fmaxf(0.0f, ceilf(xo.x - ex - (float)tx0 - 0.5f));
  const float ch = fminf(15.0f, floorf(xo.x + ex - (float)tx0 - 0.5f));
  const float rl = fmaxf(0.0f, ceilf(xo.y - ey - (float)ty0 - 0.5f));
  const float rh = fminf(15.0f, floorf(xo.y + ey - (float)ty0 - 0.5f));
  if (cl > ch || rl > rh) return 0;
  const int c0 = (int)cl, c1 = (int)ch, r0 = (int)rl, r1 = (int)rh;
  const unsigned cols = (c0 < kQuad ? 1u : 0u) | (c1 >= kQuad ? 2u : 0u);
  const unsigned rows = (r0 < kQuad ? 1u : 0u) | (r1 >= kQuad ? 2u : 0u);
  const uint8_t box = (uint8_t)(((rows & 1u) ? cols : 0u) | ((rows & 2u) ? cols << 2 : 0u));
  if (!EXACT) return box;
  const float Kt = K * 1.002f + 1e-3f;
  const float ba = __fdividef(b, a), bc = __fdividef(b, c);
  uint8_t mask = 0;
#pragma unroll 1
  for (int w = 0; w < 4; ++w) {
    if (!((box >> w) & 1)) continue;
    const int qx = kQuad * (w & 1), qy = kQuad * (w >> 1);
    const float xa = (float)(tx0 + max(c0, qx)) + 0.5f, xb = (float)(tx0 + min(c1, qx + kQuad - 1)) + 0.5f;
    const float ya = (float)(ty0 + max(r0, qy)) + 0.5f, yb = (float)(ty0 + min(r1, qy + kQuad - 1)) + 0.5f;
    if (ellipse_meets_rect(xa - xo.x, xb - xo.x, ya - xo.y, yb - xo.y, a, b, c, ba, bc, Kt))
      mask |= (uint8_t)(1u << w);
  }
  return mask;
}

template <bool EXACT>
__device__ __forceinline__ void stage_one(const ViewK& V, uint32_t g, int i, StagePtrs p, int tx0, int ty0) {
  const float4 co = V.conic[g];
  const float4 xo = V.xyzo[g];
  p.xyzo[i] = xo;
  p.quad[i] = make_float4(-0.5f * co.x, -co.y, -0.5f * co.z, co.w);
  p.cid[i] = make_float4(V.rgb[3 * (size_t)g + 0], V.rgb[3 * (size_t)g + 1], V.rgb[3 * (size_t)g + 2],
                         __int_as_float((int32_t)g));
  p.wmask[i] = warp_mask<EXACT>(xo, co, tx0, ty0);
}

// The positions (ascending) of the cnt staged Gaussians whose mask has this
// warp's bit; returns their number.  All lanes of the warp take part.
__device__ __forceinline__ int build_warp_list(const uint8_t* wmask, uint8_t* list, int cnt, int warp) {
  const int lane = threadIdx.x & 31;
  const unsigned lower = (1u << lane) - 1u;
  int n = 0;
  for (int k0 = 0; k0 < cnt; k0 += 32) {
    const int k = k0 + lane;
    const bool in = k < cnt && ((wmask[k] >> warp) & 1u);
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (in) list[n + __popc(m & lower)] = (uint8_t)k;
    n += __popc(m);
  }
  __syncwarp();
  return n;
}

// ----------------------------------------------------------------------------
// Forward
// ----------------------------------------------------------------------------
// Two pixels per thread, (x, y) and (x, y + 4), so one staged Gaussian's loads
// and the shared dx serve both, and their arithmetic runs as packed pairs
// (__fadd2_rn, __fmul2_rn, __ffma2_rn: two IEEE single-precision operations
// each, rounded exactly as the scalar ones, so every value is bit for bit the
// specified one).  A pixel that skips a Gaussian keeps its state by masking:
// its weight is set to 0 (fma(c, 0, C) = C, S + 0 = S) and T, the last
// contributor and the counters are selected.
struct FwdPix {
  float2 T, C0, C1, C2, D, S, wmax;
  int32_t id[2], last[2], used[2];
  bool done[2];
};

__device__ __forceinline__ float2 bcast(float v) { return make_float2(v, v); }

// exp_core of both lanes (same operations as the scalar one).
#if defined(SPLAT_FAST_EXP)
__device__ __forceinline__ float2 exp_core2(float2 x) { return make_float2(__expf(x.x), __expf(x.y)); }
#else
__device__ __forceinline__ float2 exp_core2(float2 x) {
  const float2 t = __fadd2_rn(__fmul2_rn(x, bcast(1.44269502f)), bcast(12582912.0f));
  const float2 k = __fadd2_rn(t, bcast(-12582912.0f));
  float2 r = __ffma2_rn(k, bcast(-0.693145751953125f), x);
  r = __ffma2_rn(k, bcast(-1.42860677e-06f), r);
  float2 q = bcast(1.98412701e-04f);
  q = __ffma2_rn(q, r, bcast(1.38888892e-03f));
  q = __ffma2_rn(q, r, bcast(8.33333377e-03f));
  q = __ffma2_rn(q, r, bcast(4.16666679e-02f));
  q = __ffma2_rn(q, r, bcast(1.66666672e-01f));
  q = __ffma2_rn(q, r, bcast(0.5f));
  q = __ffma2_rn(q, r, bcast(1.0f));
  q = __ffma2_rn(q, r, bcast(1.0f));
  const float2 sc = make_float2(__int_as_float((__float_as_int(t.x) - 0x4B400000 + 127) << 23),
                                __int_as_float((__float_as_int(t.y) - 0x4B400000 + 127) << 23));
  return __fmul2_rn(q, sc);
}
#endif

// The exponent of one staged Gaussian at the thread's two pixels (the
// specified order).  nfy = (-fy0, -fy1).
__device__ __forceinline__ float2 fwd_power(const float4 xo, const float4 qd, float fx, float2 nfy) {
  const float dx = xo.x - fx;
  const float2 dy = __fadd2_rn(bcast(xo.y), nfy);
  const float2 inner = __ffma2_rn(bcast(qd.x), bcast(dx), __fmul2_rn(bcast(qd.y), dy));
  return __ffma2_rn(__fmul2_rn(bcast(qd.z), dy), dy, __fmul2_rn(bcast(dx), inner));
}

// One front-to-back compositing step of the thread's two pixels, given the
// exponent and its exponential (evaluated whatever the tests decide).
__device__ __forceinline__ void composite_apply(FwdPix& q, const float4 xo, const float4 qd, float2 power, float2 G,
                                                const float4* cidp, int32_t pos) {
  bool in0 = !q.done[0] && !(power.x > 0.0f || power.x < qd.w);
  bool in1 = !q.done[1] && !(power.y > 0.0f || power.y < qd.w);
  if (!(in0 || in1)) return;
  const float2 raw = __fmul2_rn(bcast(xo.w), G);
  const float2 alpha = make_float2(fminf(kAlphaCap, raw.x), fminf(kAlphaCap, raw.y));
  in0 = in0 && !(alpha.x < kAlphaMin);
  in1 = in1 && !(alpha.y < kAlphaMin);
  const float2 test_T = __fmul2_rn(q.T, __ffma2_rn(alpha, bcast(-1.0f), bcast(1.0f)));
  if (in0 && test_T.x < kTStop) {
    q.done[0] = true;
    in0 = false;
  }
  if (in1 && test_T.y < kTStop) {
    q.done[1] = true;
    in1 = false;
  }
  if (!(in0 || in1)) return;
  float2 w = __fmul2_rn(alpha, q.T);
  w.x = in0 ? w.x : 0.0f;
  w.y = in1 ? w.y : 0.0f;
  const float4 c = *cidp;
  q.C0 = __ffma2_rn(bcast(c.x), w, q.C0);
  q.C1 = __ffma2_rn(bcast(c.y), w, q.C1);
  q.C2 = __ffma2_rn(bcast(c.z), w, q.C2);
  q.D = __ffma2_rn(bcast(xo.z), w, q.D);
  q.S = __fadd2_rn(q.S, w);
  if (w.x > q.wmax.x) {
    q.wmax.x = w.x;
    q.id[0] = __float_as_int(c.w);
  }
  if (w.y > q.wmax.y) {
    q.wmax.y = w.y;
    q.id[1] = __float_as_int(c.w);
  }
  q.T.x = in0 ? test_T.x : q.T.x;
  q.T.y = in1 ? test_T.y : q.T.y;
  q.last[0] = in0 ? pos + 1 : q.last[0];
  q.last[1] = in1 ? pos + 1 : q.last[1];
  q.used[0] += in0;
  q.used[1] += in1;
}

// Pixel p (0 or 1) of thread t (forward and backward): warp w covers the 8 x 8
// quadrant at (8 (w & 1), 8 (w >> 1)); lane l takes column l & 7 of it and rows
// l >> 3 and (l >> 3) + 4.
__device__ __forceinline__ void pair_pixel(int t, int p, int& lx, int& ly) {
  const int lane = t & 31, warp = t >> 5;
  lx = kQuad * (warp & 1) + (lane & 7);
  ly = kQuad * (warp >> 1) + (lane >> 3) + 4 * p;
}

// |x - t| and the subgradient sc sign(x - t) (sign(0) = 0), as splat_loss_l1.
__device__ __forceinline__ float l1_px(float x, float t, float sc, float* g) {
  const float e = x - t;
  *g = e > 0.f ? sc : (e < 0.f ? -sc : 0.f);
  return fabsf(e);
}

template <int BATCH>
__device__ __forceinline__ void fwd_tile(const ViewK& V, int tile, Stage<BATCH>& sm, float* s_loss) {
  const CamK& cam = V.cam;
  const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
  int lx, ly0, ly1;
  pair_pixel(threadIdx.x, 0, lx, ly0);
  pair_pixel(threadIdx.x, 1, lx, ly1);
  const int px = tx * kTile + lx, py0 = ty * kTile + ly0, py1 = ty * kTile + ly1;
  const bool in0 = px < cam.width && py0 < cam.height, in1 = px < cam.width && py1 < cam.height;
  const float fx = (float)px + 0.5f;
  const float2 nfy = make_float2(-((float)py0 + 0.5f), -((float)py1 + 0.5f));
  FwdPix q;
  q.T = bcast(1.0f);
  q.C0 = q.C1 = q.C2 = q.D = q.S = q.wmax = bcast(0.0f);
  q.id[0] = q.id[1] = -1;
  q.last[0] = q.last[1] = q.used[0] = q.used[1] = 0;
  q.done[0] = !in0;
  q.done[1] = !in1;
  const uint2 rg = V.ranges[tile];
  const int warp = threadIdx.x >> 5;
  const StagePtrs sp{sm.xyzo, sm.quad, sm.cid, sm.wmask};
  for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
    if (__syncthreads_count(q.done[0] && q.done[1]) == kFwdThreads) break;
    const int cnt = (int)min((uint32_t)BATCH, rg.y - start);
    for (int i = threadIdx.x; i < cnt; i += kFwdThreads)
      stage_one<false>(V, V.vals[start + i], i, sp, tx * kTile, ty * kTile);
    __syncthreads();
    const int32_t base = (int32_t)(start - rg.x);
    const int nl = build_warp_list(sm.wmask, sm.wlist[warp], cnt, warp);
    // two visits per iteration: their exponentials are independent chains
    // that overlap; the compositing stays in list order
    int e = 0;
    for (; e + 1 < nl && !(q.done[0] && q.done[1]); e += 2) {
      const int j0 = sm.wlist[warp][e], j1 = sm.wlist[warp][e + 1];
      const float4 xo0 = sm.xyzo[j0], qd0 = sm.quad[j0], xo1 = sm.xyzo[j1], qd1 = sm.quad[j1];
      const float2 p0 = fwd_power(xo0, qd0, fx, nfy), p1 = fwd_power(xo1, qd1, fx, nfy);
      const float2 G0 = exp_core2(p0), G1 = exp_core2(p1);
      composite_apply(q, xo0, qd0, p0, G0, &sm.cid[j0], base + j0);
      composite_apply(q, xo1, qd1, p1, G1, &sm.cid[j1], base + j1);
    }
    if (e < nl && !(q.done[0] && q.done[1])) {
      const int j = sm.wlist[warp][e];
      const float4 xo = sm.xyzo[j], qd = sm.quad[j];
      const float2 p = fwd_power(xo, qd, fx, nfy);
      composite_apply(q, xo, qd, p, exp_core2(p), &sm.cid[j], base + j);
    }
  }
  const LossK& L = V.l1;
  float acc_c = 0.f, acc_d = 0.f;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    if (!(p ? in1 : in0)) continue;
    const size_t i = (size_t)(p ? py1 : py0) * cam.width + px;
    const float T = p ? q.T.y : q.T.x;
    const float c0 = __fmaf_rn(T, V.bg0, p ? q.C0.y : q.C0.x);
    const float c1 = __fmaf_rn(T, V.bg1, p ? q.C1.y : q.C1.x);
    const float c2 = __fmaf_rn(T, V.bg2, p ? q.C2.y : q.C2.x);
    const float d = p ? q.D.y : q.D.x;
    V.img.rgb[3 * i + 0] = c0;
    V.img.rgb[3 * i + 1] = c1;
    V.img.rgb[3 * i + 2] = c2;
    V.img.depth[i] = d;
    V.img.sil[i] = p ? q.S.y : q.S.x;
    V.img.t_final[i] = T;
    V.img.n_contrib[i] = q.last[p];
    V.img.max_id[i] = q.id[p];
    if (V.img.n_used) V.img.n_used[i] = q.used[p];
    if (L.t_rgb) {
      acc_c += l1_px(c0, L.t_rgb[3 * i + 0], L.sc, &L.g_rgb[3 * i + 0]) +
               l1_px(c1, L.t_rgb[3 * i + 1], L.sc, &L.g_rgb[3 * i + 1]) +
               l1_px(c2, L.t_rgb[3 * i + 2], L.sc, &L.g_rgb[3 * i + 2]);
      acc_d += l1_px(d, L.t_depth[i], L.sd, &L.g_depth[i]);
    }
  }
  // per tile, one block reduction of the loss terms and the contributor
  // counts: warp sums, then thread 0 adds the warps' sums, makes one loss
  // atomic and writes the tile's cost into the schedule
  if (L.t_rgb || V.sched) {
    float acc = L.sc * acc_c + L.sd * acc_d;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const unsigned S = __reduce_add_sync(0xffffffffu, (unsigned)(q.last[0] + q.last[1]));
    if ((threadIdx.x & 31) == 0) {
      s_loss[threadIdx.x >> 5] = acc;
      s_loss[kFwdThreads / 32 + (threadIdx.x >> 5)] = __uint_as_float(S);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      unsigned St = 0u;
#pragma unroll
      for (int w = 0; w < kFwdThreads / 32; ++w) {
        t += s_loss[w];
        St += __float_as_uint(s_loss[kFwdThreads / 32 + w]);
      }
      if (L.t_rgb && L.loss) atomicAdd(L.loss, t);
      if (V.sched) V.sched[1 + cam.tiles_x * cam.tiles_y + tile] = St;  // the tile's cost
    }
  }
}

template <int BATCH>
__global__ void __launch_bounds__(kFwdThreads, 8) render_fwd_kernel(ViewK V) {
  __shared__ Stage<BATCH> sm;
  __shared__ float s_loss[2 * kFwdThreads / 32];
  fwd_tile<BATCH>(V, schedule_tile(V.sched, V.cam.tiles_x * V.cam.tiles_y, blockIdx.x), sm, s_loss);
}

// Work item -> (view, tile).
__device__ __forceinline__ int view_of(const ViewTable& T, int item, int& tile) {
  int v = 0;
  while (v + 1 < T.n && item >= T.tile_end[v]) ++v;
  tile = item - (v ? T.tile_end[v - 1] : 0);
  return v;
}

__device__ __forceinline__ int next_item(int* counter, int* s_item) {
  __syncthreads();  // every thread is done with the previous item's shared memory
  if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
  __syncthreads();
  return *s_item;
}

template <int BATCH>
__global__ void __launch_bounds__(kFwdThreads, 8) render_fwd_persistent(ViewTable T, int total, int* counter) {
  __shared__ Stage<BATCH> sm;
  __shared__ float s_loss[2 * kFwdThreads / 32];
  __shared__ int s_item;
  for (int item = next_item(counter, &s_item); item < total; item = next_item(counter, &s_item)) {
    int tile;
    const int v = view_of(T, item, tile);
    tile = schedule_tile(T.v[v].sched, T.v[v].cam.tiles_x * T.v[v].cam.tiles_y, tile);
    fwd_tile<BATCH>(T.v[v], tile, sm, s_loss);
  }
}

// ----------------------------------------------------------------------------
// Backward
// ----------------------------------------------------------------------------
// Each tile's list is split at a position m into a front part [0, m) and a
// back part [m, last), two independent work items.  With the pixel's upstream
// gradients folded into P_i = gC.c_i + gD z_i + gS and w_i = alpha_i T_i,
//   dL/dalpha_i = T_i P_i - Q_i / (1 - alpha_i),
//   Q_i = sum_{j>i} w_j P_j + (gC.bg) T_final.
// The back part walks back to front from T_final: T_i = T_{i+1} / (1 - alpha_i)
// and Q accumulates from (gC.bg) T_final.  The front part walks front to back
// with the forward's own recurrence T_{i+1} = T_i (1 - alpha_i) from T_0 = 1,
// and Q_i = R_i - w_i P_i with R_0 = sum_j w_j P_j + (gC.bg) T_final
// = gC.C + gD D + gS S, the forward's outputs (C with its background term):
// no part waits for the other, so a tile's work is two items of a persistent
// launch.  m is the tile's mean contributor count over two, so the parts are
// about even; the front part takes the early contributors (T_i large, where
// the subtraction R - w P loses nothing that matters) and the back part the
// late ones.
//
// The thread's two pixels (x, y) and (x, y + 4) share x, and their arithmetic
// runs in packed single-precision pairs.  Q holds Q (back part) or R (front).
struct BwdPair {
  float fx;
  float2 nfy, T, gC0, gC1, gC2, gD, gS, Q;
  int last[2];
};

// Per-pixel adjoint of one list position for both pixels of the pair; pixel
// p takes part when pos < last[p] and the Gaussian passes its exponent and
// alpha-floor tests (the forward's decisions, same operations).  Adds the
// pair's share of (sum dp dx, sum dp dy, sum dp dx^2, sum dp dx dy,
// sum dp dy^2, d opacity, d rgb[3], d depth) to v, dp = dL/d(power); returns
// whether either pixel took part.  A pixel that does not take part keeps T
// and Q (its alpha and weight are 0) and adds nothing (its G and raw opacity
// are set to 0).
// The exponent of one staged Gaussian at the pair's pixels, with dx and dy.
__device__ __forceinline__ float2 adjoint_power(const BwdPair& q, const float4 xo, const float4 qd, float& dx,
                                                float2& dy) {
  dx = xo.x - q.fx;
  dy = __fadd2_rn(bcast(xo.y), q.nfy);
  const float2 inner = __ffma2_rn(bcast(qd.x), bcast(dx), __fmul2_rn(bcast(qd.y), dy));
  return __ffma2_rn(__fmul2_rn(bcast(qd.z), dy), dy, __fmul2_rn(bcast(dx), inner));
}

template <bool FRONT>
__device__ __forceinline__ bool adjoint_step2(BwdPair& q, int pos, const float4 xo, const float4 qd, float dx,
                                              float2 dy, float2 power, float2 G, float c0, float c1, float c2,
                                              float (&v)[10]) {
  bool in0 = pos < q.last[0] && !(power.x > 0.0f || power.x < qd.w);
  bool in1 = pos < q.last[1] && !(power.y > 0.0f || power.y < qd.w);
  if (!__any_sync(0xffffffffu, in0 || in1)) return false;
  const float2 raw = __fmul2_rn(bcast(xo.w), G);
  float2 alpha = make_float2(fminf(kAlphaCap, raw.x), fminf(kAlphaCap, raw.y));
  in0 = in0 && !(alpha.x < kAlphaMin);
  in1 = in1 && !(alpha.y < kAlphaMin);
  if (!__any_sync(0xffffffffu, in0 || in1)) return false;
  alpha.x = in0 ? alpha.x : 0.0f;
  alpha.y = in1 ? alpha.y : 0.0f;
  const float2 om = __ffma2_rn(alpha, bcast(-1.0f), bcast(1.0f));
  const float2 r = make_float2(__fdividef(1.0f, om.x), __fdividef(1.0f, om.y));
  float2 Ti;
  if (FRONT) {
    Ti = q.T;
  } else {
    Ti = __fmul2_rn(q.T, r);  // T_i
    q.T.x = in0 ? Ti.x : q.T.x;
    q.T.y = in1 ? Ti.y : q.T.y;
  }
  const float2 w = __fmul2_rn(alpha, Ti);  // 0 for a pixel that does not take part
  const float2 t6 = __fmul2_rn(q.gC0, w), t7 = __fmul2_rn(q.gC1, w), t8 = __fmul2_rn(q.gC2, w);
  const float2 t9 = __fmul2_rn(q.gD, w);
  v[6] += t6.x + t6.y;
  v[7] += t7.x + t7.y;
  v[8] += t8.x + t8.y;
  v[9] += t9.x + t9.y;
  float2 P = __ffma2_rn(q.gC0, bcast(c0), q.gS);
  P = __ffma2_rn(q.gC1, bcast(c1), P);
  P = __ffma2_rn(q.gC2, bcast(c2), P);
  P = __ffma2_rn(q.gD, bcast(xo.z), P);
  float2 dA;
  if (FRONT) {
    const float2 Qi = __ffma2_rn(make_float2(-w.x, -w.y), P, q.Q);  // R_i - w_i P_i
    const float2 rq = __fmul2_rn(r, Qi);
    dA = __ffma2_rn(Ti, P, make_float2(-rq.x, -rq.y));
    q.Q = Qi;
    q.T = __fmul2_rn(q.T, om);  // the forward's T_{i+1}; unchanged (x 1) for a pixel not taking part
  } else {
    const float2 rq = __fmul2_rn(r, q.Q);
    dA = __ffma2_rn(Ti, P, make_float2(-rq.x, -rq.y));
    q.Q = __ffma2_rn(w, P, q.Q);
  }
  const bool l0 = in0 && !(raw.x > kAlphaCap), l1 = in1 && !(raw.y > kAlphaCap);
  const float2 Ge = make_float2(l0 ? G.x : 0.0f, l1 ? G.y : 0.0f);
  const float2 re = make_float2(l0 ? raw.x : 0.0f, l1 ? raw.y : 0.0f);
  const float2 t5 = __fmul2_rn(Ge, dA);
  v[5] += t5.x + t5.y;
  const float2 dp = __fmul2_rn(re, dA);
  const float2 m2 = __fmul2_rn(dp, dy);
  const float2 s4 = __fmul2_rn(m2, dy);
  const float sx = dx * (dp.x + dp.y), sy = m2.x + m2.y;  // the pair shares dx
  v[0] += sx;
  v[1] += sy;
  v[2] += dx * sx;
  v[3] += dx * sy;
  v[4] += s4.x + s4.y;
  return true;
}

template <int BATCH>
struct BwdShared {
  Stage<BATCH> st;
  float acc[BATCH * kAccStride];
  __align__(16) float red[kBwdThreads / 32][3 * 10 * kRedRow];  // per warp: 3 visits' 10 sums, transposed
  int maxlast, sumlast;
};

// Warp sums of up to three buffered visits (each visit: every lane wrote its
// 10 values as one column of 10 rows of kRedRow floats): lane r adds row r
// with eight 16-byte loads and a packed-pair tree, and adds the total to the
// CTA's accumulator entry of that visit's staged position (j0, j1, j2).
__device__ __forceinline__ void flush_visits(const float* rb, float* acc, int nslot, int j0, int j1, int j2, int lane) {
  __syncwarp();
  if (lane < 10 * nslot) {
    const float4* src = reinterpret_cast<const float4*>(rb + lane * kRedRow);
    float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 a = src[i];
      s0 = __fadd2_rn(s0, make_float2(a.x, a.y));
      s1 = __fadd2_rn(s1, make_float2(a.z, a.w));
    }
    const float2 t = __fadd2_rn(s0, s1);
    const float tot = t.x + t.y;
    const int slot = lane >= 20 ? 2 : (lane >= 10 ? 1 : 0);
    const int j = slot == 0 ? j0 : (slot == 1 ? j1 : j2);
    if (tot != 0.f) atomicAdd(acc + j * kAccStride + (lane - 10 * slot), tot);
  }
  __syncwarp();
}

// One part (FRONT: positions [0, m); else [m, last)) of one tile.
template <int BATCH, bool FRONT>
__device__ __forceinline__ void bwd_part(const ViewK& V, int tile, BwdShared<BATCH>& sm) {
  constexpr int NT = kBwdThreads;
  const CamK& cam = V.cam;
  const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
  const uint2 rg = V.ranges[tile];
  BwdPair q;
  int lx, ly0, ly1;
  pair_pixel(threadIdx.x, 0, lx, ly0);
  pair_pixel(threadIdx.x, 1, lx, ly1);
  const int x = tx * kTile + lx;
  q.fx = (float)x + 0.5f;
  {
    float f[2][8];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int y = ty * kTile + (p ? ly1 : ly0);
      const bool inside = x < cam.width && y < cam.height;
      const size_t i = inside ? (size_t)y * cam.width + x : 0;
      const float g0 = inside ? __ldcg(V.d_rgb + 3 * i + 0) : 0.f;
      const float g1 = inside ? __ldcg(V.d_rgb + 3 * i + 1) : 0.f;
      const float g2 = inside ? __ldcg(V.d_rgb + 3 * i + 2) : 0.f;
      const float gd = (inside && V.d_depth) ? __ldcg(V.d_depth + i) : 0.f;
      const float gs = (inside && V.d_sil) ? __ldcg(V.d_sil + i) : 0.f;
      f[p][0] = -((float)y + 0.5f);
      f[p][2] = g0;
      f[p][3] = g1;
      f[p][4] = g2;
      f[p][5] = gd;
      f[p][6] = gs;
      if (FRONT) {
        f[p][1] = 1.0f;
        const float* im = V.img.rgb + 3 * i;
        f[p][7] = inside ? ((g0 * __ldcg(im) + g1 * __ldcg(im + 1)) + g2 * __ldcg(im + 2) + gd * __ldcg(V.img.depth + i)) +
                               gs * __ldcg(V.img.sil + i)
                         : 0.f;
      } else {
        const float Tfin = inside ? __ldcg(V.img.t_final + i) : 1.0f;
        f[p][1] = Tfin;
        f[p][7] = (g0 * V.bg0 + g1 * V.bg1 + g2 * V.bg2) * Tfin;
      }
      q.last[p] = inside ? __ldcg(V.img.n_contrib + i) : 0;
    }
    q.nfy = make_float2(f[0][0], f[1][0]);
    q.T = make_float2(f[0][1], f[1][1]);
    q.gC0 = make_float2(f[0][2], f[1][2]);
    q.gC1 = make_float2(f[0][3], f[1][3]);
    q.gC2 = make_float2(f[0][4], f[1][4]);
    q.gD = make_float2(f[0][5], f[1][5]);
    q.gS = make_float2(f[0][6], f[1][6]);
    q.Q = make_float2(f[0][7], f[1][7]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const StagePtrs sp{sm.st.xyzo, sm.st.quad, sm.st.cid, sm.st.wmask};
  const int wmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)max(q.last[0], q.last[1]));
  const int wsum = (int)__reduce_add_sync(0xffffffffu, (unsigned)(q.last[0] + q.last[1]));
  if (threadIdx.x == 0) sm.maxlast = sm.sumlast = 0;
  __syncthreads();
  if (lane == 0) {
    if (wmax > 0) atomicMax(&sm.maxlast, wmax);
    atomicAdd(&sm.sumlast, wsum);
  }
  __syncthreads();
  const int maxlast = sm.maxlast;
  const int m = min(maxlast, (sm.sumlast + 2 * kTilePixels - 1) / (2 * kTilePixels));  // split position
  // the part's positions [lo, hi) and, per warp, the first position no pixel of the warp reaches
  const int lo = FRONT ? 0 : m, hi = FRONT ? m : maxlast;
  const int wlast = FRONT ? min(wmax, m) : wmax;
  const int nb = (hi - lo + BATCH - 1) / BATCH;
  for (int b = 0; b < nb; ++b) {
    // batches in walk order: ascending from lo (front), descending from hi (back)
    const int start = FRONT ? lo + b * BATCH : max(lo, hi - (b + 1) * BATCH);
    const int cnt = FRONT ? min(BATCH, hi - start) : hi - b * BATCH - start;
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += NT)
      stage_one<true>(V, V.vals[rg.x + start + i], i, sp, tx * kTile, ty * kTile);
    for (int i = threadIdx.x; i < BATCH * kAccStride; i += NT) sm.acc[i] = 0.f;
    __syncthreads();
    const int nl = build_warp_list(sm.st.wmask, sm.st.wlist[warp], cnt, warp);
    float* rb = sm.red[warp];
    int nslot = 0, j0 = 0, j1 = 0, j2 = 0;
    // the warp's visits are the staged positions before wlast: a prefix of
    // the ascending list, walked forwards (front part) or backwards
    int nv = 0;
    for (int k0 = 0; k0 < nl; k0 += 32) {
      const int k = k0 + lane;
      const unsigned ok = __ballot_sync(0xffffffffu, k < nl && start + (int)sm.st.wlist[warp][k] < wlast);
      nv += __popc(ok);
      if (ok != 0xffffffffu) break;
    }
    auto visit = [&](int j, float dx, float2 dy, float2 power, float2 G) {
      const float4 xo = sm.st.xyzo[j];
      const float4 qd = sm.st.quad[j];
      const float4 cd = sm.st.cid[j];
      float v[10];
#pragma unroll
      for (int k = 0; k < 10; ++k) v[k] = -0.0f;  // -0 + x = x exactly: the first sum folds away
      if (adjoint_step2<FRONT>(q, start + j, xo, qd, dx, dy, power, G, cd.x, cd.y, cd.z, v)) {  // warp-uniform
        float* row = rb + nslot * 10 * kRedRow + lane;
#pragma unroll
        for (int k = 0; k < 10; ++k) row[k * kRedRow] = v[k];
        j0 = nslot == 0 ? j : j0;
        j1 = nslot == 1 ? j : j1;
        j2 = nslot == 2 ? j : j2;
        if (++nslot == 3) {
          flush_visits(rb, sm.acc, 3, j0, j1, j2, lane);
          nslot = 0;
        }
      }
    };
    // two visits per iteration: both exponentials first (independent chains)
    for (int i = 0; i < nv; i += 2) {
      const bool two = i + 1 < nv;  // warp-uniform
      const int ja = sm.st.wlist[warp][FRONT ? i : nv - 1 - i];
      const int jb = two ? sm.st.wlist[warp][FRONT ? i + 1 : nv - 2 - i] : ja;
      float dxa, dxb;
      float2 dya, dyb;
      const float2 pa = adjoint_power(q, sm.st.xyzo[ja], sm.st.quad[ja], dxa, dya);
      const float2 pb = adjoint_power(q, sm.st.xyzo[jb], sm.st.quad[jb], dxb, dyb);
      const float2 Ga = exp_core2(pa), Gb = exp_core2(pb);
      visit(ja, dxa, dya, pa, Ga);
      if (two) visit(jb, dxb, dyb, pb, Gb);
    }
    if (nslot) flush_visits(rb, sm.acc, nslot, j0, j1, j2, lane);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += NT) {
      const float* a = &sm.acc[i * kAccStride];
      const float4 qd = sm.st.quad[i];
      const float ca = -2.0f * qd.x, cb = -qd.y, cc = -2.0f * qd.z;  // the conic a, b, c (exact)
      const float4 u0 = make_float4(-(ca * a[0] + cb * a[1]), -(cb * a[0] + cc * a[1]), -0.5f * a[2], -a[3]);
      const float4 u1 = make_float4(-0.5f * a[4], a[5], a[6], a[7]);
      const float4 u2 = make_float4(a[8], a[9], 0.f, 0.f);
      float4* dst = reinterpret_cast<float4*>(V.g2 + kGradStride * (size_t)__float_as_int(sm.st.cid[i].w));
      if (u0.x != 0.f || u0.y != 0.f || u0.z != 0.f || u0.w != 0.f) atomicAdd(dst, u0);
      if (u1.x != 0.f || u1.y != 0.f || u1.z != 0.f || u1.w != 0.f) atomicAdd(dst + 1, u1);
      if (u2.x != 0.f || u2.y != 0.f) atomicAdd(dst + 2, u2);
    }
  }
}

// Work item -> (view, tile, part): items 2 t and 2 t + 1 are the front and back
// parts of the t-th tile over all views (the t-th of the view's schedule,
// heaviest first, when it has one).
template <int BATCH>
__global__ void __launch_bounds__(kBwdThreads, 8) render_bwd_persistent(ViewTable T, int total, int* counter) {
  __shared__ BwdShared<BATCH> sm;
  __shared__ int s_item, s_view, s_tile;
  for (;;) {
    __syncthreads();  // every thread is done with the previous item's shared memory
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= 2 * total) break;
    if (threadIdx.x < 32) {  // the item's view and tile
      int tile;
      const int v = view_of(T, item >> 1, tile);
      tile = schedule_tile(T.v[v].sched, T.v[v].cam.tiles_x * T.v[v].cam.tiles_y, tile);
      if (threadIdx.x == 0) {
        s_view = v;
        s_tile = tile;
      }
    }
    __syncthreads();
    if (item & 1)
      bwd_part<BATCH, false>(T.v[s_view], s_tile, sm);
    else
      bwd_part<BATCH, true>(T.v[s_view], s_tile, sm);
  }
}

// ----------------------------------------------------------------------------
// Forward and backward in one launch (one view)
// ----------------------------------------------------------------------------
// The backward of a tile needs only that tile's forward outputs and loss
// gradients, so both run as items of one persistent launch: items [0, T) are
// the forward of the schedule's tiles (heaviest first), items [T, 3 T) the two
// backward parts of the tiles in the order their forwards finished.  A forward
// item ends with every thread's writes fenced, then takes the next slot of a
// completion queue and release-stores its tile there; backward items 2 j and
// 2 j + 1 wait (acquire loads) for slot j.  All forward items were taken from
// the ticket counter before any backward item, by CTAs that are running, so
// slot j is always filled; the wait is still bounded (kFlagWaitLimit polls),
// after which SPLAT_ETIMEOUT is raised and the item is skipped.  A backward
// item never waits for one particular tile, only for the j-th finished one.
// The launch is cooperative (all CTAs resident).
// The backward's reads of forward outputs bypass L1 (ld.global.cg), which is
// not coherent with other SMs' writes.
constexpr unsigned kFlagWaitLimit = 1u << 22;

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int FB, int BB>
union FusedShared {
  Stage<FB> f;
  BwdShared<BB> b;
};

template <int FB, int BB>
__global__ void __launch_bounds__(kBwdThreads, 8) render_fused_persistent(ViewK V, int n_tiles, int* counter,
                                                                         int* queue, int32_t* status) {
  static_assert(kFwdThreads == kBwdThreads, "one block shape for both item kinds");
  __shared__ FusedShared<FB, BB> sm;
  __shared__ float s_loss[2 * kFwdThreads / 32];
  __shared__ int s_item, s_tile, s_ok;
  for (;;) {
    __syncthreads();  // every thread is done with the previous item's shared memory
    if (threadIdx.x == 0) {  // the item, its tile and, for a backward item, the wait for the tile's forward
      const int item = atomicAdd(counter, 1);
      int ok = 1, tile = 0;
      if (item < n_tiles) {
        tile = schedule_tile(V.sched, n_tiles, item);
      } else if (item < 3 * n_tiles) {  // slot j of the queue holds the j-th finished tile + 1
        const int* slot = queue + 1 + ((item - n_tiles) >> 1);
        unsigned polls = 0;
        int t1;
        while ((t1 = ld_acquire(slot)) == 0) {
          if (++polls > kFlagWaitLimit) {
            ok = 0;
            raise_status(status, SPLAT_ETIMEOUT);
            break;
          }
          __nanosleep(64);
        }
        tile = ok ? t1 - 1 : 0;
      }
      s_item = item;
      s_tile = tile;
      s_ok = ok;
    }
    __syncthreads();
    const int item = s_item;
    if (item >= 3 * n_tiles) break;
    if (!s_ok) continue;
    if (item < n_tiles) {
      fwd_tile<FB>(V, s_tile, sm.f, s_loss);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) st_release(queue + 1 + atomicAdd(queue, 1), s_tile + 1);
    } else if ((item - n_tiles) & 1) {
      bwd_part<BB, false>(V, s_tile, sm.b);
    } else {
      bwd_part<BB, true>(V, s_tile, sm.b);
    }
  }
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
static int check_proj(const splat_projected* proj, int64_t n, const char* who) {
  if (!proj || (n > 0 && (!proj->xyzo || !proj->conic)) || !aligned16(proj->xyzo) || !aligned16(proj->conic))
    return fail(SPLAT_EINVAL, "%s: projected arrays null or not 16-byte aligned", who);
  return SPLAT_OK;
}

static bool image_ok(const splat_image& im) {
  return im.rgb && im.depth && im.sil && im.t_final && im.n_contrib && im.max_id;
}

static ViewK make_view(const splat_projected& proj, const float* rgb, const uint32_t* vals, const uint32_t* ranges,
                       const splat_camera& cam, const float* bg, const splat_image& im) {
  ViewK v;
  v.xyzo = reinterpret_cast<const float4*>(proj.xyzo);
  v.conic = reinterpret_cast<const float4*>(proj.conic);
  v.rgb = rgb;
  v.vals = vals;
  v.ranges = reinterpret_cast<const uint2*>(ranges);
  v.cam = make_camk(cam);
  v.bg0 = bg[0];
  v.bg1 = bg[1];
  v.bg2 = bg[2];
  v.img = ImageK{im.rgb, im.depth, im.sil, im.t_final, im.n_contrib, im.max_id, im.n_used};
  v.d_rgb = v.d_depth = v.d_sil = nullptr;
  v.g2 = nullptr;
  v.l1 = LossK{nullptr, nullptr, 0.f, 0.f, nullptr, nullptr, nullptr};
  v.sched = nullptr;
  return v;
}

static int set_loss(ViewK& v, const splat_l1* l1, const char* who) {
  if (!l1) return SPLAT_OK;
  if (!l1->t_rgb || !l1->t_depth || !l1->d_rgb || !l1->d_depth)
    return fail(SPLAT_EINVAL, "%s: L1 targets or gradient images are null", who);
  const int64_t npix = (int64_t)v.cam.width * v.cam.height;
  v.l1 = LossK{l1->t_rgb, l1->t_depth, l1->w_rgb / (float)(3 * npix), l1->w_depth / (float)npix, l1->d_rgb,
               l1->d_depth, l1->loss};
  return SPLAT_OK;
}

static int sm_count() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace splat

using namespace splat;

static int render_fwd_one(const splat_projected* proj, const float* rgb, int64_t n, const uint32_t* vals,
                          const uint32_t* ranges, const splat_camera* cam, const float* bg, const splat_image* out,
                          const splat_l1* l1, uint32_t* schedule, splat_stream_t stream, const char* who) {
  int rc = check_proj(proj, n, who);
  if (rc) return rc;
  if ((n > 0 && !rgb) || !vals || !ranges || !cam || !bg || !out || !image_ok(*out))
    return fail(SPLAT_EINVAL, "%s: null argument", who);
  if (n < 0 || cam->width <= 0 || cam->height <= 0) return fail(SPLAT_EINVAL, "%s: bad sizes", who);
  ViewK v = make_view(*proj, rgb, vals, ranges, *cam, bg, *out);
  if ((rc = set_loss(v, l1, who))) return rc;
  v.sched = schedule;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SPLAT_LAUNCH("render_fwd_kernel", s,
               render_fwd_kernel<kFwdBatch><<<v.cam.tiles_x * v.cam.tiles_y, kFwdThreads, 0, s>>>(v));
  return check_launch("render_fwd_kernel");
}

extern "C" int splat_render_fwd(const splat_projected* proj, const float* rgb, int64_t n, const uint32_t* vals,
                                const uint32_t* ranges, const splat_camera* cam, const float* bg,
                                const splat_image* out, splat_stream_t stream) {
  return render_fwd_one(proj, rgb, n, vals, ranges, cam, bg, out, nullptr, nullptr, stream, "splat_render_fwd");
}

extern "C" int splat_render_fwd_l1(const splat_projected* proj, const float* rgb, int64_t n, const uint32_t* vals,
                                   const uint32_t* ranges, const splat_camera* cam, const float* bg,
                                   const splat_image* out, const splat_l1* l1, uint32_t* schedule,
                                   splat_stream_t stream) {
  return render_fwd_one(proj, rgb, n, vals, ranges, cam, bg, out, l1, schedule, stream, "splat_render_fwd_l1");
}

extern "C" size_t splat_tile_schedule_size(int32_t n_tiles) {
  return n_tiles < 1 ? 0 : sizeof(uint32_t) * (1 + 2 * (size_t)n_tiles);
}

// Workspace of splat_render_bwd: the screen-space gradients [n, 12] and, after
// them, the work-item counter of the persistent launch.
static size_t g2_bytes(int64_t n) { return align_up(sizeof(float) * kGradStride * (size_t)std::max<int64_t>(n, 1)); }

extern "C" size_t splat_render_bwd_workspace_size(int64_t n) { return n < 0 ? 0 : g2_bytes(n) + 256; }

extern "C" int splat_render_bwd(const splat_gaussians* g, const splat_projected* proj, const splat_camera* cam,
                                const float* w2c, const uint32_t* vals, const uint32_t* ranges,
                                const uint32_t* schedule, const splat_image* fwd, const float* bg,
                                const float* d_rgb, const float* d_depth,
                                const float* d_sil, const splat_gaussians_grad* out, float* d_pose, float* d2d,
                                void* ws, size_t ws_bytes, splat_stream_t stream) {
  if (!g) return fail(SPLAT_EINVAL, "splat_render_bwd: null argument");
  int rc = check_proj(proj, g->n, "splat_render_bwd");
  if (rc) return rc;
  const bool screen_only = !out && !d_pose && !d2d;  // the screen-space gradients alone, left in ws
  if (!cam || !w2c || !vals || !ranges || !fwd || !fwd->t_final || !fwd->n_contrib || !bg || !d_rgb ||
      (!out && !screen_only) ||
      (out && g->n > 0 && (!out->mean || !out->log_scale || !out->quat || !out->opacity_logit || !out->rgb)))
    return fail(SPLAT_EINVAL, "splat_render_bwd: null argument");
  if ((g->n > 0 && (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->rgb)) || !aligned16(g->quat))
    return fail(SPLAT_EINVAL, "splat_render_bwd: gaussian arrays null or quat not 16-byte aligned");
  if (g->n < 0 || cam->width <= 0 || cam->height <= 0) return fail(SPLAT_EINVAL, "splat_render_bwd: bad sizes");
  if (g->n > 0 && !proj->radius) return fail(SPLAT_EINVAL, "splat_render_bwd: proj->radius is null");
  if (!ws || !aligned16(ws) || ws_bytes < splat_render_bwd_workspace_size(g->n))
    return fail(SPLAT_EINVAL, "splat_render_bwd: workspace missing, too small or not 16-byte aligned");
  if (!fwd->rgb || !fwd->depth || !fwd->sil) return fail(SPLAT_EINVAL, "splat_render_bwd: forward image incomplete");
  float* g2 = static_cast<float*>(ws);
  int* counter = reinterpret_cast<int*>(static_cast<char*>(ws) + g2_bytes(g->n));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t clear = g->n > 0 ? g2_bytes(g->n) + sizeof(int) : 0;
  if (clear && cudaMemsetAsync(ws, 0, clear, s) != cudaSuccess)
    return fail(SPLAT_ECUDA, "splat_render_bwd: memset failed");
  if (!clear && cudaMemsetAsync(counter, 0, sizeof(int), s) != cudaSuccess)
    return fail(SPLAT_ECUDA, "splat_render_bwd: memset failed");
  ViewTable T;
  T.v[0] = make_view(*proj, g->rgb, vals, ranges, *cam, bg, *fwd);
  T.v[0].d_rgb = d_rgb;
  T.v[0].d_depth = d_depth;
  T.v[0].d_sil = d_sil;
  T.v[0].g2 = g2;
  T.v[0].sched = const_cast<uint32_t*>(schedule);
  const int tiles = T.v[0].cam.tiles_x * T.v[0].cam.tiles_y;
  T.tile_end[0] = tiles;
  T.n = 1;
  const int grid = std::min(2 * tiles, kBwdCtasPerSm * sm_count());
  SPLAT_LAUNCH("render_bwd_persistent", s,
               render_bwd_persistent<kBwdBatch><<<grid, kBwdThreads, 0, s>>>(T, tiles, counter));
  if ((rc = check_launch("render_bwd_persistent"))) return rc;
  if (screen_only) return SPLAT_OK;
  const ViewK& v = T.v[0];
  GaussiansK gk{g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, g->n};
  GradK gr{out->mean, out->log_scale, out->quat, out->opacity_logit, out->rgb};
  return launch_project_bwd(gk, v.cam, w2c, proj->conic, proj->radius, g2, kGradStride, gr, d_pose, d2d, s);
}

// Workspace of splat_render_fwd_bwd: that of splat_render_bwd, then the
// completion queue (a count and one slot per tile).
extern "C" size_t splat_render_fwd_bwd_workspace_size(int64_t n, int32_t n_tiles) {
  if (n < 0 || n_tiles < 0) return 0;
  return g2_bytes(n) + 256 + align_up(sizeof(int) * (1 + (size_t)std::max(n_tiles, 1)));
}

extern "C" int splat_render_fwd_bwd(const splat_projected* proj, const float* rgb, int64_t n, const uint32_t* vals,
                                    const uint32_t* ranges, const splat_camera* cam, const float* bg,
                                    const splat_image* out, const splat_l1* l1, uint32_t* schedule, int32_t* status,
                                    void* ws, size_t ws_bytes, splat_stream_t stream) {
  const char* who = "splat_render_fwd_bwd";
  int rc = check_proj(proj, n, who);
  if (rc) return rc;
  if ((n > 0 && !rgb) || !vals || !ranges || !cam || !bg || !out || !image_ok(*out) || !l1 || !status)
    return fail(SPLAT_EINVAL, "%s: null argument", who);
  if (n < 0 || cam->width <= 0 || cam->height <= 0) return fail(SPLAT_EINVAL, "%s: bad sizes", who);
  ViewK v = make_view(*proj, rgb, vals, ranges, *cam, bg, *out);
  if ((rc = set_loss(v, l1, who))) return rc;
  const int tiles = v.cam.tiles_x * v.cam.tiles_y;
  if (!ws || !aligned16(ws) || ws_bytes < splat_render_fwd_bwd_workspace_size(n, tiles))
    return fail(SPLAT_EINVAL, "%s: workspace missing, too small or not 16-byte aligned", who);
  v.sched = schedule;
  v.d_rgb = l1->d_rgb;
  v.d_depth = l1->d_depth;
  v.d_sil = nullptr;
  v.g2 = static_cast<float*>(ws);
  int* counter = reinterpret_cast<int*>(static_cast<char*>(ws) + g2_bytes(n));
  int* queue = reinterpret_cast<int*>(static_cast<char*>(ws) + g2_bytes(n) + 256);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(ws, 0, g2_bytes(n) + 256 + sizeof(int) * (1 + (size_t)tiles), s) != cudaSuccess)
    return fail(SPLAT_ECUDA, "%s: memset failed", who);
  // cooperative: the grid is at most what is resident at once
  auto kern = render_fused_persistent<256, kBwdBatch>;
  int dev = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBwdThreads, 0) != cudaSuccess || per_sm < 1)
    return fail(SPLAT_ECUDA, "%s: occupancy query failed", who);
  int grid = std::min(3 * tiles, per_sm * sm_count());
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBwdThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SPLAT_LAUNCH("render_fused_persistent", s, cudaLaunchKernelEx(&cfg, kern, v, tiles, counter, queue, status));
  return check_launch("render_fused_persistent");
}

extern "C" int splat_project_bwd(const splat_gaussians* g, const splat_projected* proj, const splat_camera* cam,
                                 const float* w2c, const float* grad2d, const splat_gaussians_grad* out,
                                 float* d_pose, float* d2d, splat_stream_t stream) {
  if (!g || !cam || !w2c || !grad2d || (!out && !d_pose && !d2d))
    return fail(SPLAT_EINVAL, "splat_project_bwd: null argument");
  int rc = check_proj(proj, g->n, "splat_project_bwd");
  if (rc) return rc;
  if (g->n < 0 || (g->n > 0 && (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit)) ||
      (g->n > 0 && out && (!out->mean || !out->log_scale || !out->quat || !out->opacity_logit || !out->rgb)) ||
      !aligned16(g->quat) || !aligned16(grad2d))
    return fail(SPLAT_EINVAL, "splat_project_bwd: bad gaussian or gradient arrays");
  if (g->n > 0 && !proj->radius) return fail(SPLAT_EINVAL, "splat_project_bwd: proj->radius is null");
  GaussiansK gk{g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, g->n};
  GradK gr{};  // all null without `out`: the pose (and d2d) only
  if (out) gr = GradK{out->mean, out->log_scale, out->quat, out->opacity_logit, out->rgb};
  return launch_project_bwd(gk, make_camk(*cam), w2c, proj->conic, proj->radius, grad2d, kGradStride, gr, d_pose, d2d,
                            reinterpret_cast<cudaStream_t>(stream));
}

static int make_adam_map(const splat_gaussians* g, const splat_gaussians_grad* m, const splat_gaussians_grad* v,
                         const float* lr, float beta1, float beta2, float eps, const int32_t* step, uint32_t* seen,
                         AdamMapK* A, const char* who) {
  if (!g || !m || !v || !lr || !step) return fail(SPLAT_EINVAL, "%s: null argument", who);
  if (g->n < 0 || (g->n > 0 && (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->rgb || !m->mean ||
                                !m->log_scale || !m->quat || !m->opacity_logit || !m->rgb || !v->mean ||
                                !v->log_scale || !v->quat || !v->opacity_logit || !v->rgb)))
    return fail(SPLAT_EINVAL, "%s: bad gaussian or moment arrays", who);
  float* const P[5] = {const_cast<float*>(g->mean), const_cast<float*>(g->log_scale), const_cast<float*>(g->quat),
                       const_cast<float*>(g->opacity_logit), const_cast<float*>(g->rgb)};
  float* const Ms[5] = {m->mean, m->log_scale, m->quat, m->opacity_logit, m->rgb};
  float* const Vs[5] = {v->mean, v->log_scale, v->quat, v->opacity_logit, v->rgb};
  for (int k = 0; k < 5; ++k) {
    A->p[k] = P[k];
    A->m[k] = Ms[k];
    A->v[k] = Vs[k];
    A->lr[k] = lr[k];
    A->vec[k] = aligned16(P[k]) && aligned16(Ms[k]) && aligned16(Vs[k]);
  }
  A->b1 = beta1;
  A->b2 = beta2;
  A->eps = eps;
  A->step = step;
  A->seen = seen;
  return SPLAT_OK;
}

extern "C" int splat_project_bwd_adam(const splat_gaussians* g, const splat_projected* proj, const splat_camera* cam,
                                      const float* w2c, const float* grad2d, const splat_gaussians_grad* m,
                                      const splat_gaussians_grad* v, const float* lr, float beta1, float beta2,
                                      float eps, const int32_t* step, uint32_t* seen, int32_t culled,
                                      float* d_pose, const splat_pose_adam* pose, splat_stream_t stream) {
  if (!g || !cam || !w2c || !grad2d) return fail(SPLAT_EINVAL, "splat_project_bwd_adam: null argument");
  int rc = check_proj(proj, g->n, "splat_project_bwd_adam");
  if (rc) return rc;
  AdamMapK A;
  if ((rc = make_adam_map(g, m, v, lr, beta1, beta2, eps, step, seen, &A, "splat_project_bwd_adam"))) return rc;
  if (!aligned16(g->quat) || !aligned16(grad2d))
    return fail(SPLAT_EINVAL, "splat_project_bwd_adam: quat or grad2d not 16-byte aligned");
  if (g->n > 0 && !proj->radius) return fail(SPLAT_EINVAL, "splat_project_bwd_adam: proj->radius is null");
  GaussiansK gk{g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, g->n};
  PoseAdamK P{};
  if (pose) {
    if (!pose->w2c || !pose->m || !pose->v || !pose->step || !pose->counter || !d_pose)
      return fail(SPLAT_EINVAL, "splat_project_bwd_adam: pose step without w2c, moments, step, counter or d_pose");
    P = PoseAdamK{pose->w2c, pose->m, pose->v, pose->step, pose->lr_t, pose->lr_r, pose->beta1, pose->beta2,
                  pose->eps, pose->counter};
  }
  return launch_project_bwd_adam(gk, make_camk(*cam), w2c, proj->conic, proj->radius, grad2d, kGradStride, A, d_pose,
                                 P, culled != 0, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int splat_adam_culled(const splat_gaussians* g, const int32_t* radius, const splat_gaussians_grad* m,
                                 const splat_gaussians_grad* v, const float* lr, float beta1, float beta2, float eps,
                                 const int32_t* step, uint32_t* seen, splat_stream_t stream) {
  AdamMapK A;
  int rc = make_adam_map(g, m, v, lr, beta1, beta2, eps, step, seen, &A, "splat_adam_culled");
  if (rc) return rc;
  if (g->n > 0 && !radius) return fail(SPLAT_EINVAL, "splat_adam_culled: radius is null");
  return launch_adam_culled(g->n, radius, A, reinterpret_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// Several views in one persistent launch
// ---------------------------------------------------------------------------
static int build_table(const splat_view* views, int32_t n_views, bool bwd, ViewTable* T, int* total,
                       const char* who) {
  if (!views || n_views < 1 || n_views > kMaxViews)
    return fail(SPLAT_EINVAL, "%s: n_views must be in 1..%d", who, kMaxViews);
  int acc = 0;
  for (int i = 0; i < n_views; ++i) {
    const splat_view& w = views[i];
    if (check_proj(&w.proj, w.n, who) || w.n < 0 || (w.n > 0 && !w.rgb) || !w.vals || !w.ranges ||
        w.cam.width <= 0 || w.cam.height <= 0 || !image_ok(w.image))
      return fail(SPLAT_EINVAL, "%s: view %d is incomplete", who, i);
    if (bwd && (!w.d_rgb || !w.grad2d || !aligned16(w.grad2d)))
      return fail(SPLAT_EINVAL, "%s: view %d lacks d_rgb or a 16-byte aligned grad2d", who, i);
    ViewK v = make_view(w.proj, w.rgb, w.vals, w.ranges, w.cam, w.bg, w.image);
    if (!bwd) {
      const int rc = set_loss(v, w.l1, who);
      if (rc) return rc;
    }
    v.d_rgb = w.d_rgb;
    v.d_depth = w.d_depth;
    v.d_sil = w.d_sil;
    v.g2 = w.grad2d;
    v.sched = w.schedule;
    T->v[i] = v;
    acc += v.cam.tiles_x * v.cam.tiles_y;
    T->tile_end[i] = acc;
  }
  T->n = n_views;
  *total = acc;
  return SPLAT_OK;
}

static splat_batch_shape default_shape() { return splat_batch_shape{256, 4, kBwdBatch, kBwdCtasPerSm}; }

static bool shape_ok(const splat_batch_shape& sh) {
  auto b = [](int x) { return x == 64 || x == 128 || x == 256; };
  return b(sh.fwd_batch) && b(sh.bwd_batch) && sh.fwd_ctas_per_sm >= 1 && sh.fwd_ctas_per_sm <= 8 &&
         sh.bwd_ctas_per_sm >= 1 && sh.bwd_ctas_per_sm <= 16;
}

extern "C" size_t splat_batch_workspace_size(void) { return 256; }

extern "C" int splat_render_fwd_batch(const splat_view* views, int32_t n_views, const splat_batch_shape* shape,
                                      void* ws, size_t ws_bytes, splat_stream_t stream) {
  ViewTable T;
  int total = 0;
  int rc = build_table(views, n_views, false, &T, &total, "splat_render_fwd_batch");
  if (rc) return rc;
  const splat_batch_shape sh = shape ? *shape : default_shape();
  if (!shape_ok(sh)) return fail(SPLAT_EINVAL, "splat_render_fwd_batch: unsupported shape");
  if (!ws || ws_bytes < splat_batch_workspace_size()) return fail(SPLAT_EINVAL, "splat_render_fwd_batch: workspace");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* counter = static_cast<int*>(ws);
  if (cudaMemsetAsync(counter, 0, sizeof(int), s) != cudaSuccess)
    return fail(SPLAT_ECUDA, "splat_render_fwd_batch: memset failed");
  const int grid = std::min(total, sh.fwd_ctas_per_sm * sm_count());
  if (grid <= 0) return SPLAT_OK;
  switch (sh.fwd_batch) {
    case 64:
      SPLAT_LAUNCH("render_fwd_persistent", s,
                   render_fwd_persistent<64><<<grid, kFwdThreads, 0, s>>>(T, total, counter));
      break;
    case 128:
      SPLAT_LAUNCH("render_fwd_persistent", s,
                   render_fwd_persistent<128><<<grid, kFwdThreads, 0, s>>>(T, total, counter));
      break;
    default:
      SPLAT_LAUNCH("render_fwd_persistent", s,
                   render_fwd_persistent<256><<<grid, kFwdThreads, 0, s>>>(T, total, counter));
  }
  return check_launch("render_fwd_persistent");
}

extern "C" int splat_render_bwd_batch(const splat_view* views, int32_t n_views, const splat_batch_shape* shape,
                                      void* ws, size_t ws_bytes, splat_stream_t stream) {
  ViewTable T;
  int total = 0;
  int rc = build_table(views, n_views, true, &T, &total, "splat_render_bwd_batch");
  if (rc) return rc;
  const splat_batch_shape sh = shape ? *shape : default_shape();
  if (!shape_ok(sh)) return fail(SPLAT_EINVAL, "splat_render_bwd_batch: unsupported shape");
  if (!ws || ws_bytes < splat_batch_workspace_size()) return fail(SPLAT_EINVAL, "splat_render_bwd_batch: workspace");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* counter = static_cast<int*>(ws) + 1;
  if (cudaMemsetAsync(counter, 0, sizeof(int), s) != cudaSuccess)
    return fail(SPLAT_ECUDA, "splat_render_bwd_batch: memset failed");
  for (int i = 0; i < n_views; ++i)
    if (views[i].n > 0 &&
        cudaMemsetAsync(views[i].grad2d, 0, sizeof(float) * kGradStride * (size_t)views[i].n, s) != cudaSuccess)
      return fail(SPLAT_ECUDA, "splat_render_bwd_batch: memset failed");
  const int grid = std::min(2 * total, sh.bwd_ctas_per_sm * sm_count());
  if (grid <= 0) return SPLAT_OK;
  switch (sh.bwd_batch) {
    case 64:
      SPLAT_LAUNCH("render_bwd_persistent", s,
                   render_bwd_persistent<64><<<grid, kBwdThreads, 0, s>>>(T, total, counter));
      break;
    case 128:
      SPLAT_LAUNCH("render_bwd_persistent", s,
                   render_bwd_persistent<128><<<grid, kBwdThreads, 0, s>>>(T, total, counter));
      break;
    default:
      SPLAT_LAUNCH("render_bwd_persistent", s,
                   render_bwd_persistent<256><<<grid, kBwdThreads, 0, s>>>(T, total, counter));
  }
  return check_launch("render_bwd_persistent");
}
