// binsort.cu -- tile binning and (tile, depth) ordering of the Gaussians
// (the front-to-back order that the rendering equation of Sec. 3.3
// composites in, per 16x16 tile), plus the device-wide scan and radix sort
// primitives the library uses.
//
// Design.  Binning is a two-level (MSD) radix sort of the (tile, depth, id)
// duplicates: the top digit is the tile id, sorted by counting -- per-tile
// counts with atomics, one exclusive scan whose result is directly the tile
// ranges, and an atomic scatter of 64-bit (depth bits << 32 | id) keys into the
// tile buckets; the remaining digits are sorted inside each tile's bucket by
// one CTA in shared memory (bitonic; chunked + merged for buckets deeper than
// the shared-memory capacity).  The keys are unique, so the result is the
// ascending (tile, depth bits, id) order bit for bit, whatever order the
// atomics gave.  Three kernels per view (the tile prefix is taken inside the
// scatter), K x 24 B of traffic.
// The file also holds a general LSD radix sort (reduce-then-scan: per-block
// digit histograms, one exclusive scan of the digit-major histogram matrix, a
// stable scatter ranking each warp's 32 items per round with
// __match_any_sync) used by the association.  No kernel waits on another
// block, so nothing can hang on scheduling order.
#include <algorithm>
#include <atomic>
#include <cstdio>

#include "common.cuh"
#include "internal.cuh"
#include "segsort.cuh"

namespace splat {

// ----------------------------------------------------------------------------
// Exclusive scan (uint32), three phases over tiles of 4096 elements.
// ----------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

size_t scan_workspace_size(int64_t n) { return align_up(sizeof(uint32_t) * (size_t)std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile)); }

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n,
                                                                   uint32_t* __restrict__ partials) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  __shared__ uint32_t sh[33];
  uint32_t excl;
  const uint32_t tot = block_excl_scan<kScanThreads>(s, excl, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) scan_partials_kernel(uint32_t* __restrict__ partials, int64_t nparts) {
  __shared__ uint32_t sh[33];
  uint32_t carry = 0;
  for (int64_t base = 0; base < nparts; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const uint32_t x = i < nparts ? partials[i] : 0u;
    uint32_t excl;
    const uint32_t tot = block_excl_scan<1024>(x, excl, sh);
    if (i < nparts) partials[i] = carry + excl;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                                 int64_t n, const uint32_t* __restrict__ partials) {
  __shared__ uint32_t tile[kScanTile];
  __shared__ uint32_t sh[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    tile[k * kScanThreads + threadIdx.x] = i < n ? in[i] : 0u;
  }
  __syncthreads();
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = tile[threadIdx.x * kScanItems + k];
    s += v[k];
  }
  uint32_t excl;
  block_excl_scan<kScanThreads>(s, excl, sh);
  uint32_t run = partials[blockIdx.x] + excl;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    tile[threadIdx.x * kScanItems + k] = run;
    run += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) out[i] = tile[k * kScanThreads + threadIdx.x];
  }
}

int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* ws, cudaStream_t s) {
  if (n <= 0) return SPLAT_OK;
  const int64_t nparts = (n + kScanTile - 1) / kScanTile;
  uint32_t* partials = static_cast<uint32_t*>(ws);
  SPLAT_LAUNCH("scan_reduce_kernel", s, scan_reduce_kernel<<<(unsigned)nparts, kScanThreads, 0, s>>>(in, n, partials));
  SPLAT_LAUNCH("scan_partials_kernel", s, scan_partials_kernel<<<1, 1024, 0, s>>>(partials, nparts));
  SPLAT_LAUNCH("scan_down_kernel", s, scan_down_kernel<<<(unsigned)nparts, kScanThreads, 0, s>>>(in, out, n, partials));
  return check_launch("exclusive_scan_u32");
}

// ----------------------------------------------------------------------------
// Radix sort.
// ----------------------------------------------------------------------------
constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixRounds = 8;  // rounds of 32 items per warp
constexpr int kRadixTile = kRadixThreads * kRadixRounds;  // 2048 items per block
constexpr uint32_t kNoDigit = 0xffffffffu;

static int64_t radix_blocks(int64_t capacity) { return std::max<int64_t>(1, (capacity + kRadixTile - 1) / kRadixTile); }

size_t radix_workspace_size(int64_t capacity) {
  const int64_t nb = radix_blocks(capacity);
  const int64_t cells = 256 * nb;
  return 2 * align_up(sizeof(uint32_t) * cells) + scan_workspace_size(cells);
}

int radix_passes(int begin_bit, int end_bit) { return end_bit > begin_bit ? (end_bit - begin_bit + 7) / 8 : 0; }

__device__ __forceinline__ int64_t valid_count(const int64_t* count_dev, int64_t capacity) {
  if (!count_dev) return capacity;
  const int64_t c = *count_dev;
  return c < capacity ? (c < 0 ? 0 : c) : capacity;
}

template <typename Key>
__global__ void __launch_bounds__(kRadixThreads) radix_hist_kernel(const Key* __restrict__ keys, int64_t capacity,
                                                                   const int64_t* __restrict__ count_dev, int shift,
                                                                   int nbits, uint32_t* __restrict__ counts,
                                                                   int64_t nblocks) {
  __shared__ uint32_t hist[256];
  const int ndig = 1 << nbits;
  for (int d = threadIdx.x; d < ndig; d += kRadixThreads) hist[d] = 0;
  __syncthreads();
  const int64_t n = valid_count(count_dev, capacity);
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  const uint32_t mask = (uint32_t)ndig - 1u;
  for (int k = 0; k < kRadixRounds; ++k) {
    const int64_t i = base + (int64_t)k * kRadixThreads + threadIdx.x;
    if (i < n) atomicAdd(&hist[(uint32_t)(keys[i] >> shift) & mask], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < ndig; d += kRadixThreads) counts[(int64_t)d * nblocks + blockIdx.x] = hist[d];
}

template <typename Key>
__global__ void __launch_bounds__(kRadixThreads) radix_scatter_kernel(
    const Key* __restrict__ kin, const uint32_t* __restrict__ vin, Key* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t capacity, const int64_t* __restrict__ count_dev, int shift, int nbits,
    const uint32_t* __restrict__ offsets, int64_t nblocks) {
  __shared__ uint32_t wcount[kRadixWarps][256];
  __shared__ uint32_t gbase[256];
  const int ndig = 1 << nbits;
  const uint32_t mask = (uint32_t)ndig - 1u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < ndig; d += kRadixThreads) {
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) wcount[w][d] = 0;
    gbase[d] = offsets[(int64_t)d * nblocks + blockIdx.x];
  }
  __syncthreads();
  const int64_t n = valid_count(count_dev, capacity);
  const int64_t wbase = (int64_t)blockIdx.x * kRadixTile + (int64_t)warp * (kRadixRounds * 32);
  const uint32_t lt_mask = (1u << lane) - 1u;
  Key key[kRadixRounds];
  uint32_t val[kRadixRounds];
  uint32_t dig[kRadixRounds];
  uint32_t rank[kRadixRounds];
#pragma unroll
  for (int r = 0; r < kRadixRounds; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const bool ok = i < n;
    key[r] = ok ? kin[i] : Key(0);
    val[r] = (ok && vin) ? vin[i] : 0u;
    dig[r] = ok ? ((uint32_t)(key[r] >> shift) & mask) : kNoDigit;
    const uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
    const uint32_t before = ok ? wcount[warp][dig[r]] : 0u;
    __syncwarp();
    const int leader = __ffs(peers) - 1;
    if (ok && lane == leader) wcount[warp][dig[r]] = before + __popc(peers);
    __syncwarp();
    rank[r] = before + __popc(peers & lt_mask);
  }
  __syncthreads();
  // exclusive prefix of the per-warp counts, digit by digit
  for (int d = threadIdx.x; d < ndig; d += kRadixThreads) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) {
      const uint32_t c = wcount[w][d];
      wcount[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRadixRounds; ++r) {
    if (dig[r] == kNoDigit) continue;
    const uint32_t dst = gbase[dig[r]] + wcount[warp][dig[r]] + rank[r];
    kout[dst] = key[r];
    if (vout) vout[dst] = val[r];
  }
}

template <typename Key>
int radix_sort(Key* keys0, uint32_t* vals0, Key* keys1, uint32_t* vals1, int64_t capacity,
               const int64_t* count_dev, int begin_bit, int end_bit, void* ws, cudaStream_t s,
               int* result_buffer) {
  const int passes = radix_passes(begin_bit, end_bit);
  *result_buffer = passes & 1;
  if (passes == 0 || capacity <= 0) return SPLAT_OK;
  const int bits_per = (end_bit - begin_bit + passes - 1) / passes;
  const int64_t nb = radix_blocks(capacity);
  const int64_t cells = 256 * nb;
  char* w = static_cast<char*>(ws);
  uint32_t* counts = reinterpret_cast<uint32_t*>(w);
  w += align_up(sizeof(uint32_t) * cells);
  uint32_t* offsets = reinterpret_cast<uint32_t*>(w);
  w += align_up(sizeof(uint32_t) * cells);
  void* scan_ws = w;
  Key* kin = keys0;
  Key* kout = keys1;
  uint32_t* vin = vals0;
  uint32_t* vout = vals1;
  int shift = begin_bit;
  for (int p = 0; p < passes; ++p) {
    const int nbits = std::min(bits_per, end_bit - shift);
    const int64_t used = (int64_t)(1 << nbits) * nb;
    SPLAT_LAUNCH("radix_hist_kernel", s, radix_hist_kernel<Key><<<(unsigned)nb, kRadixThreads, 0, s>>>(kin, capacity, count_dev, shift, nbits, counts, nb));
    int rc = exclusive_scan_u32(counts, offsets, used, scan_ws, s);
    if (rc) return rc;
    SPLAT_LAUNCH("radix_scatter_kernel", s, radix_scatter_kernel<Key><<<(unsigned)nb, kRadixThreads, 0, s>>>(kin, vin, kout, vout, capacity, count_dev, shift,
                                                                     nbits, offsets, nb));
    rc = check_launch("radix_scatter_kernel");
    if (rc) return rc;
    std::swap(kin, kout);
    std::swap(vin, vout);
    shift += nbits;
  }
  return SPLAT_OK;
}

template int radix_sort<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*, int64_t, const int64_t*, int, int, void*,
                                  cudaStream_t, int*);
template int radix_sort<uint64_t>(uint64_t*, uint32_t*, uint64_t*, uint32_t*, int64_t, const int64_t*, int, int, void*,
                                  cudaStream_t, int*);

// ----------------------------------------------------------------------------
// Binning: per-tile buckets, then one shared-memory sort per tile.
// ----------------------------------------------------------------------------
constexpr int kSegCap = 2048;        // keys a CTA sorts in shared memory (16 KB per buffer)
constexpr int kSortThreads = 256;
constexpr int kCursorStride = 32;    // one 128-byte line per bucket cursor
constexpr int kDiffStride = 32;      // one 128-byte line per difference-grid cell: the row-end atomics of all
                                     // visible Gaussians spread over the L2 slices instead of a few lines
constexpr int kSmemTiles = 8192;     // tiles whose local counters fit the scatter CTA
constexpr int kScatterThreads = 256;
constexpr int kScatterLanes = 4;     // threads sharing one Gaussian's rect (rows interleaved)
constexpr int kScanGridSmem = 10240; // count-grid cells staged in shared memory (40 KB)

// Tile membership: a tile of the Gaussian's rect holds it only if some point
// of its 16 x 16 rectangle of pixel centres reaches
// opacity * exp(-Q/2) >= 0.99/255, Q = a dx^2 + 2 b dx dy + c dy^2 (below
// 1/255 every pixel skips the Gaussian, so dropping the other tiles changes
// no image).  Q is convex: its minimum over the rectangle is 0 with the centre
// inside, else on an edge, a 1-D quadratic minimised in closed form.  Every
// operation is rounded as written, in the written order (the CPU oracle takes
// the same decision bit for bit).  In each tile row the members run from the
// first to the last tile of the rect row that passes.
constexpr float kTileAlpha = 0.99f / 255.0f;

// Per-Gaussian data of the membership test.  qlo / qhi bracket the Q at which
// opacity * exp(-Q/2) crosses 0.99/255 (from logf, widened by 1e-4 relative +
// 1e-4): below qlo the test certainly passes and above qhi it certainly fails
// (the exponential's error is a few 1e-7), so the exponential is evaluated
// only in between -- the decision is the specified one either way.
struct TileTest {
  float u, v, a, b, c, b2, ra, rc, lam, qlo, qhi;
  float det, ey, dyl;  // a c - b^2; y half-extent and leftmost point's dy of {Q <= qhi}
};

__device__ __forceinline__ TileTest tile_test(const float4 xo, const float4 co) {
  TileTest t;
  t.u = xo.x;
  t.v = xo.y;
  t.lam = xo.w;
  t.a = co.x;
  t.b = co.y;
  t.c = co.z;
  t.b2 = __fmul_rn(2.0f, co.y);
  t.ra = __fdiv_rn(co.y, co.x);
  t.rc = __fdiv_rn(co.y, co.z);
  const float qt = 2.0f * (logf(xo.w) - logf(kTileAlpha));
  const float w = 1e-4f * fabsf(qt) + 1e-4f;
  t.qlo = qt - w;
  t.qhi = qt + w;
  t.det = co.x * co.z - co.y * co.y;
  const float K = fmaxf(t.qhi, 0.0f);
  t.ey = sqrtf(K * co.x / t.det);
  t.dyl = co.y * sqrtf(K / (co.z * t.det));
  return t;
}

// A range of tiles of rect row ty outside which the test certainly fails:
// the tiles whose pixel-centre columns meet the x-extent of {Q <= qhi} within
// the row's band (its leftmost and rightmost points over the band, from the
// closed-form boundary of the ellipse), widened by 1 px + 0.1%.  Scanning from
// its ends finds the same first and last passing tiles as scanning the whole
// rect row.  False when the band certainly misses the ellipse.
__device__ __forceinline__ bool row_candidates(const TileTest& t, const int4 r, int ty, int& xs, int& xe) {
  if (!(t.det > 0.0f) || !(t.ey < 3e38f)) {  // degenerate: scan the whole rect row
    xs = r.x;
    xe = r.z - 1;
    return true;
  }
  const float ya = (float)(kTile * ty) + 0.5f - t.v, yb = ya + 15.0f;
  const float eyw = t.ey * 1.001f + 1.0f;
  if (yb < -eyw || ya > eyw) return false;
  const float lo = fmaxf(ya, -t.ey), hi = fminf(yb, t.ey);
  const float K = fmaxf(t.qhi, 0.0f);
  auto half = [&](float dy) { return sqrtf(fmaxf(0.0f, K * t.a - t.det * dy * dy)) / t.a; };
  const float dl = fminf(hi, fmaxf(lo, t.dyl)), dr = fminf(hi, fmaxf(lo, -t.dyl));
  const float X0 = -t.ra * dl - half(dl), X1 = -t.ra * dr + half(dr);
  const float m = 1.0f + 1e-3f * (fabsf(X0) + fabsf(X1));
  xs = max(r.x, (int)ceilf((t.u + X0 - m - 15.5f) * (1.0f / kTile)));
  xe = min(r.z - 1, (int)floorf((t.u + X1 + m - 0.5f) * (1.0f / kTile)));
  return xs <= xe;
}

__device__ __forceinline__ bool tile_reaches(const TileTest& t, int tx, int ty) {
  const float xa = __fsub_rn(__fadd_rn((float)(kTile * tx), 0.5f), t.u);
  const float xb = __fadd_rn(xa, 15.0f);
  const float ya = __fsub_rn(__fadd_rn((float)(kTile * ty), 0.5f), t.v);
  const float yb = __fadd_rn(ya, 15.0f);
  if (xa <= 0.0f && 0.0f <= xb && ya <= 0.0f && 0.0f <= yb) return true;
  float m = __int_as_float(0x7f800000);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float dy = e ? yb : ya;
    const float dx = fminf(xb, fmaxf(xa, -__fmul_rn(t.ra, dy)));
    const float qh = __fadd_rn(__fmul_rn(__fadd_rn(__fmul_rn(t.a, dx), __fmul_rn(t.b2, dy)), dx),
                               __fmul_rn(__fmul_rn(t.c, dy), dy));
    m = fminf(m, qh);
    const float ex = e ? xb : xa;
    const float ey = fminf(yb, fmaxf(ya, -__fmul_rn(t.rc, ex)));
    const float qv = __fadd_rn(__fmul_rn(__fmul_rn(t.a, ex), ex),
                               __fmul_rn(__fadd_rn(__fmul_rn(t.b2, ex), __fmul_rn(t.c, ey)), ey));
    m = fminf(m, qv);
  }
  if (m < t.qlo) return true;
  if (m > t.qhi) return false;
  return __fmul_rn(t.lam, exp_full(__fmul_rn(-0.5f, m))) >= kTileAlpha;
}

// Member tiles [x0, x1] of rect row ty (the first and last passing tiles);
// false for an empty row.
__device__ __forceinline__ bool row_members(const TileTest& t, const int4 r, int ty, int& x0, int& x1) {
  int xs, xe;
  if (!row_candidates(t, r, ty, xs, xe)) return false;
  x0 = xs;
  while (x0 <= xe && !tile_reaches(t, x0, ty)) ++x0;
  if (x0 > xe) return false;
  x1 = xe;
  while (x1 > x0 && !tile_reaches(t, x1, ty)) --x1;
  return true;
}

// Visible Gaussians (tiles_touched > 0, a non-empty rect) are appended to
// vis[] with one atomic per warp.  A warp takes 128 consecutive Gaussians (4
// per lane, coalesced), packs its visible ones into slots in shared memory
// (one lane per slot then loads the rect and prepares the membership test),
// and then takes the rect rows of all its slots, one row per lane: the row's member tiles enter the tile counts as
// +1 / -1 at its ends in a per-row difference array (prefix sums along the
// rows in tile_scan_kernel give the counts), the duplicate total K is summed
// (one 64-bit atomic per warp), and the row's span is kept for the scatter: one
// 16-bit word per rect row (first and last member as offsets from the rect's
// left column; 0x00ff for an empty row) in a region reserved with one atomic
// per warp.  A Gaussian whose rect is wider than 255 tiles, or whose rows do
// not fit the span buffer, gets no spans (vspan = ~0) and the scatter tests its
// tiles again.
constexpr uint32_t kNoSpan = 0xffffffffu;
constexpr uint16_t kEmptySpan = 0x00ff;
constexpr int kCcWarps = 4;                // warps per CTA
constexpr int kCcPer = 4;                  // Gaussians per lane
constexpr int kCcSlots = 32 * kCcPer;      // Gaussians per warp
constexpr int kCcThreads = 32 * kCcWarps;

__global__ void __launch_bounds__(kCcThreads) compact_count_kernel(
    const int32_t* __restrict__ tiles, const int4* __restrict__ rect, const float4* __restrict__ xyzo,
    const float4* __restrict__ conic, int64_t n, int gw, uint32_t* __restrict__ vis, unsigned int* __restrict__ n_vis,
    unsigned long long* __restrict__ k_total, int* __restrict__ diff, uint16_t* __restrict__ spans, uint64_t span_cap,
    unsigned long long* __restrict__ span_top, uint32_t* __restrict__ vspan) {
  __shared__ TileTest s_tt[kCcWarps][kCcSlots];
  __shared__ int4 s_rect[kCcWarps][kCcSlots];
  __shared__ uint32_t s_row0[kCcWarps][kCcSlots + 1];  // exclusive prefix of the slots' rect heights
  __shared__ uint32_t s_hx[kCcWarps][kCcSlots];        // exclusive prefix of the span heights, or kNoSpan
  __shared__ uint32_t s_gid[kCcWarps][kCcSlots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned full = 0xffffffffu, lower = (1u << lane) - 1u;
  const int64_t w0 = ((int64_t)blockIdx.x * kCcWarps + warp) * kCcSlots;
  int tt[kCcPer];
#pragma unroll
  for (int k = 0; k < kCcPer; ++k) {
    const int64_t i = w0 + 32 * k + lane;
    tt[k] = i < n ? tiles[i] : 0;
  }
  int nvw = 0;
#pragma unroll
  for (int k = 0; k < kCcPer; ++k) {
    const unsigned b = __ballot_sync(full, tt[k] > 0);
    if (tt[k] > 0) s_gid[warp][nvw + __popc(b & lower)] = (uint32_t)(w0 + 32 * k + lane);
    nvw += __popc(b);
  }
  __syncwarp();
  for (int sl = lane; sl < nvw; sl += 32) {
    const uint32_t i = s_gid[warp][sl];
    s_rect[warp][sl] = rect[i];
    s_tt[warp][sl] = tile_test(xyzo[i], conic[i]);
  }
  __syncwarp();
  // exclusive prefixes over the slots of the rect heights (rows) and of the
  // span heights (0 for a rect wider than 255 tiles)
  uint32_t cr = 0, ch = 0;
  for (int c = 0; c < nvw; c += 32) {
    const int sl = c + lane;
    const int4 r = sl < nvw ? s_rect[warp][sl] : make_int4(0, 0, 0, 0);
    const uint32_t hr = (uint32_t)(r.w - r.y);
    const uint32_t h = r.z - r.x <= 255 ? hr : 0u;
    uint32_t xr = hr, xh = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t yr = __shfl_up_sync(full, xr, o), yh = __shfl_up_sync(full, xh, o);
      if (lane >= o) {
        xr += yr;
        xh += yh;
      }
    }
    if (sl < nvw) {
      s_row0[warp][sl] = cr + xr - hr;
      s_hx[warp][sl] = h ? ch + xh - h : kNoSpan;
    }
    cr += __shfl_sync(full, xr, 31);
    ch += __shfl_sync(full, xh, 31);
  }
  if (lane == 0) s_row0[warp][nvw] = cr;
  unsigned long long sbase = 0;
  unsigned int base = 0;
  if (lane == 0 && ch) sbase = atomicAdd(span_top, (unsigned long long)ch);
  if (lane == 0 && nvw) base = atomicAdd(n_vis, (unsigned)nvw);
  sbase = __shfl_sync(full, sbase, 0);
  base = __shfl_sync(full, base, 0);
  const bool fits = sbase + ch <= span_cap && sbase + ch < (unsigned long long)kNoSpan;
  __syncwarp();
  unsigned long long t = 0;
  for (uint32_t q = lane; q < cr; q += 32) {
    int lo = 0, hi = nvw - 1;  // the last slot whose first row is <= q
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_row0[warp][mid] <= q) lo = mid; else hi = mid - 1;
    }
    while (s_row0[warp][lo + 1] <= q) ++lo;  // slots without rows share a prefix (sentinel at nvw)
    const int4 r = s_rect[warp][lo];
    const int ty = r.y + (int)(q - s_row0[warp][lo]);
    const uint32_t hx = s_hx[warp][lo];
    int x0, x1;
    const bool any = row_members(s_tt[warp][lo], r, ty, x0, x1);
    if (hx != kNoSpan && fits)
      spans[(size_t)(sbase + hx) + (ty - r.y)] = any ? (uint16_t)((x0 - r.x) | ((x1 - r.x) << 8)) : kEmptySpan;
    if (!any) continue;
    atomicAdd(&diff[(size_t)(ty * gw + x0) * kDiffStride], 1);
    atomicAdd(&diff[(size_t)(ty * gw + x1 + 1) * kDiffStride], -1);
    t += (unsigned long long)(x1 - x0 + 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(full, t, o);
  if (lane == 0 && t) atomicAdd(k_total, t);
  for (int sl = lane; sl < nvw; sl += 32) {
    vis[base + sl] = s_gid[warp][sl];
    const uint32_t hx = s_hx[warp][sl];
    vspan[base + sl] = (hx != kNoSpan && fits) ? (uint32_t)(sbase + hx) : kNoSpan;
  }
}

// Member tiles of rect row ty from the kept span, or by testing again.
__device__ __forceinline__ bool row_span(const uint16_t* __restrict__ spans, uint32_t sb, const float4 xo,
                                         const float4 co, const int4 r, int ty, int& x0, int& x1) {
  if (sb != kNoSpan) {
    const uint16_t w = spans[(size_t)sb + (ty - r.y)];
    x0 = r.x + (w & 0xff);
    x1 = r.x + (w >> 8);
    return x0 <= x1;
  }
  return row_members(tile_test(xo, co), r, ty, x0, x1);
}

// A tile schedule's order from its costs (one CTA, any multiple of 32
// threads): a counting sort over the cost buckets, heaviest bucket first; the
// order within a bucket is that of the atomics.  Every thread takes part.
__device__ void build_tile_order(uint32_t* __restrict__ schedule, int n_tiles) {
  __shared__ uint32_t s_cnt[kCostBuckets];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t* cost = schedule + 1 + n_tiles;
  uint32_t* order = schedule + 1;
  for (int b = threadIdx.x; b < kCostBuckets; b += blockDim.x) s_cnt[b] = 0u;
  __syncthreads();
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) atomicAdd(&s_cnt[tile_cost_bucket(cost[t])], 1u);
  __syncthreads();
  if (wid == 0) {  // bucket cursors, heaviest bucket first: lane l takes buckets 127 - 4 l - j
    uint32_t c[4], tot = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      c[j] = s_cnt[kCostBuckets - 1 - 4 * lane - j];
      tot += c[j];
    }
    uint32_t run = warp_incl_scan(tot, lane) - tot;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      s_cnt[kCostBuckets - 1 - 4 * lane - j] = run;
      run += c[j];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x)
    order[atomicAdd(&s_cnt[tile_cost_bucket(cost[t])], 1u)] = (uint32_t)t;
  __syncthreads();
  if (threadIdx.x == 0) schedule[0] = (uint32_t)n_tiles;
}

__global__ void __launch_bounds__(1024) tile_order_kernel(uint32_t* __restrict__ schedule, int n_tiles) {
  build_tile_order(schedule, n_tiles);
}

// One CTA: prefix sums along the rows of the difference grid (gw = tiles_x + 1
// cells per row, kDiffStride ints apart) -> per-tile counts; exclusive scan over tiles -> ranges
// (clamped to the capacity) and bucket cursors; K and the status; with a
// tile schedule, its order (heaviest first) rebuilt from the per-tile costs
// the last forward render left (a counting sort over the cost buckets).
__global__ void __launch_bounds__(1024) tile_scan_kernel(int* __restrict__ diff, int tiles_x, int tiles_y,
                                                         const unsigned long long* __restrict__ k_total,
                                                         int64_t capacity, uint2* __restrict__ ranges,
                                                         uint32_t* __restrict__ cursor, int64_t* __restrict__ k_dev,
                                                         int32_t* __restrict__ status, uint32_t* __restrict__ schedule) {
  __shared__ uint32_t sh[33];
  __shared__ int s_grid[kScanGridSmem];
  const int gw = tiles_x + 1;
  const int cells = gw * tiles_y;
  // prefix sums in shared memory when they fit, else in place (strided)
  const bool in_smem = cells <= kScanGridSmem;
  int* grid = in_smem ? s_grid : diff;
  const int gs = in_smem ? 1 : kDiffStride;
  if (in_smem)
    for (int i = threadIdx.x; i < cells; i += blockDim.x) s_grid[i] = diff[(size_t)i * kDiffStride];
  __syncthreads();
  // prefix sums along each row (one warp per row, 32 cells per warp scan;
  // two's-complement sums, so the negative entries need no special care)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int y = wid; y < tiles_y; y += nw) {
    uint32_t carry = 0;
    for (int x0 = 0; x0 < tiles_x; x0 += 32) {
      const int x = x0 + lane;
      const uint32_t v = warp_incl_scan(x < tiles_x ? (uint32_t)grid[(size_t)(y * gw + x) * gs] : 0u, lane) + carry;
      if (x < tiles_x) grid[(size_t)(y * gw + x) * gs] = (int)v;
      carry = __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  const int n_tiles = tiles_x * tiles_y;
  const uint64_t cap = (uint64_t)capacity;
  uint32_t carry = 0;
  for (int base = 0; base < n_tiles; base += 1024) {
    const int t = base + threadIdx.x;
    const uint32_t c = t < n_tiles ? (uint32_t)grid[(size_t)((t / tiles_x) * gw + (t % tiles_x)) * gs] : 0u;
    uint32_t excl;
    const uint32_t tot = block_excl_scan<1024>(c, excl, sh);
    if (t < n_tiles) {
      const uint64_t st = (uint64_t)carry + excl;
      const uint64_t en = st + c;
      ranges[t] = c ? make_uint2((uint32_t)(st < cap ? st : cap), (uint32_t)(en < cap ? en : cap)) : make_uint2(0u, 0u);
      cursor[(size_t)t * kCursorStride] = (uint32_t)st;
    }
    carry += tot;
  }
  if (threadIdx.x == 0) {
    const int64_t k = (int64_t)*k_total;
    *k_dev = k;
    if (k > capacity) raise_status(status, SPLAT_ECAPACITY);
  }
  if (schedule) {
    __syncthreads();
    build_tile_order(schedule, n_tiles);
  }
}

// 4-byte asynchronous copy global -> shared (cp.async): the scatter stages
// the difference grid while it counts.
__device__ __forceinline__ void cp_async_i32(int* smem, const int* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(g) : "memory");
}

// Every visible Gaussian drops key (depth bits << 32 | id) into the bucket of
// each of its member tiles.  A CTA takes a contiguous slice of the visible list,
// counts its duplicates per tile in shared memory (kScatterLanes threads per
// rect, rows interleaved), reserves space in each touched bucket with one
// global atomic for the whole slice, then places its keys with shared-memory
// atomics.  The order inside a bucket is arbitrary; the keys are unique, so
// the per-tile sort below makes the result deterministic.
// With the tile grid in shared memory (n_tiles <= kSmemTiles) every CTA also
// takes the tile prefix itself, in place of a scan launch before it: the row
// prefix sums of the difference grid (staged by cp.async while the CTA
// counts) are the tile counts, their exclusive scan in tile order the bucket
// starts, and the cursors (zeroed with the grid) count from 0 inside each
// bucket.  CTA 0 writes the tile ranges, the duplicate total and the capacity
// status, as tile_scan_kernel does on the other path, where the cursors hold
// the bucket starts.
__global__ void __launch_bounds__(kScatterThreads) bucket_scatter_kernel(
    const uint32_t* __restrict__ vis, const unsigned int* __restrict__ n_vis, const float4* __restrict__ xyzo,
    const float4* __restrict__ conic, const int4* __restrict__ rect, const uint16_t* __restrict__ spans,
    const uint32_t* __restrict__ vspan, int tiles_x, int tiles_y, int n_tiles, uint32_t* __restrict__ cursor,
    int64_t capacity, uint64_t* __restrict__ skeys, const int* __restrict__ diff,
    const unsigned long long* __restrict__ k_total, uint2* __restrict__ ranges, int64_t* __restrict__ k_dev,
    int32_t* __restrict__ status) {
  extern __shared__ uint32_t s_cnt[];  // [n_tiles] local counts, then local cursors
  uint32_t* s_base = s_cnt + n_tiles;  // [n_tiles] tile counts, then the bucket positions reserved
  int* s_grid = reinterpret_cast<int*>(s_base + n_tiles);  // [(tiles_x + 1) tiles_y] the difference grid
  __shared__ uint32_t s_sh[33];
  constexpr int kChunk = kScatterThreads / kScatterLanes;  // Gaussians per round
  const unsigned int nv = *n_vis;
  const int sub = threadIdx.x % kScatterLanes;  // this thread takes rect rows ty = y0 + sub (mod kScatterLanes)
  if (n_tiles > kSmemTiles) {  // too many tiles for shared memory: one global atomic per duplicate
    for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < nv; c0 += (int64_t)gridDim.x * kChunk) {
      const int64_t i = c0 + threadIdx.x / kScatterLanes;
      if (i >= nv) continue;
      const uint32_t g = vis[i];
      const int4 r = rect[g];
      const float4 xo = xyzo[g], co = conic[g];
      const uint32_t sb = vspan[i];
      const uint64_t key = ((uint64_t)__float_as_uint(xo.z) << 32) | (uint64_t)g;
      for (int ty = r.y + sub; ty < r.w; ty += kScatterLanes) {
        int x0, x1;
        if (!row_span(spans, sb, xo, co, r, ty, x0, x1)) continue;
        for (int tx = x0; tx <= x1; ++tx) {
          const uint32_t pos = atomicAdd(&cursor[(size_t)(ty * tiles_x + tx) * kCursorStride], 1u);
          if (pos < capacity) skeys[pos] = key;
        }
      }
    }
    return;
  }
  const int gw = tiles_x + 1, cells = gw * tiles_y;
  for (int i = threadIdx.x; i < cells; i += kScatterThreads) cp_async_i32(s_grid + i, diff + (size_t)i * kDiffStride);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  const int64_t per = ((int64_t)nv + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < (int64_t)nv ? lo + per : (int64_t)nv;
  for (int t = threadIdx.x; t < n_tiles; t += kScatterThreads) s_cnt[t] = 0u;
  __syncthreads();
  for (int64_t c0 = lo; c0 < hi; c0 += kChunk) {  // count
    const int64_t i = c0 + threadIdx.x / kScatterLanes;
    if (i >= hi) continue;
    const uint32_t g = vis[i];
    const int4 r = rect[g];
    const uint32_t sb = vspan[i];
    const float4 xo = sb == kNoSpan ? xyzo[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 co = sb == kNoSpan ? conic[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int ty = r.y + sub; ty < r.w; ty += kScatterLanes) {
      int x0, x1;
      if (!row_span(spans, sb, xo, co, r, ty, x0, x1)) continue;
      for (int tx = x0; tx <= x1; ++tx) atomicAdd(&s_cnt[ty * tiles_x + tx], 1u);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  {  // row prefix sums of the difference grid: the tile counts (two's-complement sums)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int y = wid; y < tiles_y; y += kScatterThreads / 32) {
      uint32_t carry = 0;
      for (int x0 = 0; x0 < tiles_x; x0 += 32) {
        const int x = x0 + lane;
        const uint32_t v = warp_incl_scan(x < tiles_x ? (uint32_t)s_grid[y * gw + x] : 0u, lane) + carry;
        if (x < tiles_x) s_base[y * tiles_x + x] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
      }
    }
  }
  __syncthreads();
  // bucket starts: exclusive scan in tile order, thread k taking a run of
  // consecutive tiles; then the reservation of this CTA's share of each bucket
  const int run_len = (n_tiles + kScatterThreads - 1) / kScatterThreads;
  const int t0 = min(n_tiles, (int)threadIdx.x * run_len), t1 = min(n_tiles, t0 + run_len);
  uint32_t part = 0;
  for (int t = t0; t < t1; ++t) part += s_base[t];
  uint32_t run;
  block_excl_scan<kScatterThreads>(part, run, s_sh);
  const uint64_t cap = (uint64_t)capacity;
  for (int t = t0; t < t1; ++t) {  // reserve
    const uint32_t c = s_base[t], mine = s_cnt[t];
    if (blockIdx.x == 0) {
      const uint64_t st = run, en = st + c;
      ranges[t] = c ? make_uint2((uint32_t)(st < cap ? st : cap), (uint32_t)(en < cap ? en : cap)) : make_uint2(0u, 0u);
    }
    s_base[t] = run + (mine ? atomicAdd(&cursor[(size_t)t * kCursorStride], mine) : 0u);
    s_cnt[t] = 0u;
    run += c;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t k = (int64_t)*k_total;
    *k_dev = k;
    if (k > capacity) raise_status(status, SPLAT_ECAPACITY);
  }
  __syncthreads();
  for (int64_t c0 = lo; c0 < hi; c0 += kChunk) {  // place
    const int64_t i = c0 + threadIdx.x / kScatterLanes;
    if (i >= hi) continue;
    const uint32_t g = vis[i];
    const int4 r = rect[g];
    const float4 xo = xyzo[g];
    const uint32_t sb = vspan[i];
    const float4 co = sb == kNoSpan ? conic[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint64_t key = ((uint64_t)__float_as_uint(xo.z) << 32) | (uint64_t)g;
    for (int ty = r.y + sub; ty < r.w; ty += kScatterLanes) {
      int x0, x1;
      if (!row_span(spans, sb, xo, co, r, ty, x0, x1)) continue;
      for (int tx = x0; tx <= x1; ++tx) {
        const int t = ty * tiles_x + tx;
        const uint32_t pos = s_base[t] + atomicAdd(&s_cnt[t], 1u);
        if (pos < capacity) skeys[pos] = key;
      }
    }
  }
}

// One CTA per tile: sort its bucket ascending by (depth bits, id) and write
// the ids (and optionally the (tile, depth) keys).  Buckets of up to 32 keys
// are bitonic-sorted; longer ones are bucket-sorted on the depth range in
// shared memory, or radix-sorted when the depths cluster (chunks of kSegCap
// keys, merged in global memory above that).  Dynamic
// shared memory: two key buffers of kSegCap, 8 x 256 digit counters, scan
// scratch.
// Shared memory of a tile sort with CAP keys per shared-memory pass.
template <int CAP>
constexpr size_t sort_smem_bytes() {
  return 2 * sizeof(uint64_t) * CAP + sizeof(uint32_t) * (kSegRadixWarps * 256 + 64);
}
constexpr int kSortBitonicMax = 32;

template <int CAP>
__global__ void __launch_bounds__(kSortThreads) tile_sort_kernel(const uint2* __restrict__ ranges,
                                                                 uint64_t* __restrict__ skeys,
                                                                 uint64_t* __restrict__ skeys2,
                                                                 uint32_t* __restrict__ vals,
                                                                 uint64_t* __restrict__ keys_out) {
  extern __shared__ __align__(16) unsigned char sort_smem[];
  uint64_t* bufa = reinterpret_cast<uint64_t*>(sort_smem);
  uint64_t* bufb = bufa + CAP;
  uint32_t* cnt = reinterpret_cast<uint32_t*>(bufb + CAP);
  uint32_t* sh = cnt + kSegRadixWarps * 256;
  const int tile = blockIdx.x;
  const uint2 rg = ranges[tile];
  const int n = (int)(rg.y - rg.x);
  if (n <= 0) return;
  auto sort_chunk = [&](const uint64_t* src, int m) -> const uint64_t* {
    if (m <= kSortBitonicMax) {
      cta_sort_small(src, m, bufa);
      return bufa;
    }
    for (int i = threadIdx.x; i < m; i += kSortThreads) bufa[i] = src[i];
    __syncthreads();
    if (uint64_t* r = cta_bucket_sort_hi32(bufa, bufb, m, cnt, sh)) return r;
    return cta_radix_sort_hi32(bufa, bufb, m, cnt, sh);
  };
  const uint64_t* sorted;
  if (n <= CAP) {
    sorted = sort_chunk(skeys + rg.x, n);
  } else {
    cta_sort_segment_with(skeys + rg.x, skeys2 + rg.x, skeys + rg.x, n, CAP, sort_chunk);
    sorted = skeys2 + rg.x;
  }
  const uint64_t thi = (uint64_t)tile << 32;
  for (int i = threadIdx.x; i < n; i += kSortThreads) {
    const uint64_t k = sorted[i];
    vals[rg.x + i] = (uint32_t)k;
    if (keys_out) keys_out[rg.x + i] = thi | (k >> 32);
  }
}

// ----------------------------------------------------------------------------
// Workspace layout and the entry point.
// ----------------------------------------------------------------------------
struct BinWs {
  uint32_t *vis, *vspan, *cursor;
  int* diff;
  uint64_t *skeys, *skeys2;  // skeys2 also holds the row spans until the tile sort
  unsigned long long *k_total, *span_top;
  unsigned int* n_vis;
};

static size_t carve_bin_ws(int64_t n, int64_t tiles_x, int64_t tiles_y, int64_t capacity, char* base, BinWs* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  const size_t nn = (size_t)std::max<int64_t>(n, 1), cc = (size_t)std::max<int64_t>(capacity, 1);
  const size_t nt = (size_t)std::max<int64_t>(tiles_x * tiles_y, 1);
  BinWs t;
  t.vis = (uint32_t*)take(4 * nn);
  t.vspan = (uint32_t*)take(4 * nn);
  t.cursor = (uint32_t*)take(4 * kCursorStride * nt);
  // the difference grid and the three counters are contiguous: one memset clears them
  t.diff = (int*)take(4 * (size_t)kDiffStride * (tiles_x + 1) * (tiles_y + 1));
  t.k_total = (unsigned long long*)take(8);
  t.span_top = (unsigned long long*)take(8);
  t.n_vis = (unsigned int*)take(8);
  t.skeys = (uint64_t*)take(8 * cc);
  t.skeys2 = (uint64_t*)take(8 * cc);
  if (w) *w = t;
  return off;
}

}  // namespace splat

using namespace splat;

// The workspace depends on the tile grid (w + 1)(h + 1) cells of the count
// grid); with only the tile count known, size it for a 1 x n_tiles grid, which
// bounds (w + 1)(h + 1) = n_tiles + w + h + 1 <= 2 n_tiles + 2 for any w h = n_tiles.
extern "C" size_t splat_bin_sort_workspace_size(int64_t n, int64_t capacity, int32_t n_tiles) {
  if (n < 0 || capacity < 0 || n_tiles < 1) return 0;
  return carve_bin_ws(n, n_tiles, 1, capacity, nullptr, nullptr);
}

extern "C" int splat_tile_schedule_order(uint32_t* schedule, int32_t n_tiles, splat_stream_t stream) {
  if (!schedule || n_tiles < 1) return fail(SPLAT_EINVAL, "splat_tile_schedule_order: bad argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SPLAT_LAUNCH("tile_order_kernel", s, tile_order_kernel<<<1, 1024, 0, s>>>(schedule, n_tiles));
  return check_launch("tile_order_kernel");
}

extern "C" int splat_bin_sort(const splat_projected* proj, int64_t n, const splat_camera* cam, uint64_t* keys,
                              uint32_t* vals, int64_t capacity, int64_t* k_dev, uint32_t* ranges, uint32_t* schedule,
                              int32_t* status, void* ws, size_t ws_bytes, splat_stream_t stream) {
  if (!proj || !cam || !vals || !k_dev || !ranges || !status || !ws)
    return fail(SPLAT_EINVAL, "splat_bin_sort: null argument");
  if (n < 0 || n > 0x7fffffff || capacity < 0 || capacity > 0x7fffffff)
    return fail(SPLAT_EINVAL, "splat_bin_sort: n=%lld capacity=%lld out of range", (long long)n, (long long)capacity);
  if (cam->width <= 0 || cam->height <= 0) return fail(SPLAT_EINVAL, "splat_bin_sort: bad image size");
  if (n > 0 && (!proj->xyzo || !proj->conic || !proj->rect || !proj->tiles_touched || !aligned16(proj->xyzo) ||
                !aligned16(proj->conic) || !aligned16(proj->rect)))
    return fail(SPLAT_EINVAL, "splat_bin_sort: projected arrays null or not 16-byte aligned");
  const CamK ck = make_camk(*cam);
  const int64_t n_tiles = (int64_t)ck.tiles_x * ck.tiles_y;
  const size_t need = carve_bin_ws(n, ck.tiles_x, ck.tiles_y, capacity, nullptr, nullptr);
  if (ws_bytes < need || !aligned16(ws) || !aligned16(ranges))
    return fail(SPLAT_EINVAL, "splat_bin_sort: workspace %zu < %zu bytes, or ws/ranges misaligned", ws_bytes, need);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  BinWs w;
  carve_bin_ws(n, ck.tiles_x, ck.tiles_y, capacity, static_cast<char*>(ws), &w);
  const bool local = n_tiles <= kSmemTiles;
  // local counts, bucket positions and the difference grid ((w + 1) h <= 2 n_tiles cells)
  const size_t scatter_smem =
      local ? sizeof(uint32_t) * (size_t)(2 * n_tiles + (int64_t)(ck.tiles_x + 1) * ck.tiles_y) : 0;
  if (scatter_smem > 48 * 1024) {  // more than the default: opt in once per device
    static std::atomic<unsigned long long> attr_done{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(SPLAT_ECUDA, "splat_bin_sort: no current device");
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_done.load() & bit)) {
      if (cudaFuncSetAttribute(bucket_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(4 * sizeof(uint32_t) * kSmemTiles)) != cudaSuccess)
        return fail(SPLAT_ECUDA, "splat_bin_sort: cannot enable shared memory for the scatter");
      attr_done.fetch_or(bit);
    }
  }
  // the cursors, the difference grid and the three counters
  const size_t clear_bytes = (size_t)(reinterpret_cast<char*>(w.n_vis) - reinterpret_cast<char*>(w.cursor)) + 8;
  if (cudaMemsetAsync(w.cursor, 0, clear_bytes, s) != cudaSuccess)
    return fail(SPLAT_ECUDA, "splat_bin_sort: memset failed");
  const float4* xyzo = reinterpret_cast<const float4*>(proj->xyzo);
  const int4* rect = reinterpret_cast<const int4*>(proj->rect);
  const float4* conic = reinterpret_cast<const float4*>(proj->conic);
  const int nb = std::max(1, ceil_div(n, kCcWarps * kCcSlots));
  if (n > 0)
    SPLAT_LAUNCH("compact_count_kernel", s,
                 compact_count_kernel<<<nb, kCcThreads, 0, s>>>(proj->tiles_touched, rect, xyzo, conic, n, ck.tiles_x + 1,
                                                         w.vis, w.n_vis, w.k_total, w.diff,
                                                         reinterpret_cast<uint16_t*>(w.skeys2),
                                                         4 * (uint64_t)std::max<int64_t>(capacity, 1), w.span_top,
                                                         w.vspan));
  int rc = SPLAT_OK;
  if (!local || n == 0 || capacity == 0) {  // a scan launch: ranges, cursors (bucket starts), the total
    SPLAT_LAUNCH("tile_scan_kernel", s,
                 tile_scan_kernel<<<1, 1024, 0, s>>>(w.diff, ck.tiles_x, ck.tiles_y, w.k_total, capacity,
                                                     reinterpret_cast<uint2*>(ranges), w.cursor, k_dev, status,
                                                     schedule));
    rc = check_launch("tile_scan_kernel");
    if (rc || n == 0 || capacity == 0) return rc;
  } else if (schedule) {  // the scatter takes the prefix; the schedule's order by its own launch
    SPLAT_LAUNCH("tile_order_kernel", s, tile_order_kernel<<<1, 1024, 0, s>>>(schedule, (int32_t)n_tiles));
    if ((rc = check_launch("tile_order_kernel"))) return rc;
  }
  int sms = 152;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int sgrid = std::max(1, std::min(ceil_div(n, kScatterThreads / kScatterLanes), 2 * sms));
  SPLAT_LAUNCH("bucket_scatter_kernel", s,
               bucket_scatter_kernel<<<sgrid, kScatterThreads, scatter_smem, s>>>(
                   w.vis, w.n_vis, xyzo, conic, rect, reinterpret_cast<const uint16_t*>(w.skeys2), w.vspan,
                   ck.tiles_x, ck.tiles_y, (int)n_tiles, w.cursor, capacity, w.skeys, w.diff, w.k_total,
                   reinterpret_cast<uint2*>(ranges), k_dev, status));
  if ((rc = check_launch("bucket_scatter_kernel"))) return rc;
  {
    static std::atomic<unsigned long long> sort_attr_done{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(SPLAT_ECUDA, "splat_bin_sort: no current device");
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(sort_attr_done.load() & bit)) {
      if (cudaFuncSetAttribute(tile_sort_kernel<kSegCap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sort_smem_bytes<kSegCap>()) != cudaSuccess)
        return fail(SPLAT_ECUDA, "splat_bin_sort: cannot enable shared memory for the tile sort");
      sort_attr_done.fetch_or(bit);
    }
  }
  SPLAT_LAUNCH("tile_sort_kernel", s,
               tile_sort_kernel<kSegCap><<<(unsigned)n_tiles, kSortThreads, sort_smem_bytes<kSegCap>(), s>>>(
                   reinterpret_cast<const uint2*>(ranges), w.skeys, w.skeys2, vals, keys));
  return check_launch("tile_sort_kernel");
}
