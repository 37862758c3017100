// binsort.cu -- tile binning and (tile, depth) ordering of the Gaussians
// (the front-to-back order that the rendering equation of Sec. 3.3
// composites in, per 16x16 tile), plus the device-wide scan and radix sort
// primitives the library uses.
//
// Design.  Sorting K (tile, depth, id) duplicates with 64-bit keys would need
// ~6 radix passes over 12 B items.  Instead:
//   1. the N Gaussians are radix-sorted once by the bit pattern of their depth
//      (4 passes over N, stable, so equal depths keep ascending id);
//   2. duplicates are emitted in that depth order, each carrying only its tile
//      id and Gaussian id;
//   3. a stable radix sort on the tile id alone (ceil(log2 n_tiles) bits: 2
//      passes for up to 65536 tiles) then leaves every tile's list in
//      ascending (depth, id) order -- the same order as a sort of the full
//      (tile, depth bits, id) key, bit for bit;
//   4. tile ranges are the boundaries of equal tile ids.
// The radix sort is LSD, reduce-then-scan: a per-block digit histogram, one
// exclusive scan of the digit-major histogram matrix, and a stable scatter in
// which each warp ranks its 32 items per round with __match_any_sync.  No
// kernel waits on another block, so nothing can hang on scheduling order.
#include <algorithm>
#include <cstdio>

#include "common.cuh"
#include "internal.cuh"

namespace splat {

// ----------------------------------------------------------------------------
// Exclusive scan (uint32), three phases over tiles of 4096 elements.
// ----------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

size_t scan_workspace_size(int64_t n) { return align_up(sizeof(uint32_t) * (size_t)std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile)); }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t& excl, uint32_t* sh /*[32]*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_scan(x, lane);
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < NT / 32 ? sh[lane] : 0u;
    const uint32_t wi = warp_incl_scan(w, lane);
    sh[lane] = wi - w;
    if (lane == 31) sh[32] = wi;
  }
  __syncthreads();
  excl = sh[warp] + inc - x;
  const uint32_t total = sh[32];
  __syncthreads();
  return total;
}

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
// Binning kernels.
// ----------------------------------------------------------------------------
__global__ void depth_keys_kernel(const float4* __restrict__ xyzo, const int32_t* __restrict__ tiles, int64_t n,
                                  uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                  unsigned long long* __restrict__ k_total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long t = 0;
  if (i < n) {
    const int tt = tiles[i];
    keys[i] = tt > 0 ? __float_as_uint(xyzo[i].z) : 0xffffffffu;
    vals[i] = (uint32_t)i;
    t = (unsigned long long)(tt > 0 ? tt : 0);
  }
  // 64-bit duplicate total
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0 && t) atomicAdd(k_total, t);
}

__global__ void gather_counts_kernel(const uint32_t* __restrict__ order, const int32_t* __restrict__ tiles, int64_t n,
                                     uint32_t* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cnt[i] = (uint32_t)tiles[order[i]];
}

__global__ void finalize_count_kernel(const unsigned long long* __restrict__ k_total, int64_t capacity,
                                      int64_t* __restrict__ k_dev, int64_t* __restrict__ cnt_dev,
                                      int32_t* __restrict__ status) {
  const int64_t k = (int64_t)*k_total;
  *k_dev = k;
  *cnt_dev = k < capacity ? k : capacity;
  if (k > capacity) raise_status(status, SPLAT_ECAPACITY);
}

// One thread per Gaussian in depth order writes (tile id, Gaussian id) for
// every tile of its rect, row-major.
__global__ void emit_kernel(const uint32_t* __restrict__ order, const uint32_t* __restrict__ cnt,
                            const uint32_t* __restrict__ offs, const int4* __restrict__ rect, int64_t n,
                            int tiles_x, int64_t capacity, uint32_t* __restrict__ tkey,
                            uint32_t* __restrict__ tval) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cnt[i] == 0) return;
  const uint32_t g = order[i];
  const int4 r = rect[g];
  int64_t o = offs[i];
  for (int ty = r.y; ty < r.w; ++ty)
    for (int tx = r.x; tx < r.z; ++tx, ++o)
      if (o < capacity) {
        tkey[o] = (uint32_t)(ty * tiles_x + tx);
        tval[o] = g;
      }
}

__global__ void ranges_kernel(const uint32_t* __restrict__ tkey, const int64_t* __restrict__ cnt_dev,
                              int64_t capacity, uint32_t* __restrict__ ranges) {
  const int64_t n = valid_count(cnt_dev, capacity);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t t = tkey[i];
  if (i == 0 || tkey[i - 1] != t) ranges[2 * (int64_t)t] = (uint32_t)i;
  if (i == n - 1 || tkey[i + 1] != t) ranges[2 * (int64_t)t + 1] = (uint32_t)(i + 1);
}

__global__ void full_keys_kernel(const uint32_t* __restrict__ tkey, const uint32_t* __restrict__ vals,
                                 const float4* __restrict__ xyzo, const int64_t* __restrict__ cnt_dev,
                                 int64_t capacity, uint64_t* __restrict__ keys) {
  const int64_t n = valid_count(cnt_dev, capacity);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = ((uint64_t)tkey[i] << 32) | (uint64_t)__float_as_uint(xyzo[vals[i]].z);
}

// ----------------------------------------------------------------------------
// Workspace layout and the entry point.
// ----------------------------------------------------------------------------
struct BinWs {
  uint32_t *dk0, *dv0, *dk1, *dv1, *cnt, *offs, *tk0, *tk1, *valt;
  int64_t* cnt_dev;
  unsigned long long* k_total;
  void* radix;
  void* scan;
};

static size_t carve_bin_ws(int64_t n, int64_t capacity, char* base, BinWs* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  const size_t nn = (size_t)std::max<int64_t>(n, 1), cc = (size_t)std::max<int64_t>(capacity, 1);
  BinWs t;
  t.dk0 = (uint32_t*)take(4 * nn);
  t.dv0 = (uint32_t*)take(4 * nn);
  t.dk1 = (uint32_t*)take(4 * nn);
  t.dv1 = (uint32_t*)take(4 * nn);
  t.cnt = (uint32_t*)take(4 * nn);
  t.offs = (uint32_t*)take(4 * nn);
  t.tk0 = (uint32_t*)take(4 * cc);
  t.tk1 = (uint32_t*)take(4 * cc);
  t.valt = (uint32_t*)take(4 * cc);
  t.cnt_dev = (int64_t*)take(8);
  t.k_total = (unsigned long long*)take(8);
  t.scan = take(scan_workspace_size((int64_t)nn));
  t.radix = take(radix_workspace_size(std::max<int64_t>(n, capacity)));
  if (w) *w = t;
  return off;
}

static int tile_bits(int64_t n_tiles) {
  int b = 0;
  while (((int64_t)1 << b) < n_tiles) ++b;
  return b;
}

}  // namespace splat

using namespace splat;

extern "C" size_t splat_bin_sort_workspace_size(int64_t n, int64_t capacity, int32_t n_tiles) {
  (void)n_tiles;
  if (n < 0 || capacity < 0) return 0;
  return carve_bin_ws(n, capacity, nullptr, nullptr);
}

extern "C" int splat_bin_sort(const splat_projected* proj, int64_t n, const splat_camera* cam, uint64_t* keys,
                              uint32_t* vals, int64_t capacity, int64_t* k_dev, uint32_t* ranges, int32_t* status,
                              void* ws, size_t ws_bytes, splat_stream_t stream) {
  if (!proj || !cam || !vals || !k_dev || !ranges || !status || !ws)
    return fail(SPLAT_EINVAL, "splat_bin_sort: null argument");
  if (n < 0 || n > 0x7fffffff || capacity < 0 || capacity > 0x7fffffff)
    return fail(SPLAT_EINVAL, "splat_bin_sort: n=%lld capacity=%lld out of range", (long long)n, (long long)capacity);
  if (cam->width <= 0 || cam->height <= 0) return fail(SPLAT_EINVAL, "splat_bin_sort: bad image size");
  if (n > 0 && (!proj->xyzo || !proj->rect || !proj->tiles_touched || !aligned16(proj->xyzo) || !aligned16(proj->rect)))
    return fail(SPLAT_EINVAL, "splat_bin_sort: projected arrays null or not 16-byte aligned");
  const size_t need = carve_bin_ws(n, capacity, nullptr, nullptr);
  if (ws_bytes < need) return fail(SPLAT_EINVAL, "splat_bin_sort: workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const CamK ck = make_camk(*cam);
  const int64_t n_tiles = (int64_t)ck.tiles_x * ck.tiles_y;
  BinWs w;
  carve_bin_ws(n, capacity, static_cast<char*>(ws), &w);
  if (cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * n_tiles, s) != cudaSuccess ||
      cudaMemsetAsync(w.k_total, 0, sizeof(unsigned long long), s) != cudaSuccess)
    return fail(SPLAT_ECUDA, "splat_bin_sort: memset failed");
  const float4* xyzo = reinterpret_cast<const float4*>(proj->xyzo);
  const int nb = std::max(1, ceil_div(n, 256));
  // 1. depth keys of the visible Gaussians (culled ones sort last), K total
  if (n > 0) SPLAT_LAUNCH("depth_keys_kernel", s, depth_keys_kernel<<<nb, 256, 0, s>>>(xyzo, proj->tiles_touched, n, w.dk0, w.dv0, w.k_total));
  int rc = check_launch("depth_keys_kernel");
  if (rc) return rc;
  SPLAT_LAUNCH("finalize_count_kernel", s, finalize_count_kernel<<<1, 1, 0, s>>>(w.k_total, capacity, k_dev, w.cnt_dev, status));
  if ((rc = check_launch("finalize_count_kernel"))) return rc;
  if (n == 0) return SPLAT_OK;
  int which = 0;
  if ((rc = radix_sort<uint32_t>(w.dk0, w.dv0, w.dk1, w.dv1, n, nullptr, 0, 32, w.radix, s, &which))) return rc;
  const uint32_t* order = which ? w.dv1 : w.dv0;
  // 2. duplicate offsets in depth order, emission
  SPLAT_LAUNCH("gather_counts_kernel", s, gather_counts_kernel<<<nb, 256, 0, s>>>(order, proj->tiles_touched, n, w.cnt));
  if ((rc = exclusive_scan_u32(w.cnt, w.offs, n, w.scan, s))) return rc;
  if (capacity == 0) return SPLAT_OK;
  const int tb = tile_bits(n_tiles);
  const int passes = radix_passes(0, tb);
  uint32_t* v0 = (passes & 1) ? w.valt : vals;
  uint32_t* v1 = (passes & 1) ? vals : w.valt;
  SPLAT_LAUNCH("emit_kernel", s, emit_kernel<<<nb, 256, 0, s>>>(order, w.cnt, w.offs, reinterpret_cast<const int4*>(proj->rect), n, ck.tiles_x,
                                 capacity, w.tk0, v0));
  if ((rc = check_launch("emit_kernel"))) return rc;
  // 3. stable sort by tile id
  if ((rc = radix_sort<uint32_t>(w.tk0, v0, w.tk1, v1, capacity, w.cnt_dev, 0, tb, w.radix, s, &which))) return rc;
  const uint32_t* tk = which ? w.tk1 : w.tk0;
  // 4. ranges, optional full keys
  const int kb = std::max(1, ceil_div(capacity, 256));
  SPLAT_LAUNCH("ranges_kernel", s, ranges_kernel<<<kb, 256, 0, s>>>(tk, w.cnt_dev, capacity, ranges));
  if ((rc = check_launch("ranges_kernel"))) return rc;
  if (keys) {
    SPLAT_LAUNCH("full_keys_kernel", s, full_keys_kernel<<<kb, 256, 0, s>>>(tk, vals, xyzo, w.cnt_dev, capacity, keys));
    if ((rc = check_launch("full_keys_kernel"))) return rc;
  }
  return SPLAT_OK;
}
