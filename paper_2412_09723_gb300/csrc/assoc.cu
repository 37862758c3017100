// assoc.cu -- render-based Gaussian association between two maps (Sec. 3.5
// step 2: correspondences between co-visible Gaussians, obtained here from two
// renders of the same viewpoint).  At every pixel where both renders have a
// maximum-weight Gaussian and both final transmittances are <= t_max, the pair
// (id_a, id_b) is formed; the output is the sorted set of distinct pairs with
// the number of pixels of each.
//
// Design: a maximum-weight Gaussian covers runs of neighbouring pixels, so
// every thread reads kAsRun consecutive pixels and merges runs of the same
// pair into one weighted entry (key = id_a << 32 | id_b, weight = pixels).
// Entries are bucketed by ranges of id_a (monotone buckets, so bucket order
// is key order), with per-CTA counts in shared memory and one global atomic
// per (CTA, bucket) to reserve space; each bucket's distinct keys are then
// summed by one CTA in a shared-memory hash table (weights added) and only
// the distinct keys are sorted; a bucket with more distinct keys than the
// table holds uses a hash table in global memory instead.  The distinct pairs
// are written at the offsets of an exclusive scan over the buckets.  Four
// kernels (the scans are folded into the kernels that need them).
#include <algorithm>

#include "common.cuh"
#include "segsort.cuh"

namespace splat {

constexpr int kAsThreads = 256;
constexpr int kAsRun = 8;             // consecutive pixels a thread merges into runs
constexpr int kAsBucketKeys = 1024;   // expected keys per bucket
constexpr int kAsMaxBuckets = 4096;   // shared-memory counters per CTA
constexpr int kAsSegCap = 4096;       // keys a CTA sorts in shared memory
constexpr int kAsStride = 32;         // one 128-byte line per global counter

__device__ __forceinline__ int assoc_bucket(int32_t a, int64_t n_a, int nb) {
  const int64_t b = ((int64_t)a * nb) / n_a;
  return (int)(b < nb ? b : nb - 1);
}

// Pixel range of CTA `blk` out of `grid` (contiguous, so neighbouring pixels,
// which tend to share ids, land in the same CTA; a multiple of kAsRun long, so
// that every thread's chunk starts on a 32-byte boundary).
__device__ __forceinline__ void cta_range(int64_t npix, int64_t& p0, int64_t& p1) {
  int64_t per = (npix + gridDim.x - 1) / gridDim.x;
  per = (per + kAsRun - 1) / kAsRun * kAsRun;
  p0 = (int64_t)blockIdx.x * per;
  p1 = p0 + per < npix ? p0 + per : npix;
}

// Walks the kAsRun-pixel chunks of this CTA's range; calls emit(key, weight)
// once per run of equal valid pairs (in pixel order).
// vec: all four images 16-byte aligned, so a full chunk is read with 128-bit loads.
template <class Emit>
__device__ __forceinline__ void for_each_run(const int32_t* __restrict__ ia, const float* __restrict__ ta,
                                             const int32_t* __restrict__ ib, const float* __restrict__ tb,
                                             int64_t p0, int64_t p1, float tmax, bool vec, Emit emit) {
  for (int64_t c = p0 + (int64_t)threadIdx.x * kAsRun; c < p1; c += (int64_t)kAsThreads * kAsRun) {
    int32_t a[kAsRun], b[kAsRun];
    float u[kAsRun], v[kAsRun];
    const int len = c + kAsRun <= p1 ? kAsRun : (int)(p1 - c);
    if (vec && len == kAsRun) {
#pragma unroll
      for (int h = 0; h < kAsRun; h += 4) {
        const int4 x = *reinterpret_cast<const int4*>(ia + c + h);
        const int4 y = *reinterpret_cast<const int4*>(ib + c + h);
        const float4 tx = *reinterpret_cast<const float4*>(ta + c + h);
        const float4 ty = *reinterpret_cast<const float4*>(tb + c + h);
        a[h] = x.x; a[h + 1] = x.y; a[h + 2] = x.z; a[h + 3] = x.w;
        b[h] = y.x; b[h + 1] = y.y; b[h + 2] = y.z; b[h + 3] = y.w;
        u[h] = tx.x; u[h + 1] = tx.y; u[h + 2] = tx.z; u[h + 3] = tx.w;
        v[h] = ty.x; v[h + 1] = ty.y; v[h + 2] = ty.z; v[h + 3] = ty.w;
      }
    } else {
#pragma unroll
      for (int h = 0; h < kAsRun; ++h) {
        const bool in = h < len;
        a[h] = in ? ia[c + h] : -1;
        b[h] = in ? ib[c + h] : -1;
        u[h] = in ? ta[c + h] : 0.f;
        v[h] = in ? tb[c + h] : 0.f;
      }
    }
    uint64_t cur = 0;
    uint32_t w = 0;
#pragma unroll
    for (int h = 0; h < kAsRun; ++h) {
      if (!(a[h] >= 0 && b[h] >= 0 && u[h] <= tmax && v[h] <= tmax)) continue;
      const uint64_t key = ((uint64_t)(uint32_t)a[h] << 32) | (uint64_t)(uint32_t)b[h];
      if (w && key == cur) {
        ++w;
      } else {
        if (w) emit(cur, w);
        cur = key;
        w = 1;
      }
    }
    if (w) emit(cur, w);
  }
}

__global__ void __launch_bounds__(kAsThreads) assoc_count_kernel(const int32_t* __restrict__ ia,
                                                                 const float* __restrict__ ta,
                                                                 const int32_t* __restrict__ ib,
                                                                 const float* __restrict__ tb, int64_t npix,
                                                                 float tmax, int64_t n_a, int nb, bool vec,
                                                                 uint32_t* __restrict__ bcnt) {
  __shared__ uint32_t s_cnt[kAsMaxBuckets];
  for (int b = threadIdx.x; b < nb; b += kAsThreads) s_cnt[b] = 0u;
  __syncthreads();
  int64_t p0, p1;
  cta_range(npix, p0, p1);
  for_each_run(ia, ta, ib, tb, p0, p1, tmax, vec, [&](uint64_t key, uint32_t) {
    atomicAdd(&s_cnt[assoc_bucket((int32_t)(key >> 32), n_a, nb)], 1u);
  });
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += kAsThreads)
    if (s_cnt[b]) atomicAdd(&bcnt[(size_t)b * kAsStride], s_cnt[b]);
}

__global__ void __launch_bounds__(kAsThreads) assoc_scatter_kernel(
    const int32_t* __restrict__ ia, const float* __restrict__ ta, const int32_t* __restrict__ ib,
    const float* __restrict__ tb, int64_t npix, float tmax, int64_t n_a, int nb, bool vec,
    const uint32_t* __restrict__ bcnt, uint32_t* __restrict__ cursor, uint32_t* __restrict__ bstart,
    uint64_t* __restrict__ skeys, uint32_t* __restrict__ sw) {
  __shared__ uint32_t s_cnt[kAsMaxBuckets];
  __shared__ uint32_t s_base[kAsMaxBuckets];  // bucket starts, then this CTA's reserved positions
  __shared__ uint32_t sh[33];
  // bucket starts: exclusive scan of the bucket counts (every CTA computes it;
  // CTA 0 also publishes it, with the total, for the per-bucket kernel)
  {
    const int per = (nb + kAsThreads - 1) / kAsThreads;
    const int b0 = min(nb, (int)threadIdx.x * per), b1 = min(nb, b0 + per);
    uint32_t loc = 0;
    for (int b = b0; b < b1; ++b) loc += bcnt[(size_t)b * kAsStride];
    uint32_t excl;
    const uint32_t tot = block_excl_scan<kAsThreads>(loc, excl, sh);
    for (int b = b0; b < b1; ++b) {
      s_base[b] = excl;
      if (blockIdx.x == 0) bstart[b] = excl;
      excl += bcnt[(size_t)b * kAsStride];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) bstart[nb] = tot;
  }
  for (int b = threadIdx.x; b < nb; b += kAsThreads) s_cnt[b] = 0u;
  __syncthreads();
  int64_t p0, p1;
  cta_range(npix, p0, p1);
  for_each_run(ia, ta, ib, tb, p0, p1, tmax, vec, [&](uint64_t key, uint32_t) {
    atomicAdd(&s_cnt[assoc_bucket((int32_t)(key >> 32), n_a, nb)], 1u);
  });
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += kAsThreads) {  // cursors count from 0 within each bucket
    const uint32_t c = s_cnt[b];
    if (c) s_base[b] += atomicAdd(&cursor[(size_t)b * kAsStride], c);
    s_cnt[b] = 0u;
  }
  __syncthreads();
  for_each_run(ia, ta, ib, tb, p0, p1, tmax, vec, [&](uint64_t key, uint32_t w) {
    const int b = assoc_bucket((int32_t)(key >> 32), n_a, nb);
    const uint32_t pos = s_base[b] + atomicAdd(&s_cnt[b], 1u);
    skeys[pos] = key;
    sw[pos] = w;
  });
}

constexpr int kAsHash = 2048;             // shared-memory hash slots per bucket
constexpr int kAsHashMaxDistinct = 1536;  // at most 75% load, else the global-memory table
constexpr uint64_t kAsEmpty = ~0ull;

__device__ __forceinline__ uint32_t assoc_hash(uint64_t key) {
  return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 32);
}

// One CTA per bucket.  The weights of equal keys are summed in a hash table
// (linear probing, bounded by the table size): in shared memory when the
// bucket has at most kAsHashMaxDistinct distinct keys, else in the bucket's
// own global region of 2n slots (gkey/gcnt at 2 * start).  The distinct keys
// are then sorted (bitonic in shared memory, or the segment sort through
// global memory) and written with their summed weights at the bucket's start
// of ukeys / ucnt; nuniq[b] = number of distinct keys.
__global__ void __launch_bounds__(kAsThreads) assoc_sort_rle_kernel(const uint32_t* __restrict__ bstart,
                                                                    const uint64_t* __restrict__ skeys,
                                                                    const uint32_t* __restrict__ sw,
                                                                    uint64_t* __restrict__ skeys2,
                                                                    uint64_t* __restrict__ skeys3,
                                                                    uint64_t* __restrict__ gkey,
                                                                    uint32_t* __restrict__ gcnt,
                                                                    uint64_t* __restrict__ ukeys,
                                                                    uint32_t* __restrict__ ucnt,
                                                                    uint32_t* __restrict__ nuniq) {
  __shared__ uint64_t smem[kAsSegCap];  // hash keys (first kAsHash), then the distinct keys
  __shared__ uint32_t s_hcnt[kAsHash];
  __shared__ uint32_t sh[33];
  __shared__ int s_overflow;
  __shared__ uint32_t s_ndist;
  const int b = blockIdx.x;
  const uint32_t s0 = bstart[b];
  const int n = (int)(bstart[b + 1] - s0);
  if (n <= 0) {
    if (threadIdx.x == 0) nuniq[b] = 0u;
    return;
  }
  // 1. shared-memory table
  uint64_t* hkey = smem;
  for (int i = threadIdx.x; i < kAsHash; i += kAsThreads) {
    hkey[i] = kAsEmpty;
    s_hcnt[i] = 0u;
  }
  if (threadIdx.x == 0) {
    s_overflow = 0;
    s_ndist = 0u;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n && !s_overflow; i += kAsThreads) {
    const uint64_t key = skeys[s0 + i];
    uint32_t h = assoc_hash(key) & (kAsHash - 1);
    int probes = 0;
    for (; probes < kAsHash; ++probes, h = (h + 1) & (kAsHash - 1)) {
      const uint64_t prev = atomicCAS(reinterpret_cast<unsigned long long*>(&hkey[h]), kAsEmpty, key);
      if (prev == kAsEmpty) {
        if (atomicAdd(&s_ndist, 1u) >= (uint32_t)kAsHashMaxDistinct) s_overflow = 1;
        break;
      }
      if (prev == key) break;
    }
    if (probes == kAsHash) s_overflow = 1;
    else atomicAdd(&s_hcnt[h], sw[s0 + i]);
  }
  __syncthreads();
  if (!s_overflow) {
    // compact the occupied slots, sort the distinct keys, look their sums up
    uint32_t mine = 0;
    const int per = kAsHash / kAsThreads;
    for (int i = threadIdx.x * per; i < (threadIdx.x + 1) * per; ++i) mine += hkey[i] != kAsEmpty ? 1u : 0u;
    uint32_t off;
    const uint32_t nd = block_excl_scan<kAsThreads>(mine, off, sh);
    uint64_t* dk = smem + kAsHash;  // nd <= 1536 <= kAsSegCap - kAsHash
    for (int i = threadIdx.x * per; i < (threadIdx.x + 1) * per; ++i)
      if (hkey[i] != kAsEmpty) dk[off++] = hkey[i];
    __syncthreads();
    const int n2 = next_pow2((int)nd);
    for (int i = (int)nd + threadIdx.x; i < n2; i += kAsThreads) dk[i] = kAsEmpty;
    __syncthreads();
    cta_bitonic_u64(dk, n2);
    for (int u = threadIdx.x; u < (int)nd; u += kAsThreads) {
      const uint64_t key = dk[u];
      uint32_t h = assoc_hash(key) & (kAsHash - 1);
      for (int probes = 0; probes < kAsHash && hkey[h] != key; ++probes) h = (h + 1) & (kAsHash - 1);
      ukeys[s0 + u] = key;
      ucnt[s0 + u] = s_hcnt[h];
    }
    if (threadIdx.x == 0) nuniq[b] = nd;
    return;
  }
  // 2. global-memory table of 2n slots (never more than half full)
  const uint32_t T = 2u * (uint32_t)n;
  uint64_t* tk = gkey + 2 * (size_t)s0;
  uint32_t* tc = gcnt + 2 * (size_t)s0;
  for (uint32_t i = threadIdx.x; i < T; i += kAsThreads) {
    tk[i] = kAsEmpty;
    tc[i] = 0u;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kAsThreads) {
    const uint64_t key = skeys[s0 + i];
    uint32_t h = assoc_hash(key) % T;
    for (uint32_t probes = 0; probes < T; ++probes, h = h + 1 == T ? 0u : h + 1) {
      const uint64_t prev = atomicCAS(reinterpret_cast<unsigned long long*>(&tk[h]), kAsEmpty, key);
      if (prev == kAsEmpty || prev == key) {
        atomicAdd(&tc[h], sw[s0 + i]);
        break;
      }
    }
  }
  __syncthreads();
  // distinct keys -> skeys2[s0, s0 + nd) in slot order, then sorted into ukeys
  uint32_t carry = 0;
  for (uint32_t base = 0; base < T; base += kAsThreads) {
    const uint32_t i = base + threadIdx.x;
    const bool occ = i < T && tk[i] != kAsEmpty;
    uint32_t off;
    const uint32_t tot = block_excl_scan<kAsThreads>(occ ? 1u : 0u, off, sh);
    if (occ) skeys2[s0 + carry + off] = tk[i];
    carry += tot;
  }
  __syncthreads();
  const int nd = (int)carry;
  cta_sort_segment(skeys2 + s0, ukeys + s0, skeys3 + s0, nd, smem, kAsSegCap);
  __syncthreads();
  for (int u = threadIdx.x; u < nd; u += kAsThreads) {
    const uint64_t key = ukeys[s0 + u];
    uint32_t h = assoc_hash(key) % T;
    for (uint32_t probes = 0; probes < T && tk[h] != key; ++probes) h = h + 1 == T ? 0u : h + 1;
    ucnt[s0 + u] = tc[h];
  }
  if (threadIdx.x == 0) nuniq[b] = (uint32_t)nd;
}

// One CTA per bucket: its distinct pairs go to the output at the sum of the
// distinct counts of the buckets before it; the last bucket's CTA writes M
// and raises SPLAT_ECAPACITY when M exceeds the capacity.
__global__ void __launch_bounds__(kAsThreads) assoc_write_kernel(const uint32_t* __restrict__ bstart,
                                                                 const uint32_t* __restrict__ nuniq, int nb,
                                                                 const uint64_t* __restrict__ ukeys,
                                                                 const uint32_t* __restrict__ ucnt, int64_t capacity,
                                                                 int32_t* __restrict__ pairs,
                                                                 int32_t* __restrict__ counts,
                                                                 int64_t* __restrict__ m_dev,
                                                                 int32_t* __restrict__ status) {
  __shared__ unsigned long long red[kAsThreads / 32];
  const int b = blockIdx.x;
  unsigned long long part = 0;
  for (int k = threadIdx.x; k < b; k += kAsThreads) part += nuniq[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  unsigned long long o0 = 0;
  for (int w = 0; w < kAsThreads / 32; ++w) o0 += red[w];
  const uint32_t s0 = bstart[b], nu = nuniq[b];
  if (b == nb - 1 && threadIdx.x == 0) {
    *m_dev = (int64_t)(o0 + nu);
    if ((int64_t)(o0 + nu) > capacity) raise_status(status, SPLAT_ECAPACITY);
  }
  for (uint32_t u = threadIdx.x; u < nu; u += kAsThreads) {
    const int64_t o = (int64_t)o0 + u;
    if (o >= capacity) break;
    const uint64_t key = ukeys[s0 + u];
    pairs[2 * o] = (int32_t)(key >> 32);
    pairs[2 * o + 1] = (int32_t)(key & 0xffffffffu);
    counts[o] = (int32_t)ucnt[s0 + u];
  }
}

struct AssocWs {
  uint32_t *bcnt, *cursor, *bstart, *nuniq, *ucnt, *sw, *gcnt;
  uint64_t *skeys, *skeys2, *skeys3, *ukeys, *gkey;
};

static int assoc_buckets(int64_t npix) {
  const int64_t nb = (npix + kAsBucketKeys - 1) / kAsBucketKeys;
  return (int)std::max<int64_t>(1, std::min<int64_t>(nb, kAsMaxBuckets));
}

static size_t carve_assoc(int64_t npix, char* base, AssocWs* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  const size_t n = (size_t)std::max<int64_t>(npix, 1);
  const size_t nb = (size_t)assoc_buckets(npix);
  AssocWs t;
  t.bcnt = (uint32_t*)take(4 * kAsStride * nb);
  t.cursor = (uint32_t*)take(4 * kAsStride * nb);
  t.bstart = (uint32_t*)take(4 * (nb + 1));
  t.nuniq = (uint32_t*)take(4 * nb);
  t.ucnt = (uint32_t*)take(4 * n);
  t.sw = (uint32_t*)take(4 * n);
  t.gcnt = (uint32_t*)take(4 * 2 * n);
  t.skeys = (uint64_t*)take(8 * n);
  t.skeys2 = (uint64_t*)take(8 * n);
  t.skeys3 = (uint64_t*)take(8 * n);
  t.ukeys = (uint64_t*)take(8 * n);
  t.gkey = (uint64_t*)take(8 * 2 * n);
  if (w) *w = t;
  return off;
}

}  // namespace splat

using namespace splat;

extern "C" size_t splat_assoc_workspace_size(int64_t npix) { return npix < 0 ? 0 : carve_assoc(npix, nullptr, nullptr); }

extern "C" int splat_assoc(const int32_t* id_a, const float* t_a, const int32_t* id_b, const float* t_b, int64_t npix,
                           int64_t n_a, int64_t n_b, float t_max, int32_t* pairs, int32_t* counts, int64_t capacity,
                           int64_t* m_dev, int32_t* status, void* ws, size_t ws_bytes, splat_stream_t stream) {
  if (!id_a || !t_a || !id_b || !t_b || !m_dev || !status || !ws || npix < 0 || capacity < 0 || n_a < 1 || n_b < 1 ||
      n_a > 0x7fffffff || n_b > 0x7fffffff || npix > 0x7fffffff)
    return fail(SPLAT_EINVAL, "splat_assoc: bad argument");
  if (capacity > 0 && (!pairs || !counts)) return fail(SPLAT_EINVAL, "splat_assoc: null output");
  if (ws_bytes < carve_assoc(npix, nullptr, nullptr) || !aligned16(ws))
    return fail(SPLAT_EINVAL, "splat_assoc: workspace too small or misaligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (npix == 0) {
    if (cudaMemsetAsync(m_dev, 0, sizeof(int64_t), s) != cudaSuccess) return fail(SPLAT_ECUDA, "splat_assoc: memset");
    return SPLAT_OK;
  }
  AssocWs w;
  carve_assoc(npix, static_cast<char*>(ws), &w);
  const int nb = assoc_buckets(npix);
  // bucket counts and cursors are adjacent in the workspace: one memset
  const size_t zero_bytes = (size_t)((char*)(w.cursor + (size_t)kAsStride * nb) - (char*)w.bcnt);
  if (cudaMemsetAsync(w.bcnt, 0, zero_bytes, s) != cudaSuccess) return fail(SPLAT_ECUDA, "splat_assoc: memset failed");
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((npix + 1023) / 1024, 2 * sms));
  const bool vec = aligned16(id_a) && aligned16(t_a) && aligned16(id_b) && aligned16(t_b);
  SPLAT_LAUNCH("assoc_count_kernel", s,
               assoc_count_kernel<<<grid, kAsThreads, 0, s>>>(id_a, t_a, id_b, t_b, npix, t_max, n_a, nb, vec,
                                                              w.bcnt));
  SPLAT_LAUNCH("assoc_scatter_kernel", s,
               assoc_scatter_kernel<<<grid, kAsThreads, 0, s>>>(id_a, t_a, id_b, t_b, npix, t_max, n_a, nb, vec,
                                                                w.bcnt, w.cursor, w.bstart, w.skeys, w.sw));
  SPLAT_LAUNCH("assoc_sort_rle_kernel", s,
               assoc_sort_rle_kernel<<<nb, kAsThreads, 0, s>>>(w.bstart, w.skeys, w.sw, w.skeys2, w.skeys3, w.gkey,
                                                                w.gcnt, w.ukeys, w.ucnt, w.nuniq));
  SPLAT_LAUNCH("assoc_write_kernel", s,
               assoc_write_kernel<<<nb, kAsThreads, 0, s>>>(w.bstart, w.nuniq, nb, w.ukeys, w.ucnt, capacity, pairs,
                                                            counts, m_dev, status));
  return check_launch("assoc_write_kernel");
}
