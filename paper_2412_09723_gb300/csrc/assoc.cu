// assoc.cu -- render-based Gaussian association between two maps (Sec. 3.5
// step 2: correspondences between co-visible Gaussians, obtained here from two
// renders of the same viewpoint).  At every pixel where both renders have a
// maximum-weight Gaussian and both final transmittances are <= t_max, the pair
// (id_a, id_b) is formed; the output is the sorted set of distinct pairs with
// the number of pixels of each.
//
// Design: the 64-bit pair keys (id_a << 32 | id_b) are bucketed by ranges of
// id_a (monotone buckets, so bucket order is key order), with per-CTA counts in
// shared memory and one global atomic per (CTA, bucket) to reserve space; each
// bucket's distinct keys are then counted by one CTA in a shared-memory hash
// table and only the distinct keys are sorted (a bucket with too many distinct
// keys is sorted whole and run-length encoded); the distinct pairs are written
// at the offsets of an exclusive scan over the buckets.  Six kernels.
#include <algorithm>

#include "common.cuh"
#include "segsort.cuh"

namespace splat {

constexpr int kAsThreads = 256;
constexpr int kAsBucketKeys = 1024;   // expected keys per bucket
constexpr int kAsMaxBuckets = 4096;   // shared-memory counters per CTA
constexpr int kAsSegCap = 4096;       // keys a CTA sorts in shared memory
constexpr int kAsStride = 32;         // one 128-byte line per global counter

__device__ __forceinline__ bool assoc_valid(const int32_t* ia, const float* ta, const int32_t* ib, const float* tb,
                                            int64_t p, float tmax) {
  return ia[p] >= 0 && ib[p] >= 0 && ta[p] <= tmax && tb[p] <= tmax;
}

__device__ __forceinline__ int assoc_bucket(int32_t a, int64_t n_a, int nb) {
  const int64_t b = ((int64_t)a * nb) / n_a;
  return (int)(b < nb ? b : nb - 1);
}

// Pixel range of CTA `blk` out of `grid` (contiguous, so neighbouring pixels,
// which tend to share ids, land in the same CTA).
__device__ __forceinline__ void cta_range(int64_t npix, int64_t& p0, int64_t& p1) {
  const int64_t per = (npix + gridDim.x - 1) / gridDim.x;
  p0 = (int64_t)blockIdx.x * per;
  p1 = p0 + per < npix ? p0 + per : npix;
}

__global__ void __launch_bounds__(kAsThreads) assoc_count_kernel(const int32_t* __restrict__ ia,
                                                                 const float* __restrict__ ta,
                                                                 const int32_t* __restrict__ ib,
                                                                 const float* __restrict__ tb, int64_t npix,
                                                                 float tmax, int64_t n_a, int nb,
                                                                 uint32_t* __restrict__ bcnt) {
  __shared__ uint32_t s_cnt[kAsMaxBuckets];
  for (int b = threadIdx.x; b < nb; b += kAsThreads) s_cnt[b] = 0u;
  __syncthreads();
  int64_t p0, p1;
  cta_range(npix, p0, p1);
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kAsThreads)
    if (assoc_valid(ia, ta, ib, tb, p, tmax)) atomicAdd(&s_cnt[assoc_bucket(ia[p], n_a, nb)], 1u);
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += kAsThreads)
    if (s_cnt[b]) atomicAdd(&bcnt[(size_t)b * kAsStride], s_cnt[b]);
}

// One CTA: bucket starts (exclusive scan) and cursors.
__global__ void __launch_bounds__(1024) assoc_scan_kernel(const uint32_t* __restrict__ bcnt, int nb,
                                                          uint32_t* __restrict__ bstart,
                                                          uint32_t* __restrict__ cursor) {
  __shared__ uint32_t sh[33];
  uint32_t carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    const int b = base + threadIdx.x;
    const uint32_t c = b < nb ? bcnt[(size_t)b * kAsStride] : 0u;
    uint32_t excl;
    const uint32_t tot = block_excl_scan<1024>(c, excl, sh);
    if (b < nb) {
      bstart[b] = carry + excl;
      cursor[(size_t)b * kAsStride] = carry + excl;
    }
    carry += tot;
  }
  if (threadIdx.x == 0) bstart[nb] = carry;
}

__global__ void __launch_bounds__(kAsThreads) assoc_scatter_kernel(
    const int32_t* __restrict__ ia, const float* __restrict__ ta, const int32_t* __restrict__ ib,
    const float* __restrict__ tb, int64_t npix, float tmax, int64_t n_a, int nb, uint32_t* __restrict__ cursor,
    uint64_t* __restrict__ skeys) {
  __shared__ uint32_t s_cnt[kAsMaxBuckets];
  __shared__ uint32_t s_base[kAsMaxBuckets];
  for (int b = threadIdx.x; b < nb; b += kAsThreads) s_cnt[b] = 0u;
  __syncthreads();
  int64_t p0, p1;
  cta_range(npix, p0, p1);
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kAsThreads)
    if (assoc_valid(ia, ta, ib, tb, p, tmax)) atomicAdd(&s_cnt[assoc_bucket(ia[p], n_a, nb)], 1u);
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += kAsThreads) {
    const uint32_t c = s_cnt[b];
    s_base[b] = c ? atomicAdd(&cursor[(size_t)b * kAsStride], c) : 0u;
    s_cnt[b] = 0u;
  }
  __syncthreads();
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kAsThreads)
    if (assoc_valid(ia, ta, ib, tb, p, tmax)) {
      const int b = assoc_bucket(ia[p], n_a, nb);
      const uint32_t pos = s_base[b] + atomicAdd(&s_cnt[b], 1u);
      skeys[pos] = ((uint64_t)(uint32_t)ia[p] << 32) | (uint64_t)(uint32_t)ib[p];
    }
}

constexpr int kAsHash = 2048;          // shared-memory hash slots per bucket
constexpr int kAsHashMaxDistinct = 1536;  // at most 75% load, else the sort path
constexpr uint64_t kAsEmpty = ~0ull;

// One CTA per bucket.  Distinct keys and their multiplicities are collected in
// a shared-memory hash table (linear probing, bounded by the table size); the
// distinct keys are then bitonic-sorted and written with their counts at the
// bucket's own start of ukeys / ucnt; nuniq[b] = number of distinct keys.  If
// a bucket holds more distinct keys than the table takes, the CTA sorts the
// whole bucket and run-length encodes it instead.
__global__ void __launch_bounds__(kAsThreads) assoc_sort_rle_kernel(const uint32_t* __restrict__ bstart,
                                                                    uint64_t* __restrict__ skeys,
                                                                    uint64_t* __restrict__ skeys2,
                                                                    uint64_t* __restrict__ ukeys,
                                                                    uint32_t* __restrict__ ucnt,
                                                                    uint32_t* __restrict__ nuniq) {
  __shared__ uint64_t smem[kAsSegCap];  // hash keys (first kAsHash), later the sort buffer
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
  // 1. hash count
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
  for (int i = threadIdx.x; i < n; i += kAsThreads) {
    const uint64_t key = skeys[s0 + i];
    uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 53);  // 11 bits
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
    else atomicAdd(&s_hcnt[h], 1u);
  }
  __syncthreads();
  if (!s_overflow) {
    // 2. compact the occupied slots (slot order), then sort the distinct keys
    //    together with their counts (count in a parallel array, moved by rank)
    uint32_t mine = 0;
    const int per = kAsHash / kAsThreads;
    for (int i = threadIdx.x * per; i < (threadIdx.x + 1) * per; ++i) mine += hkey[i] != kAsEmpty ? 1u : 0u;
    uint32_t off;
    const uint32_t nd = block_excl_scan<kAsThreads>(mine, off, sh);
    uint64_t* dk = smem + kAsHash;  // distinct keys (nd <= 1536 <= kAsSegCap - kAsHash)
    for (int i = threadIdx.x * per; i < (threadIdx.x + 1) * per; ++i)
      if (hkey[i] != kAsEmpty) dk[off++] = hkey[i];
    __syncthreads();
    const int n2 = next_pow2((int)nd);
    for (int i = (int)nd + threadIdx.x; i < n2; i += kAsThreads) dk[i] = kAsEmpty;
    __syncthreads();
    cta_bitonic_u64(dk, n2);
    for (int u = threadIdx.x; u < (int)nd; u += kAsThreads) {
      const uint64_t key = dk[u];
      uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 53);
      for (int probes = 0; probes < kAsHash && hkey[h] != key; ++probes) h = (h + 1) & (kAsHash - 1);
      ukeys[s0 + u] = key;
      ucnt[s0 + u] = s_hcnt[h];
    }
    if (threadIdx.x == 0) nuniq[b] = nd;
    return;
  }
  __syncthreads();
  // 3. too many distinct keys: sort the bucket and run-length encode it
  const uint64_t* k;
  if (n <= kAsSegCap) {
    cta_sort_small(skeys + s0, n, smem);
    k = smem;
  } else {
    cta_sort_segment(skeys + s0, skeys2 + s0, skeys + s0, n, smem, kAsSegCap);
    k = skeys2 + s0;
  }
  const int per = (n + kAsThreads - 1) / kAsThreads;
  const int i0 = threadIdx.x * per;
  const int i1 = min(n, i0 + per);
  uint32_t heads = 0;
  for (int i = i0; i < i1; ++i) heads += (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
  uint32_t u;
  const uint32_t total = block_excl_scan<kAsThreads>(heads, u, sh);
  for (int i = i0; i < i1; ++i) {
    if (!(i == 0 || k[i] != k[i - 1])) continue;
    int j = i + 1;
    while (j < n && k[j] == k[i]) ++j;
    ukeys[s0 + u] = k[i];
    ucnt[s0 + u] = (uint32_t)(j - i);
    ++u;
  }
  if (threadIdx.x == 0) nuniq[b] = total;
}

__global__ void __launch_bounds__(1024) assoc_offsets_kernel(const uint32_t* __restrict__ nuniq, int nb,
                                                             uint32_t* __restrict__ uoff, int64_t capacity,
                                                             int64_t* __restrict__ m_dev,
                                                             int32_t* __restrict__ status) {
  __shared__ uint32_t sh[33];
  uint32_t carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    const int b = base + threadIdx.x;
    const uint32_t c = b < nb ? nuniq[b] : 0u;
    uint32_t excl;
    const uint32_t tot = block_excl_scan<1024>(c, excl, sh);
    if (b < nb) uoff[b] = carry + excl;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    *m_dev = (int64_t)carry;
    if ((int64_t)carry > capacity) raise_status(status, SPLAT_ECAPACITY);
  }
}

__global__ void __launch_bounds__(kAsThreads) assoc_write_kernel(const uint32_t* __restrict__ bstart,
                                                                 const uint32_t* __restrict__ nuniq,
                                                                 const uint32_t* __restrict__ uoff,
                                                                 const uint64_t* __restrict__ ukeys,
                                                                 const uint32_t* __restrict__ ucnt, int64_t capacity,
                                                                 int32_t* __restrict__ pairs,
                                                                 int32_t* __restrict__ counts) {
  const int b = blockIdx.x;
  const uint32_t s0 = bstart[b], nu = nuniq[b], o0 = uoff[b];
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
  uint32_t *bcnt, *cursor, *bstart, *nuniq, *uoff, *ucnt;
  uint64_t *skeys, *skeys2, *ukeys;
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
  t.uoff = (uint32_t*)take(4 * nb);
  t.ucnt = (uint32_t*)take(4 * n);
  t.skeys = (uint64_t*)take(8 * n);
  t.skeys2 = (uint64_t*)take(8 * n);
  t.ukeys = (uint64_t*)take(8 * n);
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
  if (cudaMemsetAsync(w.bcnt, 0, sizeof(uint32_t) * kAsStride * nb, s) != cudaSuccess)
    return fail(SPLAT_ECUDA, "splat_assoc: memset failed");
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((npix + 1023) / 1024, 2 * sms));
  SPLAT_LAUNCH("assoc_count_kernel", s,
               assoc_count_kernel<<<grid, kAsThreads, 0, s>>>(id_a, t_a, id_b, t_b, npix, t_max, n_a, nb, w.bcnt));
  SPLAT_LAUNCH("assoc_scan_kernel", s, assoc_scan_kernel<<<1, 1024, 0, s>>>(w.bcnt, nb, w.bstart, w.cursor));
  SPLAT_LAUNCH("assoc_scatter_kernel", s,
               assoc_scatter_kernel<<<grid, kAsThreads, 0, s>>>(id_a, t_a, id_b, t_b, npix, t_max, n_a, nb, w.cursor,
                                                                w.skeys));
  SPLAT_LAUNCH("assoc_sort_rle_kernel", s,
               assoc_sort_rle_kernel<<<nb, kAsThreads, 0, s>>>(w.bstart, w.skeys, w.skeys2, w.ukeys, w.ucnt,
                                                                w.nuniq));
  SPLAT_LAUNCH("assoc_offsets_kernel", s,
               assoc_offsets_kernel<<<1, 1024, 0, s>>>(w.nuniq, nb, w.uoff, capacity, m_dev, status));
  int rc = check_launch("assoc_offsets_kernel");
  if (rc || capacity == 0) return rc;
  SPLAT_LAUNCH("assoc_write_kernel", s,
               assoc_write_kernel<<<nb, kAsThreads, 0, s>>>(w.bstart, w.nuniq, w.uoff, w.ukeys, w.ucnt, capacity,
                                                            pairs, counts));
  return check_launch("assoc_write_kernel");
}
