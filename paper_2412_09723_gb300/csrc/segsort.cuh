// segsort.cuh -- CTA-level primitives: block scan, and one CTA sorting one
// segment of 64-bit keys ascending.
//
// Segments up to the shared-memory capacity are loaded, padded to a power of
// two with all-ones keys and bitonic-sorted in shared memory.  Longer segments
// are sorted in capacity-sized chunks (same routine), then merged pairwise
// with a merge-path rank per element (a binary search into the other run;
// equal keys of the left run go first, so duplicates are allowed),
// ping-ponging between the caller's output and temporary arrays.
#pragma once

#include "common.cuh"

namespace splat {

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

// Bitonic sort of s[0, n2) ascending; n2 a power of two; all threads of the CTA.
__device__ __forceinline__ void cta_bitonic_u64(uint64_t* s, int n2) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < (n2 >> 1); i += blockDim.x) {
        const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
        const int hi = lo + j;
        const bool up = (lo & k) == 0;
        const uint64_t a = s[lo], b = s[hi];
        if ((a > b) == up) {
          s[lo] = b;
          s[hi] = a;
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ int next_pow2(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

// ---------------------------------------------------------------------------
// Register-blocked bitonic sort: thread t holds elements [t E, t E + E) of the
// n2 = E * blockDim.x keys.  Compare-exchange partners at distance j < E are in
// the same thread, at E <= j < 32 E in another lane of the same warp (shuffle),
// and only the stages with j >= 32 E go through shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t x, int m) {
  const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)x, m);
  const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(x >> 32), m);
  return ((uint64_t)hi << 32) | lo;
}

template <int E, int J>
__device__ __forceinline__ void bitonic_inreg(uint64_t (&v)[E], int t, int k) {
#pragma unroll
  for (int i = 0; i < E; ++i) {
    if (i & J) continue;
    const bool up = ((t * E + i) & k) == 0;
    const uint64_t a = v[i], b = v[i + J];
    const bool sw = (a > b) == up;
    v[i] = sw ? b : a;
    v[i + J] = sw ? a : b;
  }
}

template <int E>
__device__ __forceinline__ void bitonic_inreg_any(uint64_t (&v)[E], int t, int k, int j) {
  if constexpr (E > 8) {
    if (j == 8) { bitonic_inreg<E, 8>(v, t, k); return; }
  }
  if constexpr (E > 4) {
    if (j == 4) { bitonic_inreg<E, 4>(v, t, k); return; }
  }
  if constexpr (E > 2) {
    if (j == 2) { bitonic_inreg<E, 2>(v, t, k); return; }
  }
  if constexpr (E > 1) {
    if (j == 1) { bitonic_inreg<E, 1>(v, t, k); return; }
  }
}

template <int E>
__device__ void cta_bitonic_reg(uint64_t* s, int n2) {
  const int t = threadIdx.x;
  uint64_t v[E];
#pragma unroll
  for (int i = 0; i < E; ++i) v[i] = s[t * E + i];
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < E) {
        bitonic_inreg_any<E>(v, t, k, j);
      } else if (j < 32 * E) {
        const int m = j / E;
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int g = t * E + i;
          const bool keep_min = (((g & k) == 0) == ((g & j) == 0));
          const uint64_t o = shfl_xor_u64(v[i], m);
          v[i] = keep_min ? (o < v[i] ? o : v[i]) : (o > v[i] ? o : v[i]);
        }
      } else {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < E; ++i) s[t * E + i] = v[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int g = t * E + i;
          const bool keep_min = (((g & k) == 0) == ((g & j) == 0));
          const uint64_t o = s[g ^ j];
          v[i] = keep_min ? (o < v[i] ? o : v[i]) : (o > v[i] ? o : v[i]);
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < E; ++i) s[t * E + i] = v[i];
  __syncthreads();
}

// Bitonic sort of smem[0, n2) (n2 a power of two, already padded).
// blockDim.x must be 256 when n2 can exceed 256 (register-blocked stages).
__device__ __forceinline__ void cta_bitonic_any(uint64_t* smem, int n2) {
  if (blockDim.x != 256 || n2 <= 256) {
    cta_bitonic_u64(smem, n2);
    return;
  }
  switch (n2 >> 8) {
    case 2: cta_bitonic_reg<2>(smem, n2); break;
    case 4: cta_bitonic_reg<4>(smem, n2); break;
    case 8: cta_bitonic_reg<8>(smem, n2); break;
    default: cta_bitonic_u64(smem, n2); break;  // 4096: shared-memory stages only
  }
}

// Sort in[0, n) into smem (n <= cap) and leave the result in smem[0, n).
__device__ __forceinline__ void cta_sort_small(const uint64_t* in, int n, uint64_t* smem) {
  const int n2 = next_pow2(n < 1 ? 1 : n);
  for (int i = threadIdx.x; i < n2; i += blockDim.x) smem[i] = i < n ? in[i] : ~0ull;
  __syncthreads();
  cta_bitonic_any(smem, n2);
}

// ---------------------------------------------------------------------------
// LSD radix sort in shared memory of 64-bit keys whose high word is the
// primary key and whose low word breaks ties (depth bits | id).  Only the
// high-word bits that differ within the segment are sorted, 8 per pass, each
// pass a stable counting sort: every warp owns a contiguous slice and counts
// its digits in its own 256 counters (shared-memory atomics), the (digit,
// warp) counters are turned into exclusive offsets, and every key goes to its
// counter's offset plus the number of lower lanes with the same digit (lanes
// with equal digits found with ballots, the lowest one advancing the counter).  Keys
// with equal high words then still sit in input order, so each run of equal
// high words is re-sorted by the full key (runs longer than 32 make the CTA
// bitonic-sort the whole segment instead).  256 threads; a and b hold cap
// keys each (cap a power of two >= n); cnt: 8 x 256 counters; sh: 34 words.
// Returns the buffer (a or b) holding the sorted keys.
// ---------------------------------------------------------------------------
constexpr int kSegRadixThreads = 256;
constexpr int kSegRadixWarps = kSegRadixThreads / 32;
constexpr int kRadixBatch = 4;  // rounds of 32 keys a warp loads and ranks before placing them

// Active lanes of the warp whose 8-bit digit equals this lane's (eight ballots).
__device__ __forceinline__ unsigned same_digit_lanes(uint32_t d, bool act) {
  unsigned m = __ballot_sync(0xffffffffu, act);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (d >> b) & 1u;
    const unsigned v = __ballot_sync(0xffffffffu, bit);
    m &= bit ? v : ~v;
  }
  return m;
}

__device__ __forceinline__ uint64_t* cta_radix_sort_hi32(uint64_t* a, uint64_t* b, int n, uint32_t* cnt,
                                                         uint32_t* sh) {
  const unsigned full = 0xffffffffu;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // 1. the high-word bits that differ
  uint32_t mn = 0xffffffffu, mx = 0u;
  for (int i = t; i < n; i += kSegRadixThreads) {
    const uint32_t h = (uint32_t)(a[i] >> 32);
    mn = min(mn, h);
    mx = max(mx, h);
  }
  mn = __reduce_min_sync(full, mn);
  mx = __reduce_max_sync(full, mx);
  if (lane == 0) {
    sh[warp] = mn;
    sh[kSegRadixWarps + warp] = mx;
  }
  __syncthreads();
  for (int w = 0; w < kSegRadixWarps; ++w) {
    mn = min(mn, sh[w]);
    mx = max(mx, sh[kSegRadixWarps + w]);
  }
  __syncthreads();  // sh is reused by the scans below
  const uint32_t diff = mn ^ mx;
  const int top = diff ? 64 - __clz(diff) : 32;  // sort bits [32, top)
  // 2. counting-sort passes over 8-bit digits
  const int per = (n + kSegRadixWarps - 1) / kSegRadixWarps;
  const int w0 = min(n, warp * per), w1 = min(n, w0 + per);
  const unsigned lower = (1u << lane) - 1u;
  uint32_t* wc = cnt + warp * 256;
  uint64_t* src = a;
  uint64_t* dst = b;
  for (int shift = 32; shift < top; shift += 8) {
    for (int i = t; i < kSegRadixWarps * 256; i += kSegRadixThreads) cnt[i] = 0u;
    __syncthreads();
    for (int i = w0 + lane; i < w1; i += 32) atomicAdd(&wc[(uint32_t)(src[i] >> shift) & 0xffu], 1u);
    __syncthreads();
    {
      const int d = t;  // one digit per thread
      uint32_t tot = 0u;
      for (int w = 0; w < kSegRadixWarps; ++w) tot += cnt[w * 256 + d];
      uint32_t off;
      block_excl_scan<kSegRadixThreads>(tot, off, sh);
      for (int w = 0; w < kSegRadixWarps; ++w) {
        const uint32_t c = cnt[w * 256 + d];
        cnt[w * 256 + d] = off;
        off += c;
      }
    }
    __syncthreads();
    for (int base = w0; base < w1; base += 32 * kRadixBatch) {
      uint64_t key[kRadixBatch];
      uint32_t dg[kRadixBatch];
      unsigned peers[kRadixBatch];
#pragma unroll
      for (int r = 0; r < kRadixBatch; ++r) {
        const int i = base + 32 * r + lane;
        const bool act = i < w1;
        key[r] = act ? src[i] : 0ull;
        dg[r] = (uint32_t)(key[r] >> shift) & 0xffu;
        peers[r] = same_digit_lanes(dg[r], act);
      }
#pragma unroll
      for (int r = 0; r < kRadixBatch; ++r) {
        if (base + 32 * r >= w1) break;  // warp-uniform
        const bool act = base + 32 * r + lane < w1;
        const unsigned before = peers[r] & lower;
        const uint32_t pos = act ? wc[dg[r]] + (uint32_t)__popc(before) : 0u;
        __syncwarp();
        if (act) {
          dst[pos] = key[r];
          if (before == 0u) wc[dg[r]] += (uint32_t)__popc(peers[r]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    uint64_t* tmp = src;
    src = dst;
    dst = tmp;
  }
  // 3. runs of equal high words, ordered by the full key
  bool long_run = false;
  for (int i = t + 1; i < n; i += kSegRadixThreads) {
    const uint32_t h = (uint32_t)(src[i] >> 32);
    if (h != (uint32_t)(src[i - 1] >> 32)) continue;
    if (i >= 2 && (uint32_t)(src[i - 2] >> 32) == h) continue;  // only the run's second key acts
    const int r0 = i - 1;
    int r1 = i + 1;
    while (r1 < n && (uint32_t)(src[r1] >> 32) == h && r1 - r0 <= 32) ++r1;
    if (r1 - r0 > 32) {
      long_run = true;
      continue;
    }
    for (int x = r0 + 1; x < r1; ++x) {  // insertion sort of a short run
      const uint64_t k = src[x];
      int y = x - 1;
      while (y >= r0 && src[y] > k) {
        src[y + 1] = src[y];
        --y;
      }
      src[y + 1] = k;
    }
  }
  if (__syncthreads_or(long_run)) {
    const int n2 = next_pow2(n);
    for (int i = n + t; i < n2; i += kSegRadixThreads) src[i] = ~0ull;
    __syncthreads();
    cta_bitonic_any(src, n2);
  }
  return src;
}

// Bucket sort by the high word's value range: the high words h are mapped
// linearly onto `bins` buckets, d = (h - min h) >> s (bins a power of two
// between n and kBucketBins, s the smallest shift that fits the range), a
// counting pass places every key of a[0, n) in its bucket of b (the order
// inside a bucket comes from shared atomics), and one thread per bucket
// insertion-sorts it by the full key.  The keys are distinct, so the result is
// the ascending order whatever the atomics did.  Returns b, or nullptr
// (uniformly over the CTA, a untouched) when a bucket would hold more than
// kBucketMax keys -- clustered depths, which the radix sort handles.
// cnt: kBucketBins counters; sh: 64 words.  All threads of the CTA.
constexpr int kBucketMax = 16;
constexpr int kBucketBins = kSegRadixWarps * 256;

__device__ __forceinline__ uint64_t* cta_bucket_sort_hi32(const uint64_t* a, uint64_t* b, int n, uint32_t* cnt,
                                                          uint32_t* sh) {
  const unsigned full = 0xffffffffu;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint32_t mn = 0xffffffffu, mx = 0u;
  for (int i = t; i < n; i += kSegRadixThreads) {
    const uint32_t h = (uint32_t)(a[i] >> 32);
    mn = min(mn, h);
    mx = max(mx, h);
  }
  mn = __reduce_min_sync(full, mn);
  mx = __reduce_max_sync(full, mx);
  if (lane == 0) {
    sh[warp] = mn;
    sh[kSegRadixWarps + warp] = mx;
  }
  const int bins = min(kBucketBins, max(32, next_pow2(n)));
  const int lb = 31 - __clz(bins);
  for (int i = t; i < bins; i += kSegRadixThreads) cnt[i] = 0u;
  __syncthreads();
  for (int w = 0; w < kSegRadixWarps; ++w) {
    mn = min(mn, sh[w]);
    mx = max(mx, sh[kSegRadixWarps + w]);
  }
  const uint32_t rng = mx - mn;
  const int width = rng ? 32 - __clz(rng) : 0;
  const int sft = max(0, width - lb);
  for (int i = t; i < n; i += kSegRadixThreads) atomicAdd(&cnt[((uint32_t)(a[i] >> 32) - mn) >> sft], 1u);
  __syncthreads();
  const int per = max(1, bins / kSegRadixThreads);  // consecutive buckets per thread
  const int b0 = t * per;
  uint32_t loc = 0u, bmax = 0u;
  for (int k = 0; k < per; ++k)
    if (b0 + k < bins) {
      const uint32_t c = cnt[b0 + k];
      loc += c;
      bmax = max(bmax, c);
    }
  bmax = __reduce_max_sync(full, bmax);
  if (lane == 0) sh[40 + warp] = bmax;
  uint32_t ex;
  block_excl_scan<kSegRadixThreads>(loc, ex, sh);  // its barriers also publish sh[40 ..]
  uint32_t gmax = 0u;
  for (int w = 0; w < kSegRadixWarps; ++w) gmax = max(gmax, sh[40 + w]);
  if (gmax > (uint32_t)kBucketMax) return nullptr;
  for (int k = 0; k < per; ++k)
    if (b0 + k < bins) {
      const uint32_t c = cnt[b0 + k];
      cnt[b0 + k] = ex;
      ex += c;
    }
  __syncthreads();
  for (int i = t; i < n; i += kSegRadixThreads) {
    const uint64_t key = a[i];
    b[atomicAdd(&cnt[((uint32_t)(key >> 32) - mn) >> sft], 1u)] = key;
  }
  __syncthreads();
  for (int d = t; d < bins; d += kSegRadixThreads) {  // bucket d now spans [end of d - 1, end of d)
    const int lo = d ? (int)cnt[d - 1] : 0, hi = (int)cnt[d];
    for (int x = lo + 1; x < hi; ++x) {
      const uint64_t k = b[x];
      int y = x - 1;
      while (y >= lo && b[y] > k) {
        b[y + 1] = b[y];
        --y;
      }
      b[y + 1] = k;
    }
  }
  __syncthreads();
  return b;
}

// Number of elements of the sorted run r[0, m) that are < key (or <= key).
__device__ __forceinline__ int rank_lt(const uint64_t* r, int m, uint64_t key) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (r[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int rank_le(const uint64_t* r, int m, uint64_t key) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (r[mid] <= key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Sort the segment in[0, n) (global) into out[0, n) (global).  tmp: global
// scratch of n keys.  sort_chunk(src, m) sorts the m <= cap keys src[0, m)
// (global) into shared memory and returns where they are; cap is a power of
// two.  `in` may alias `tmp` but not `out`.
template <class SortChunk>
__device__ void cta_sort_segment_with(const uint64_t* in, uint64_t* out, uint64_t* tmp, int n, int cap,
                                      SortChunk sort_chunk) {
  if (n <= cap) {
    const uint64_t* r = sort_chunk(in, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = r[i];
    __syncthreads();
    return;
  }
  // 1. sorted chunks of `cap` keys; choose the chunk destination so that the
  //    last merge level writes into `out`.
  int levels = 0;
  for (int L = cap; L < n; L <<= 1) ++levels;
  uint64_t* a = (levels & 1) ? tmp : out;
  uint64_t* b = (levels & 1) ? out : tmp;
  for (int c0 = 0; c0 < n; c0 += cap) {
    const int m = min(cap, n - c0);
    __syncthreads();
    const uint64_t* r = sort_chunk(in + c0, m);
    for (int i = threadIdx.x; i < m; i += blockDim.x) a[c0 + i] = r[i];
  }
  __syncthreads();
  // 2. merge runs of length L into runs of 2L
  for (int L = cap; L < n; L <<= 1) {
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int r0 = (e / (2 * L)) * (2 * L);
      const int mid = min(r0 + L, n);
      const int r1 = min(r0 + 2 * L, n);
      const uint64_t key = a[e];
      int pos;
      if (e < mid) pos = (e - r0) + rank_lt(a + mid, r1 - mid, key);   // ties: left run first
      else pos = (e - mid) + rank_le(a + r0, mid - r0, key);
      b[r0 + pos] = key;
    }
    __syncthreads();
    uint64_t* t = a;
    a = b;
    b = t;
  }
}

// The same with bitonic chunk sorts in smem[0, cap).
__device__ __forceinline__ void cta_sort_segment(const uint64_t* in, uint64_t* out, uint64_t* tmp, int n,
                                                 uint64_t* smem, int cap) {
  cta_sort_segment_with(in, out, tmp, n, cap, [smem](const uint64_t* src, int m) -> const uint64_t* {
    cta_sort_small(src, m, smem);
    return smem;
  });
}

}  // namespace splat
