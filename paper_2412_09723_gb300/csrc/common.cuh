// common.cuh -- definitions shared by the kernels of the splat library.
//
// Build note: every translation unit is compiled with --fmad=false, so that a
// product followed by a sum is never fused behind the source's back.  Fused
// multiply-adds appear only where they are written (__fmaf_rn), at the places
// the operation-order specification names; this is what makes the tile rects,
// the sort keys, the alpha decisions and the maximum-weight ids reproducible
// bit for bit on any IEEE-754 implementation that follows the same order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/splat.h"

namespace splat {

constexpr int kTile = 16;
constexpr int kTilePixels = kTile * kTile;

// Rasterizer constants (the paper fixes none; 3DGS-style readings).
constexpr float kAlphaCap = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;
constexpr float kLowPass = 0.3f;
constexpr float kClip = 1.3f;
// Margin (in exponent units) below which the alpha floor is certainly missed;
// covers the error of logf and of the exponential (both far below 1e-5).
constexpr float kPowerCutMargin = 1e-3f;

// ----------------------------------------------------------------------------
// Exponential: Cody & Waite range reduction x = k ln2 + r (ln2 split in a
// 15-significant-bit head and a tail), exp(r) by the degree-7 Taylor
// polynomial in Horner form with fused multiply-adds, 2^k from exponent bits.
// ----------------------------------------------------------------------------
#if defined(SPLAT_FAST_EXP)
// Measurement build: the hardware exponential (not bit-exact with the oracle).
__device__ __forceinline__ float exp_core(float x) { return __expf(x); }
#else
__device__ __forceinline__ float exp_core(float x) {  // x in [-87, 88]
  // k = rint(x log2 e): adding 1.5 * 2^23 rounds to an integer (to nearest,
  // ties to even) and leaves k in the low mantissa bits
  const float t = __fadd_rn(__fmul_rn(x, 1.44269502f), 12582912.0f);
  const float k = __fsub_rn(t, 12582912.0f);
  float r = __fmaf_rn(-k, 0.693145751953125f, x);
  r = __fmaf_rn(-k, 1.42860677e-06f, r);
  float p = 1.98412701e-04f;
  p = __fmaf_rn(p, r, 1.38888892e-03f);
  p = __fmaf_rn(p, r, 8.33333377e-03f);
  p = __fmaf_rn(p, r, 4.16666679e-02f);
  p = __fmaf_rn(p, r, 1.66666672e-01f);
  p = __fmaf_rn(p, r, 0.5f);
  p = __fmaf_rn(p, r, 1.0f);
  p = __fmaf_rn(p, r, 1.0f);
  const int ki = __float_as_int(t) - 0x4B400000;
  return __fmul_rn(p, __int_as_float((ki + 127) << 23));
}
#endif

__device__ __forceinline__ float exp_full(float x) {
  if (x != x) return x;
  if (x > 88.0f) return __int_as_float(0x7f800000);
  if (x < -87.0f) return 0.0f;
  return exp_core(x);
}

// Status word helpers (sticky: only ever raised).
// Tile schedule layout (uint32): [0] = n_tiles once an order has been
// written, [1, 1 + n_tiles) = tile ids heaviest first, [1 + n_tiles,
// 1 + 2 n_tiles) = per-tile cost (summed contributor counts of the tile's
// pixels, written by the forward render).  Costs are ordered by bucket
// 1 + floor(8 log2 cost) (the float exponent and three mantissa bits; 0 for
// cost 0), heaviest bucket first.
constexpr int kCostBuckets = 128;
__device__ __forceinline__ int tile_cost_bucket(uint32_t S) {
  if (S == 0u) return 0;
  const int b = (int)((__float_as_uint((float)S) >> 20) - (127u << 3)) + 1;
  return b < kCostBuckets ? b : kCostBuckets - 1;
}
// The k-th tile of a view's schedule, or k when the schedule holds no order
// (or an entry out of range: a schedule written by anything but the binning).
__device__ __forceinline__ int schedule_tile(const uint32_t* sched, int n_tiles, int k) {
  if (!sched || sched[0] != (uint32_t)n_tiles) return k;
  const uint32_t t = sched[1 + k];
  return t < (uint32_t)n_tiles ? (int)t : k;
}

__device__ __forceinline__ void raise_status(int32_t* status, int32_t code) {
  if (status) atomicCAS(status, 0, code);
}

// ----------------------------------------------------------------------------
// Host-side error plumbing.
// ----------------------------------------------------------------------------
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);
int check_launch(const char* what);
// Launch accounting: construct a LaunchScope right before a kernel launch and
// let it end right after; it counts the launch and, while per-kernel timing is
// enabled, brackets it with CUDA events on `s`.
void count_launch(int n = 1);
class LaunchScope {
 public:
  LaunchScope(const char* name, cudaStream_t s);
  ~LaunchScope();
  LaunchScope(const LaunchScope&) = delete;
  LaunchScope& operator=(const LaunchScope&) = delete;

 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_;
};
#define SPLAT_LAUNCH(name, stream, ...)         \
  do {                                          \
    ::splat::LaunchScope splat_scope_(name, stream); \
    __VA_ARGS__;                                \
  } while (0)

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ----------------------------------------------------------------------------
// Device-wide primitives (binsort.cu).
// ----------------------------------------------------------------------------
// Exclusive prefix sum of n uint32 (n_dev, when not null, overrides n with a
// device-resident count <= n).  Scratch: scan_workspace_size(n) bytes.
size_t scan_workspace_size(int64_t n);
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* ws, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on bits [begin_bit, end_bit).
// Keys are uint32 or uint64, values uint32 (or absent: vals == nullptr).
// `count_dev` (optional) holds the number of valid items (<= capacity) on the
// device.  The result ends in (keys0, vals0) when the number of passes is even,
// else in (keys1, vals1); radix_sort returns 0 or 1 accordingly.
size_t radix_workspace_size(int64_t capacity);
template <typename Key>
int radix_sort(Key* keys0, uint32_t* vals0, Key* keys1, uint32_t* vals1, int64_t capacity,
               const int64_t* count_dev, int begin_bit, int end_bit, void* ws, cudaStream_t s,
               int* result_buffer);
int radix_passes(int begin_bit, int end_bit);

}  // namespace splat
