// noalloc.cu -- splat_bin_sort for callers that cannot allocate device memory.
//
// Some callers cannot hand the library a workspace: code that runs with a
// fixed device-memory budget reserved once at start-up (a real-time loop that
// must never enter the allocator), or a host framework whose allocator is not
// reachable from the place that issues the render.  For them this entry point
// runs the same binning and sort as splat_bin_sort, with its scratch taken
// from one statically sized device array that lives in this library's module.
//
// The array (kStaticScratchBytes) is allocated by the CUDA module loader on
// every device that loads the library and stays there until the process
// exits.  Host code cannot pass the array's symbol to a kernel (on the host
// the name stands for a host-side shadow, not a device address), so the
// device address is looked up with cudaGetSymbolAddress, with the device
// current: on the first call made on it, and again on every later call whose
// stream is not capturing (after a device reset the module, and with it the
// array, may sit at a new address).
#include <mutex>

#include "common.cuh"
#include "internal.cuh"

namespace splat {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_bin_sort_scratch[kStaticScratchBytes];

static std::mutex g_scratch_mu;
static void* g_scratch_ptr[kMaxDevices] = {nullptr};

static int static_scratch(cudaStream_t s, void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(SPLAT_ECUDA, "splat_bin_sort_static: no current CUDA device");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess)
    return fail(SPLAT_ECUDA, "splat_bin_sort_static: cudaStreamIsCapturing failed");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev] && cs != cudaStreamCaptureStatusNone)
    return fail(SPLAT_EINVAL, "splat_bin_sort_static: first call on device %d made during stream capture", dev);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_sort_scratch);
    if (e != cudaSuccess || !p)
      return fail(SPLAT_ECUDA, "splat_bin_sort_static: cudaGetSymbolAddress failed on device %d: %s", dev,
                  cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return SPLAT_OK;
}

}  // namespace splat

using namespace splat;

extern "C" size_t splat_bin_sort_static_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" int splat_bin_sort_static(const splat_projected* proj, int64_t n, const splat_camera* cam, uint64_t* keys,
                                     uint32_t* vals, int64_t capacity, int64_t* k_dev, uint32_t* ranges,
                                     int32_t* status, splat_stream_t stream) {
  if (!cam) return fail(SPLAT_EINVAL, "splat_bin_sort_static: null camera");
  if (n < 0 || capacity < 0) return fail(SPLAT_EINVAL, "splat_bin_sort_static: negative size");
  if (cam->width <= 0 || cam->height <= 0) return fail(SPLAT_EINVAL, "splat_bin_sort_static: bad image size");
  const CamK ck = make_camk(*cam);
  const int64_t n_tiles = (int64_t)ck.tiles_x * ck.tiles_y;
  const size_t need = splat_bin_sort_workspace_size(n, capacity, (int32_t)n_tiles);
  if (need == 0 || need > kStaticScratchBytes)
    return fail(SPLAT_EINVAL,
                "splat_bin_sort_static: n=%lld, capacity=%lld need %zu bytes of scratch, more than the %zu-byte "
                "static array; use splat_bin_sort with a caller workspace",
                (long long)n, (long long)capacity, need, kStaticScratchBytes);
  void* ws = nullptr;
  const int rc = static_scratch(reinterpret_cast<cudaStream_t>(stream), &ws);
  if (rc) return rc;
  return splat_bin_sort(proj, n, cam, keys, vals, capacity, k_dev, ranges, nullptr, status, ws, kStaticScratchBytes,
                        stream);
}
