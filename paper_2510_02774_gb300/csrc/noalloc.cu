// Search-entry computation that allocates no device memory.
//
// grnnd_entry_point asks its caller for a few megabytes of device scratch.  Some callers
// cannot provide that at the moment they need the entry point: a host program whose GPU
// memory is entirely owned by its own arena and that is not allowed to call cudaMalloc,
// a latency-critical loop where cudaMalloc's implicit device-wide synchronisation is not
// acceptable, or a plugin that is handed device buffers but no allocator.  This variant
// keeps its scratch in one fixed array that lives in the library's device memory, so the
// caller passes only its inputs (the points) and its output (one int32).
//
// Costs and rules of the shared array:
//   * it occupies kNoAllocScratchBytes of device memory on every GPU that loads the
//     library, until the process exits;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it together with the
//     identity of the CUDA context that was current; a later call under another context
//     (after cudaDeviceReset, for instance, the module is loaded again and the array can
//     move) looks the address up again.  Make the first call on a device, and the first
//     after a reset, before any stream capture;
//   * every call on a device uses the same array and leaves its contents behind; each
//     kernel of the computation writes every scratch word it later reads, so nothing has
//     to start at zero;
//   * calls whose work overlaps on the GPU (different streams, or host threads without
//     ordering) race on the array: order them on one stream.
#include <mutex>
#include <string>

#include <cuda.h>

#include "grnnd.h"
#include "internal.h"

namespace {

constexpr int32_t kNoAllocMaxD = 1024;
// Layout of grnnd::launch_entry's workspace for d = 1024: 512 x 1024 column sums (FP64),
// the mean (1024 FP64), 512 block minima (FP64 + int32), each region 256-byte aligned.
constexpr size_t kNoAllocScratchBytes = 4208640;

static __device__ __align__(256) unsigned char g_entry_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
// Per device: the array's device address and the id of the context it was looked up under
// (context ids are never reused within a process, unlike context handles).
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Id of the current context, through the driver entry points that the runtime hands out (no
// link against the driver library).  Returns false if it cannot be read.
bool current_context_id(unsigned long long* id) {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
      cudaGetLastError();
      return false;
    }
    get_current = reinterpret_cast<GetCurrent>(f1);
    get_id = reinterpret_cast<GetId>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

int noalloc_fail(int code, const std::string& msg) {
  grnnd::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int grnnd_entry_point_noalloc(const float* points, int64_t n, int32_t d, int32_t ld,
                                         int32_t metric, int32_t* entry_out, void* stream) {
  if (!points || !entry_out) return noalloc_fail(GRNND_EINVAL, "points/entry_out is NULL");
  if (n < 1 || n > 0x7FFFFFFELL) return noalloc_fail(GRNND_EINVAL, "n out of range");
  if (d < 1 || ld < d || (ld & 3) != 0)
    return noalloc_fail(GRNND_EINVAL, "need d >= 1, ld >= d, ld % 4 == 0");
  if (d > kNoAllocMaxD)
    return noalloc_fail(GRNND_EINVAL, "grnnd_entry_point_noalloc supports d <= 1024 (its fixed "
                                      "scratch holds 512 x 1024 column sums); use grnnd_entry_point");
  if (((uintptr_t)points & 15u) != 0) return noalloc_fail(GRNND_EINVAL, "points must be 16-byte aligned");
  if (metric != GRNND_L2SQ && metric != GRNND_IP) return noalloc_fail(GRNND_EINVAL, "unknown metric");
  if (grnnd::entry_workspace_bytes(n, d) > kNoAllocScratchBytes)
    return noalloc_fail(GRNND_EINVAL, "entry workspace exceeds the fixed scratch");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(GRNND_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(GRNND_EINVAL, "device index above 63");
  // make the device's primary context current (it already is after any earlier runtime call
  // on this device), so that its id is readable; this initialises, it allocates nothing
  if ((e = cudaSetDevice(dev)) != cudaSuccess)
    return noalloc_fail(GRNND_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  unsigned long long ctx = 0;
  if (!current_context_id(&ctx)) return noalloc_fail(GRNND_ECUDA, "cannot read the current CUDA context");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
      // once per device and context, with that device current: the host-side name of the
      // array is not a device address, so ask the runtime for the real one.
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_entry_scratch);
      if (e != cudaSuccess || !p)
        return noalloc_fail(GRNND_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
      g_scratch_ctx[dev] = ctx;
    }
    scratch = g_scratch_addr[dev];
  }
  e = grnnd::launch_entry(points, n, d, ld, metric, entry_out, scratch, kNoAllocScratchBytes,
                          (cudaStream_t)stream);
  if (e != cudaSuccess) return noalloc_fail(GRNND_ECUDA, std::string("entry kernels: ") + cudaGetErrorString(e));
  return GRNND_OK;
}
