// lre_assemble_noalloc: step (ii) without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need rho:
// an application whose own allocator has already reserved (nearly) all of
// the GPU's memory, a long-running service that forbids allocation on its
// request path because cudaMalloc can synchronise the device and its cost
// varies, or a host program that only accounts for memory it allocated
// itself.  lre_assemble needs FP64 scratch for its butterfly passes and
// takes it from a context's workspace, which lre_create and the call may
// have to allocate.  This variant takes its scratch from one fixed array that
// is part of the library's device image instead, and needs no context.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds it (32 MiB) until the process exits.  CUDA loads a library's
// device code and variables lazily by default, so that memory is taken when
// the first call on a device sets that device up: the set-up looks up the
// array's device address (in host code its name is only a host-side
// stand-in) and loads every assembly kernel the call may launch.  That first
// call therefore needs about 32 MiB of free device memory; make it at
// start-up, before the caller's allocator reserves the device, and before
// any stream capture.  Later calls on that device allocate nothing.  Every
// call shares the array, so calls that overlap on the GPU (different
// streams, or other host threads) race on it; serialise them.  Nothing in
// the array has to start at zero: every pass overwrites all of its output.
// A failure's text is kept per host thread (lre_last_error(NULL)).
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "lre_internal.cuh"

namespace {

constexpr int kNoallocMaxN = 10;
constexpr size_t kNoallocScratchBytes = ((size_t)2 * 16) << (2 * kNoallocMaxN);  // 32 MiB

static __device__ __align__(256) unsigned char g_assemble_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};
thread_local char g_error[256];  // text of this thread's last failure ("" if none)

lre_status fail(lre_status st, const char *what, cudaError_t e) {
  if (e != cudaSuccess)
    std::snprintf(g_error, sizeof g_error, "%s: %s", what, cudaGetErrorString(e));
  else
    std::snprintf(g_error, sizeof g_error, "%s", what);
  return st;
}

// Per-device set-up (the current device): the scratch array's device
// address, the assembly kernels loaded, and the SM count.
lre_status setup_device(int dev, void **scratch, int *sms) {
  if (dev < 0 || dev >= kMaxDevices) return fail(LRE_ERR_UNSUPPORTED, "device ordinal above 63", cudaSuccess);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_assemble_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return fail(LRE_ERR_CUDA, "cudaGetSymbolAddress(scratch array)", e);
    }
    if (lre::assemble_preload() != LRE_OK) {
      e = cudaGetLastError();
      return fail(LRE_ERR_CUDA, "loading the assembly kernels", e);
    }
    int n_sms = 0;
    e = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(LRE_ERR_CUDA, "cudaDeviceGetAttribute", e);
    }
    g_num_sms[dev] = n_sms;
    g_scratch_ptr[dev] = p;
  }
  *scratch = g_scratch_ptr[dev];
  *sms = g_num_sms[dev];
  return LRE_OK;
}

}  // namespace

namespace lre {
const char *noalloc_last_error() { return g_error; }
}  // namespace lre

extern "C" lre_status lre_assemble_noalloc(const double *theta, int n, lre_c64 *rho, lre_stream stream) {
  g_error[0] = '\0';
  if (!theta || !rho || n < 1) return fail(LRE_ERR_INVALID_ARG, "null pointer or n < 1", cudaSuccess);
  if (n > kNoallocMaxN)  // scratch would exceed the 32 MiB array
    return fail(LRE_ERR_UNSUPPORTED, "n above 10: the fixed scratch array holds n <= 10", cudaSuccess);
  static_assert(kNoallocScratchBytes == (size_t)2 * ((((size_t)16 << (2 * kNoallocMaxN)) + 255) & ~(size_t)255),
                "scratch size must equal the assembly workspace at the largest n");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(LRE_ERR_CUDA, "cudaGetDevice", e);
  }
  void *scratch = nullptr;
  int sms = 0;
  lre_status st = setup_device(dev, &scratch, &sms);
  if (st != LRE_OK) return st;
  lre_ctx local;  // host-side bookkeeping only: no device memory, no handles
  local.device = dev;
  local.num_sms = sms;
  if (lre::assemble_workspace_bytes(n) > kNoallocScratchBytes)
    return fail(LRE_ERR_UNSUPPORTED, "scratch above the fixed array", cudaSuccess);
  st = lre::assemble_run(&local, theta, n, rho, scratch, reinterpret_cast<cudaStream_t>(stream));
  if (st != LRE_OK) std::snprintf(g_error, sizeof g_error, "%s", local.last_error.c_str());
  return st;
}
