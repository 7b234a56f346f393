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
// library holds it (32 MiB) until the process exits.  In host code its name
// is only a host-side stand-in, so its device address is looked up once per
// device with cudaGetSymbolAddress (the first call on a device does that
// set-up; make that first call before any stream capture).  Every call
// shares the array, so calls that overlap on the GPU (different streams, or
// other host threads) race on it; serialise them.  Nothing in the array has
// to start at zero: every pass overwrites all of its output.
#include <cuda_runtime.h>

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

// Per-device set-up: the scratch array's device address and the SM count.
lre_status setup_device(int dev, void **scratch, int *sms) {
  if (dev < 0 || dev >= kMaxDevices) return LRE_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_assemble_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return LRE_ERR_CUDA;
    }
    int n_sms = 0;
    e = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return LRE_ERR_CUDA;
    }
    g_num_sms[dev] = n_sms;
    g_scratch_ptr[dev] = p;
  }
  *scratch = g_scratch_ptr[dev];
  *sms = g_num_sms[dev];
  return LRE_OK;
}

}  // namespace

extern "C" lre_status lre_assemble_noalloc(const double *theta, int n, lre_c64 *rho, lre_stream stream) {
  if (!theta || !rho || n < 1) return LRE_ERR_INVALID_ARG;
  if (n > kNoallocMaxN) return LRE_ERR_UNSUPPORTED;  // scratch would exceed the 32 MiB array
  static_assert(kNoallocScratchBytes == (size_t)2 * ((((size_t)16 << (2 * kNoallocMaxN)) + 255) & ~(size_t)255),
                "scratch size must equal the assembly workspace at the largest n");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LRE_ERR_CUDA;
  }
  void *scratch = nullptr;
  int sms = 0;
  lre_status st = setup_device(dev, &scratch, &sms);
  if (st != LRE_OK) return st;
  lre_ctx local;  // host-side bookkeeping only: no device memory, no handles
  local.device = dev;
  local.num_sms = sms;
  if (lre::assemble_workspace_bytes(n) > kNoallocScratchBytes) return LRE_ERR_UNSUPPORTED;
  return lre::assemble_run(&local, theta, n, rho, scratch, reinterpret_cast<cudaStream_t>(stream));
}
