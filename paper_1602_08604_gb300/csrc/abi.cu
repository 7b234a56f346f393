// C ABI of liblre (declarations and documentation in include/lre.h):
// argument validation, the context and its workspace, and the count-ingest
// (shot-record histogram) kernel.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <new>
#include <string>

#include "lre_internal.cuh"

namespace lre {

lre_status cuda_fail(lre_ctx *ctx, cudaError_t e, const char *where) {
  if (ctx) ctx->last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return (e == cudaErrorMemoryAllocation) ? LRE_ERR_OOM : LRE_ERR_CUDA;
}

lre_status ensure_workspace(lre_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return LRE_OK;
  if (ctx->ws_limit != 0 && bytes > ctx->ws_limit) {
    ctx->last_error = "workspace of " + std::to_string(bytes) + " bytes exceeds the limit of " +
                      std::to_string(ctx->ws_limit);
    return LRE_ERR_OOM;
  }
  if (ctx->ws) {
    cudaError_t e = cudaFree(ctx->ws);  // implicit device synchronisation
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree(workspace)");
  }
  const size_t guard = ctx->canaries ? kCanaryBytes : 0;
  cudaError_t e = cudaMalloc(&ctx->ws, bytes + guard);
  if (e != cudaSuccess) {
    ctx->ws = nullptr;
    cudaGetLastError();
    return cuda_fail(ctx, e, "cudaMalloc(workspace)");
  }
  if (guard) {  // the pattern every kernel must leave alone
    e = cudaMemset(static_cast<char *>(ctx->ws) + bytes, kCanaryByte, guard);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "workspace guard");
  }
  ctx->ws_bytes = bytes;
  return LRE_OK;
}

Launch::Launch(lre_ctx *ctx, const char *name, cudaStream_t s, int own) : ctx_(ctx), s_(s) {
  ctx->launches += (uint64_t)own;
  if (!ctx->prof) return;
  if (ctx->prof_used == ctx->prof_pool.size()) {
    lre_prof_entry e{name, nullptr, nullptr};
    if (cudaEventCreate(&e.start) != cudaSuccess || cudaEventCreate(&e.stop) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    ctx->prof_pool.push_back(e);
  }
  idx_ = (long)ctx->prof_used++;
  ctx->prof_pool[idx_].name = name;
  cudaEventRecord(ctx->prof_pool[idx_].start, s);
}

Launch::~Launch() {
  if (idx_ >= 0) cudaEventRecord(ctx_->prof_pool[idx_].stop, s_);
}

namespace {

// One CTA per basis (grid-stride): a shared-memory histogram of the basis'
// shot records, then one coalesced write of its 2^n counts.
template <typename OutT>
__global__ void histogram_kernel(const uint16_t *__restrict__ rec, int64_t B, int64_t S, int n,
                                 OutT *__restrict__ counts, int *status) {
  extern __shared__ int32_t h[];
  const int d = 1 << n;
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    for (int o = threadIdx.x; o < d; o += blockDim.x) h[o] = 0;
    __syncthreads();
    const uint16_t *r = rec + b * S;
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
      const int o = r[s];
      if (o < d) atomicAdd(&h[o], 1);
      else latch(status, LRE_ERR_INVALID_ARG);
    }
    __syncthreads();
    OutT *c = counts + b * (int64_t)d;
    for (int o = threadIdx.x; o < d; o += blockDim.x) c[o] = (OutT)h[o];
    __syncthreads();
  }
}

// int16 counts (shots per basis <= 32767, so no bin carries into its
// neighbour): two bins per 32-bit word of shared memory, so a basis of n = 14
// takes 32 KB and seven CTAs fit an SM; zeroing and the store to HBM move 16
// bytes (eight bins) per thread, and VEC reads eight records per load.
template <bool VEC>
__global__ void __launch_bounds__(256) histogram16_kernel(const uint16_t *__restrict__ rec, int64_t B, int64_t S,
                                                         int n, int16_t *__restrict__ counts, int *status) {
  extern __shared__ uint4 h4[];
  uint32_t *h = reinterpret_cast<uint32_t *>(h4);
  const int d = 1 << n, nv = d >> 3;
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    for (int i = threadIdx.x; i < nv; i += blockDim.x) h4[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const uint16_t *r = rec + b * S;
    bool bad = false;
    auto add = [&](uint32_t o) {
      if (o < (uint32_t)d) atomicAdd(&h[o >> 1], 1u << ((o & 1u) << 4));
      else bad = true;
    };
    if constexpr (VEC) {
      const uint4 *r4 = reinterpret_cast<const uint4 *>(r);
      for (int64_t v = threadIdx.x; v < (S >> 3); v += blockDim.x) {
        const uint4 q = __ldcs(r4 + v);
        add(q.x & 0xFFFFu); add(q.x >> 16); add(q.y & 0xFFFFu); add(q.y >> 16);
        add(q.z & 0xFFFFu); add(q.z >> 16); add(q.w & 0xFFFFu); add(q.w >> 16);
      }
    } else {
      for (int64_t t = threadIdx.x; t < S; t += blockDim.x) add(r[t]);
    }
    if (bad) latch(status, LRE_ERR_INVALID_ARG);
    __syncthreads();
    uint4 *c = reinterpret_cast<uint4 *>(counts + b * (int64_t)d);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) c[i] = h4[i];
    __syncthreads();
  }
}

}  // namespace

lre_status histogram_run(lre_ctx *ctx, const uint16_t *records, int64_t num_bases,
                         int64_t shots_per_basis, int n, void *counts, lre_count_kind kind,
                         cudaStream_t s) {
  const size_t smem = sizeof(int32_t) << n;
  int grid = ctx->num_sms * 4;
  if (grid > num_bases) grid = (int)num_bases;
  Launch L(ctx, "histogram", s);
  if (kind == LRE_COUNTS_I16 && n >= 3 && (reinterpret_cast<uintptr_t>(counts) & 15) == 0) {
    const size_t smem16 = sizeof(int16_t) << n;
    int grid16 = ctx->num_sms * 8;
    if (grid16 > num_bases) grid16 = (int)num_bases;
    const bool vec = (shots_per_basis & 7) == 0 && (reinterpret_cast<uintptr_t>(records) & 15) == 0;
    auto k = vec ? histogram16_kernel<true> : histogram16_kernel<false>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem16);
    k<<<grid16, 256, smem16, s>>>(records, num_bases, shots_per_basis, n, static_cast<int16_t *>(counts),
                                  ctx->d_status);
  } else if (kind == LRE_COUNTS_I16) {
    cudaFuncSetAttribute(histogram_kernel<int16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    histogram_kernel<int16_t><<<grid, 512, smem, s>>>(records, num_bases, shots_per_basis, n,
                                                      static_cast<int16_t *>(counts), ctx->d_status);
  } else {
    cudaFuncSetAttribute(histogram_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    histogram_kernel<int32_t><<<grid, 512, smem, s>>>(records, num_bases, shots_per_basis, n,
                                                      static_cast<int32_t *>(counts), ctx->d_status);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "histogram launch");
}

}  // namespace lre

using namespace lre;

namespace {
constexpr int kMaxN = 14;

lre_status check_ctx(lre_ctx *ctx) { return ctx ? LRE_OK : LRE_ERR_INVALID_ARG; }

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

lre_status check_n(int n) {
  if (n < 1) return LRE_ERR_INVALID_ARG;
  if (n > kMaxN) return LRE_ERR_UNSUPPORTED;
  return LRE_OK;
}

lre_status set_device(lre_ctx *ctx) {
  cudaError_t e = cudaSetDevice(ctx->device);
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "cudaSetDevice");
}
}  // namespace

extern "C" {

lre_status lre_create(lre_ctx **out, int device) {
  if (!out) return LRE_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return LRE_ERR_INVALID_ARG;
  }
  lre_ctx *ctx = new (std::nothrow) lre_ctx();
  if (!ctx) return LRE_ERR_OOM;
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->mma_operand, lre::mma_operand_bytes());
  if (e != cudaSuccess) {
    lre_status st = cuda_fail(ctx, e, "lre_create");
    lre_destroy(ctx);
    return st;
  }
  lre_status st = lre::mma_operand_upload(ctx, ctx->mma_operand, nullptr);
  if (st == LRE_OK && (e = cudaStreamSynchronize(nullptr)) != cudaSuccess) st = cuda_fail(ctx, e, "lre_create");
  if (st != LRE_OK) {
    lre_destroy(ctx);
    return st;
  }
  *out = ctx;
  return LRE_OK;
}

void lre_destroy(lre_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->solver) cusolverDnDestroy(reinterpret_cast<cusolverDnHandle_t>(ctx->solver));
  if (ctx->blas) cublasDestroy(reinterpret_cast<cublasHandle_t>(ctx->blas));
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->mma_operand) cudaFree(ctx->mma_operand);
  for (auto &en : ctx->batch_cache) cudaFree(en.table);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  for (int k = 0; k < 2; ++k) {
    if (ctx->ev_copied[k]) cudaEventDestroy(ctx->ev_copied[k]);
    if (ctx->ev_free[k]) cudaEventDestroy(ctx->ev_free[k]);
  }
  if (ctx->ev_theta) cudaEventDestroy(ctx->ev_theta);
  for (auto &e : ctx->prof_pool) {
    cudaEventDestroy(e.start);
    cudaEventDestroy(e.stop);
  }
  delete ctx;
}

lre_status lre_set_workspace_limit(lre_ctx *ctx, size_t bytes) {
  if (check_ctx(ctx) != LRE_OK) return LRE_ERR_INVALID_ARG;
  ctx->ws_limit = bytes;
  return LRE_OK;
}

lre_status lre_workspace_size(lre_ctx *ctx, int n, lre_count_kind kind, int per_basis_shots,
                              size_t *bytes) {
  if (check_ctx(ctx) != LRE_OK || !bytes) return LRE_ERR_INVALID_ARG;
  lre_status st = check_n(n);
  if (st != LRE_OK) return st;
  if (kind != LRE_COUNTS_I32 && kind != LRE_COUNTS_I16 && kind != LRE_SHOTS_U16) return LRE_ERR_INVALID_ARG;
  if (kind == LRE_SHOTS_U16 && per_basis_shots) return LRE_ERR_INVALID_ARG;
  const lre_count_kind ck = kind == LRE_SHOTS_U16 ? LRE_COUNTS_I16 : kind;
  const size_t f = fold_workspace_bytes(n, ck, per_basis_shots != 0, per_basis_shots ? 0 : 1, ctx->first_variant);
  const size_t a = assemble_workspace_bytes(n);
  const size_t t = per_basis_shots ? 0 : up256((size_t)8 << (2 * n));  // exact-integer assembly
  const size_t dense = kind == LRE_SHOTS_U16 ? up256((size_t)ipow(3, n) * ((size_t)1 << n) * 2) : 0;
  *bytes = (f > a ? f : a) + t + dense;
  return LRE_OK;
}

lre_status lre_parity_sums(lre_ctx *ctx, const void *counts, lre_count_kind kind, int n,
                           int64_t row_total_bound, int64_t *S, lre_stream stream) {
  if (check_ctx(ctx) != LRE_OK || !counts || !S || row_total_bound < 0) return LRE_ERR_INVALID_ARG;
  lre_status st = check_n(n);
  if (st != LRE_OK) return st;
  if (kind != LRE_COUNTS_I32 && kind != LRE_COUNTS_I16) return LRE_ERR_INVALID_ARG;
  if ((st = set_device(ctx)) != LRE_OK) return st;
  // Without a bound every partial sum is int64.
  const size_t need = fold_workspace_bytes(n, kind, false, row_total_bound, ctx->first_variant);
  if ((st = ensure_workspace(ctx, need)) != LRE_OK) return st;
  FoldArgs a{counts, kind, n, nullptr, row_total_bound, nullptr, S};
  return fold_run(ctx, a, ctx->ws, ctx->ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

lre_status lre_estimate(lre_ctx *ctx, const void *counts, lre_count_kind kind, const int64_t *shots,
                        int64_t shots_uniform, int n, double *theta, lre_c64 *rho,
                        lre_stream stream) {
  if (check_ctx(ctx) != LRE_OK || !counts || !theta) return LRE_ERR_INVALID_ARG;
  lre_status st = check_n(n);
  if (st != LRE_OK) return st;
  if (kind != LRE_COUNTS_I32 && kind != LRE_COUNTS_I16 && kind != LRE_SHOTS_U16) return LRE_ERR_INVALID_ARG;
  if (!shots && shots_uniform <= 0) return LRE_ERR_INVALID_ARG;
  // shot records: uniform shots only; histogrammed into dense counts in the
  // workspace (int16 while a count cannot exceed 32767)
  const bool records = kind == LRE_SHOTS_U16;
  if (records && (shots || shots_uniform > INT32_MAX)) return LRE_ERR_INVALID_ARG;
  const lre_count_kind ck = records ? (shots_uniform <= 32767 ? LRE_COUNTS_I16 : LRE_COUNTS_I32) : kind;
  const size_t dense = records ? up256((size_t)ipow(3, n) * ((size_t)1 << n) * (ck == LRE_COUNTS_I16 ? 2 : 4)) : 0;
  if ((st = set_device(ctx)) != LRE_OK) return st;
  const size_t f = fold_workspace_bytes(n, ck, shots != nullptr, shots ? 0 : shots_uniform, ctx->first_variant);
  const size_t a = rho ? assemble_workspace_bytes(n) : 0;
  const size_t shared = f > a ? f : a;
  // uniform shots: rho is assembled from the exact integers T = S 3^(n-k)
  const bool int_asm = rho && !shots;
  const size_t tbytes = int_asm ? up256((size_t)8 << (2 * n)) : 0;
  if ((st = ensure_workspace(ctx, shared + tbytes + dense)) != LRE_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int64_t *T = int_asm ? reinterpret_cast<int64_t *>(static_cast<char *>(ctx->ws) + shared) : nullptr;
  if (records) {
    void *dc = static_cast<char *>(ctx->ws) + shared + tbytes;
    st = histogram_run(ctx, static_cast<const uint16_t *>(counts), ipow(3, n), shots_uniform, n, dc, ck, s);
    if (st != LRE_OK) return st;
    counts = dc;
    kind = ck;
  }
  FoldArgs fa{counts, kind, n, shots, shots_uniform, theta, nullptr};
  fa.T = T;
  if ((st = fold_run(ctx, fa, ctx->ws, shared, s)) != LRE_OK) return st;
  if (rho)
    st = int_asm ? assemble_int_run(ctx, T, n, shots_uniform, rho, ctx->ws, s)
                 : assemble_run(ctx, theta, n, rho, ctx->ws, s);
  return st;
}

lre_status lre_assemble(lre_ctx *ctx, const double *theta, int n, lre_c64 *rho, lre_stream stream) {
  if (check_ctx(ctx) != LRE_OK || !theta || !rho) return LRE_ERR_INVALID_ARG;
  lre_status st = check_n(n);
  if (st != LRE_OK) return st;
  if ((st = set_device(ctx)) != LRE_OK) return st;
  if ((st = ensure_workspace(ctx, assemble_workspace_bytes(n))) != LRE_OK) return st;
  return assemble_run(ctx, theta, n, rho, ctx->ws, reinterpret_cast<cudaStream_t>(stream));
}

lre_status lre_project(lre_ctx *ctx, const lre_c64 *rho_in, int n, lre_c64 *rho_out,
                       double *eig_mu, double *eig_rho, lre_stream stream) {
  if (check_ctx(ctx) != LRE_OK || !rho_in || !rho_out) return LRE_ERR_INVALID_ARG;
  lre_status st = check_n(n);
  if (st != LRE_OK) return st;
  if ((st = set_device(ctx)) != LRE_OK) return st;
  return project_run(ctx, rho_in, n, rho_out, eig_mu, eig_rho, reinterpret_cast<cudaStream_t>(stream));
}

lre_status lre_histogram(lre_ctx *ctx, const uint16_t *records, int64_t num_bases,
                         int64_t shots_per_basis, int n, void *counts, lre_count_kind kind,
                         lre_stream stream) {
  if (check_ctx(ctx) != LRE_OK || !records || !counts || num_bases <= 0 || shots_per_basis <= 0)
    return LRE_ERR_INVALID_ARG;
  lre_status st = check_n(n);
  if (st != LRE_OK) return st;
  if (kind != LRE_COUNTS_I32 && kind != LRE_COUNTS_I16) return LRE_ERR_INVALID_ARG;
  if (kind == LRE_COUNTS_I16 && shots_per_basis > 32767) return LRE_ERR_INVALID_ARG;
  if ((st = set_device(ctx)) != LRE_OK) return st;
  return histogram_run(ctx, records, num_bases, shots_per_basis, n, counts, kind,
                       reinterpret_cast<cudaStream_t>(stream));
}

lre_status lre_estimate_host(lre_ctx *ctx, const void *host_in, lre_host_kind host_kind,
                             int64_t shots_uniform, int n, double *theta_host, lre_c64 *rho_host,
                             lre_stream stream) {
  if (check_ctx(ctx) != LRE_OK || !host_in || !theta_host || shots_uniform <= 0)
    return LRE_ERR_INVALID_ARG;
  lre_status st = check_n(n);
  if (st != LRE_OK) return st;
  if (host_kind != LRE_HOST_COUNTS_I32 && host_kind != LRE_HOST_COUNTS_I16 &&
      host_kind != LRE_HOST_RECORDS_U16)
    return LRE_ERR_INVALID_ARG;
  if ((st = set_device(ctx)) != LRE_OK) return st;
  return estimate_host_run(ctx, host_in, host_kind, shots_uniform, n, theta_host, rho_host,
                           reinterpret_cast<cudaStream_t>(stream));
}

lre_status lre_sync(lre_ctx *ctx, lre_stream stream) {
  if (check_ctx(ctx) != LRE_OK) return LRE_ERR_INVALID_ARG;
  lre_status st = set_device(ctx);
  if (st != LRE_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int code = 0;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&code, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && code != 0) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lre_sync");
  return static_cast<lre_status>(code);
}

const char *lre_status_string(lre_status s) {
  switch (s) {
    case LRE_OK: return "ok";
    case LRE_ERR_INVALID_ARG: return "invalid argument";
    case LRE_ERR_UNSUPPORTED: return "unsupported size";
    case LRE_ERR_SHOTS_MISMATCH: return "counts do not add up to the stated shots";
    case LRE_ERR_OOM: return "out of device memory / workspace limit";
    case LRE_ERR_CUDA: return "CUDA error";
    case LRE_ERR_TIMEOUT: return "bounded device wait timed out";
    case LRE_ERR_EIG_FAILED: return "eigensolver failed";
  }
  return "unknown status";
}

const char *lre_last_error(lre_ctx *ctx) { return ctx ? ctx->last_error.c_str() : lre::noalloc_last_error(); }

lre_status lre_profile(lre_ctx *ctx, int enable) {
  if (check_ctx(ctx) != LRE_OK) return LRE_ERR_INVALID_ARG;
  ctx->prof = enable != 0;
  ctx->prof_used = 0;
  return LRE_OK;
}

int lre_profile_count(lre_ctx *ctx) { return ctx ? (int)ctx->prof_used : 0; }

lre_status lre_profile_get(lre_ctx *ctx, int i, const char **name, float *ms) {
  if (check_ctx(ctx) != LRE_OK || i < 0 || (size_t)i >= ctx->prof_used || !name || !ms)
    return LRE_ERR_INVALID_ARG;
  const lre_prof_entry &e = ctx->prof_pool[i];
  *name = e.name;
  cudaError_t err = cudaEventElapsedTime(ms, e.start, e.stop);
  return err == cudaSuccess ? LRE_OK : cuda_fail(ctx, err, "lre_profile_get");
}

uint64_t lre_launch_count(lre_ctx *ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"

// Test hook (not part of include/lre.h): choose the ALU first fold pass of
// later calls on this context: 0 register kernel, 1 TMA pipeline (the default), 2
// TMA pipeline fused with the second pass where the plan allows.
extern "C" lre_status lre_debug_set_first_pass(lre_ctx *ctx, int variant) {
  if (!ctx || variant < 0 || variant > 2) return LRE_ERR_INVALID_ARG;
  ctx->first_variant = variant;
  return LRE_OK;
}

// Test hook (not part of include/lre.h): CTAs that run the second pass in
// the fused tensor-core first pass (0: the default, a sixth of the SMs), and
// whether its second pass drops the ring lines it has read from L2 (1) or
// leaves them to be overwritten (0, the default).
extern "C" lre_status lre_debug_set_fused_consumers(lre_ctx *ctx, int ctas, int discard) {
  if (!ctx || ctas < 0 || (ctas > 0 && ctas >= ctx->num_sms) || discard < 0 || discard > 1)
    return LRE_ERR_INVALID_ARG;
  ctx->fused_consumers = ctas;
  ctx->fused_discard = discard;
  return LRE_OK;
}

// Test hook (not part of include/lre.h): 1 lets the raw tensor-core first
// pass of a whole fold (not a streamed one) fold seven qubits where it
// applies (n >= 8); 0 (the default) keeps it at six.
extern "C" lre_status lre_debug_set_first7(lre_ctx *ctx, int on) {
  if (!ctx || on < 0 || on > 1) return LRE_ERR_INVALID_ARG;
  ctx->first7 = on;
  return LRE_OK;
}

// Test hook (not part of include/lre.h): CTAs of the tensor-core first pass
// (0: one per SM, the default; fewer leave SMs idle, to measure how its rate
// grows with the SMs that run it).
extern "C" lre_status lre_debug_set_first_grid(lre_ctx *ctx, int ctas) {
  if (!ctx || ctas < 0 || ctas > ctx->num_sms) return LRE_ERR_INVALID_ARG;
  ctx->first_grid = ctas;
  return LRE_OK;
}

// Test hook (not part of include/lre.h): step (iii) through the default
// choice (1: the Krylov path from d = 2048 on when eig_mu is not asked for,
// else the eigenvalue-first path for d >= 64), always the eigenvalue-first
// path with its tridiagonal reduction (2), or always the full
// eigendecomposition (0).
extern "C" lre_status lre_debug_set_project_mode(lre_ctx *ctx, int mode) {
  if (!ctx || mode < 0 || mode > 2) return LRE_ERR_INVALID_ARG;
  ctx->project_mode = mode;
  return LRE_OK;
}

// Test hook (not part of include/lre.h): fold passes after the first read
// their inputs through TMA boxes in shared memory (1, the default, where the
// pass allows) or with per-thread global loads (0).
extern "C" lre_status lre_debug_set_generic_tma(lre_ctx *ctx, int on) {
  if (!ctx || on < 0 || on > 1) return LRE_ERR_INVALID_ARG;
  ctx->generic_tma = on;
  return LRE_OK;
}

// Test hook (not part of include/lre.h): lre_estimate_host with shot records
// takes the records-fed tensor-core first pass (no dense device counts)
// whenever it applies (1), or only when the workspace limit requires it (0,
// the default).
extern "C" lre_status lre_debug_set_records_direct(lre_ctx *ctx, int on) {
  if (!ctx || on < 0 || on > 1) return LRE_ERR_INVALID_ARG;
  ctx->records_direct = on;
  return LRE_OK;
}

// Test hook (not part of include/lre.h): bytes of host input per streamed
// chunk of lre_estimate_host (rounded to whole tile rows where the first pass
// runs per chunk); small values exercise many chunks on small inputs.
extern "C" lre_status lre_debug_set_host_chunk(lre_ctx *ctx, int64_t bytes) {
  if (!ctx || bytes <= 0) return LRE_ERR_INVALID_ARG;
  ctx->host_chunk_bytes = (size_t)bytes;
  return LRE_OK;
}

// Test hook (not part of include/lre.h): operand encoding of the tensor-core
// first pass: 0 counts below 2048 used as fp16 bit patterns (the default), 1
// counts below 1024 converted to fp16(1024 + c) in shared memory.
extern "C" lre_status lre_debug_set_mma_variant(lre_ctx *ctx, int biased) {
  if (!ctx || biased < 0 || biased > 1) return LRE_ERR_INVALID_ARG;
  ctx->mma_biased = biased;
  return LRE_OK;
}

// Test hook: set the batched schedule directly (any of the autotuner's
// candidates: jmax 2 or 3, 1 or 2 CTAs per SM, units that are multiples of
// 256 items).
extern "C" lre_status lre_debug_set_batch_schedule(lre_ctx *ctx, int jmax, int ctas_per_sm, int first_unit,
                                                   int unit) {
  if (!ctx || jmax < 2 || jmax > 3 || ctas_per_sm < 1 || ctas_per_sm > 2 || first_unit < 256 ||
      first_unit % 256 != 0 || unit < 256 || unit % 256 != 0)
    return LRE_ERR_INVALID_ARG;
  ctx->batch_jmax = jmax;
  ctx->batch_ctas_per_sm = ctas_per_sm;
  ctx->batch_first_unit = first_unit;
  ctx->batch_unit = unit;
  return LRE_OK;
}

extern "C" lre_status lre_batch_run(lre_ctx *ctx, const lre_instance *descs, int count, lre_stream stream) {
  if (!ctx) return LRE_ERR_INVALID_ARG;
  lre_status st = set_device(ctx);
  if (st != LRE_OK) return st;
  return lre::batch_run(ctx, descs, count, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" lre_status lre_batch_tune(lre_ctx *ctx, const lre_instance *descs, int count, lre_stream stream,
                                     float *best_ms) {
  if (!ctx) return LRE_ERR_INVALID_ARG;
  lre_status st = set_device(ctx);
  if (st != LRE_OK) return st;
  return lre::batch_tune(ctx, descs, count, reinterpret_cast<cudaStream_t>(stream), best_ms);
}

extern "C" lre_status lre_batch_schedule(const lre_ctx *ctx, int *jmax, int *ctas_per_sm, int *first_unit,
                                         int *unit) {
  if (!ctx) return LRE_ERR_INVALID_ARG;
  if (jmax) *jmax = ctx->batch_jmax;
  if (ctas_per_sm) *ctas_per_sm = ctx->batch_ctas_per_sm;
  if (first_unit) *first_unit = ctx->batch_first_unit;
  if (unit) *unit = ctx->batch_unit;
  return LRE_OK;
}

extern "C" lre_status lre_set_fold_path(lre_ctx *ctx, int path) {
  if (!ctx || (path != LRE_FOLD_FWHT && path != LRE_FOLD_TENSOR && path != LRE_FOLD_TENSOR_SPLIT))
    return LRE_ERR_INVALID_ARG;
  ctx->fold_path = path;
  return LRE_OK;
}

// Test hook (not part of include/lre.h): workspace canaries.  on = 1 frees
// the workspace and makes every later allocation carry a 64 KiB guard of a
// fixed byte pattern after its usable end; lre_debug_check_canaries
// synchronises the device and reports in *intact whether the guard is still
// whole (1) or some call wrote past the workspace (0) -- a substitute for a
// memory checker, on a pool where none runs.
extern "C" lre_status lre_debug_set_canaries(lre_ctx *ctx, int on) {
  if (!ctx || on < 0 || on > 1) return LRE_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LRE_ERR_CUDA;
  if (ctx->ws) {
    cudaError_t e = cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    for (auto &en : ctx->batch_cache) cudaFree(en.table);  // plans point into the old workspace
    ctx->batch_cache.clear();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree(workspace)");
  }
  ctx->canaries = on;
  return LRE_OK;
}

extern "C" lre_status lre_debug_check_canaries(lre_ctx *ctx, int *intact) {
  if (!ctx || !intact) return LRE_ERR_INVALID_ARG;
  *intact = 1;
  if (!ctx->canaries || !ctx->ws) return LRE_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LRE_ERR_CUDA;
  std::string host(kCanaryBytes, '\0');
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(&host[0], static_cast<char *>(ctx->ws) + ctx->ws_bytes, kCanaryBytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "workspace guard read");
  for (size_t i = 0; i < kCanaryBytes; ++i)
    if ((unsigned char)host[i] != kCanaryByte) {
      *intact = 0;
      break;
    }
  return LRE_OK;
}
