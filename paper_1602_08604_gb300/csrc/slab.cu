// One instance of step (i) split over GPUs by the axis of qubit 1 (the basis
// groups of Sec. III partitioned by their first letter).
//
// A slab holds the 3^(n-1) bases whose qubit-1 axis is a.  Per qubit, the
// map T of Eq. (3) sends (a_1, o_1) to the Pauli letter p_1: I takes
// c(a_1, 0) + c(a_1, 1) from every axis, the letter a_1 + 1 takes
// c(a_1, 0) - c(a_1, 1) from axis a_1 only.  So with the slab's counts
// split by the outcome bit of qubit 1 (the most significant outcome bit),
// c0 = the first half of every row and c1 the second, the parity sums over
// qubits 2..n (the same fold, n - 1 qubits) of
//     c0 + c1   give the slab's share of the strings with p_1 = I, and
//     c0 - c1   give every string with p_1 = a + 1 (no other slab has them).
// The three shares of the p_1 = I block add up across slabs (one
// reduce-scatter); the final weight 1/(N 3^k) of Eq. (3) is lre_weight.
#include <cuda_runtime.h>

#include "lre_internal.cuh"
#include "passes.cuh"

namespace lre {
namespace {

// plus = c0 + c1, minus = c0 - c1 per row (rows of 2h counts in, h out).
template <typename InT, typename OutT>
__global__ void slab_split(const InT *__restrict__ c, int64_t rows, int64_t h, OutT *__restrict__ plus,
                           OutT *__restrict__ minus) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * h;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / h, o = e - r * h;
    const int32_t a = c[r * 2 * h + o], b = c[r * 2 * h + h + o];
    plus[e] = (OutT)(a + b);
    minus[e] = (OutT)(a - b);
  }
}

struct WeightArgs {
  double recip[16];
  int64_t dint[16];
};

// theta[j] = S[j] / (N 3^k(first + j)), correctly rounded (passes.cuh).
__global__ void weight_kernel(const int64_t *__restrict__ S, int n, int64_t first, int64_t count, WeightArgs W,
                              double *__restrict__ theta) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t i = (uint64_t)(first + j);
    int k = 0;
    for (int q = 0; q < n; ++q) k += ((i >> (2 * q)) & 3u) == 0;
    theta[j] = passes::div_int_rn(S[j], W.dint[k], W.recip[k]);
  }
}

}  // namespace
}  // namespace lre

using namespace lre;

extern "C" lre_status lre_slab_sums(lre_ctx *ctx, const void *slab, lre_count_kind kind, int n,
                                    int64_t row_total_bound, int64_t *ident, int64_t *own, lre_stream stream) {
  if (!ctx || !slab || !ident || !own || row_total_bound < 0) return LRE_ERR_INVALID_ARG;
  if (n < 2) return LRE_ERR_INVALID_ARG;
  if (n > 14) return LRE_ERR_UNSUPPORTED;
  if (kind != LRE_COUNTS_I32 && kind != LRE_COUNTS_I16) return LRE_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int m = n - 1;
  const int64_t rows = ipow(3, m), h = 1ll << m;
  // c0 + c1 and |c0 - c1| are bounded by the row total: int16 while it fits
  const bool narrow = row_total_bound > 0 && row_total_bound <= 32767;
  const lre_count_kind sk = narrow ? LRE_COUNTS_I16 : LRE_COUNTS_I32;
  const size_t half = (((size_t)rows * h * (narrow ? 2 : 4)) + 255) & ~(size_t)255;
  const size_t fold = fold_workspace_bytes(m, sk, false, row_total_bound, ctx->first_variant);
  lre_status st = ensure_workspace(ctx, fold + 2 * half);
  if (st != LRE_OK) return st;
  char *p = static_cast<char *>(ctx->ws);
  void *plus = p + fold, *minus = p + fold + half;
  const int grid = ctx->num_sms * 8;
  {
    Launch L(ctx, "slab_split", s);
    if (kind == LRE_COUNTS_I16 && narrow)
      slab_split<int16_t, int16_t><<<grid, 256, 0, s>>>(static_cast<const int16_t *>(slab), rows, h,
                                                         static_cast<int16_t *>(plus), static_cast<int16_t *>(minus));
    else if (kind == LRE_COUNTS_I16)
      slab_split<int16_t, int32_t><<<grid, 256, 0, s>>>(static_cast<const int16_t *>(slab), rows, h,
                                                         static_cast<int32_t *>(plus), static_cast<int32_t *>(minus));
    else if (narrow)
      slab_split<int32_t, int16_t><<<grid, 256, 0, s>>>(static_cast<const int32_t *>(slab), rows, h,
                                                         static_cast<int16_t *>(plus), static_cast<int16_t *>(minus));
    else
      slab_split<int32_t, int32_t><<<grid, 256, 0, s>>>(static_cast<const int32_t *>(slab), rows, h,
                                                         static_cast<int32_t *>(plus), static_cast<int32_t *>(minus));
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "slab split");
  FoldArgs a{plus, sk, m, nullptr, row_total_bound, nullptr, ident};
  if ((st = fold_run(ctx, a, ctx->ws, fold, s)) != LRE_OK) return st;
  // c0 - c1 has negative entries, which the tensor-core first pass does not
  // encode: this fold runs on the FWHT path
  FoldArgs b{minus, sk, m, nullptr, row_total_bound, nullptr, own};
  const int path = ctx->fold_path;
  ctx->fold_path = 0;
  st = fold_run(ctx, b, ctx->ws, fold, s);
  ctx->fold_path = path;
  return st;
}

extern "C" lre_status lre_weight(lre_ctx *ctx, const int64_t *S, int n, int64_t first, int64_t count, int64_t shots,
                                 double *theta, lre_stream stream) {
  if (!ctx || !S || !theta || count < 0 || first < 0 || shots <= 0) return LRE_ERR_INVALID_ARG;
  if (n < 1) return LRE_ERR_INVALID_ARG;
  if (n > 14) return LRE_ERR_UNSUPPORTED;
  if (first + count > ipow(4, n) || (double)shots * (double)ipow(3, n) >= 9007199254740992.0)
    return LRE_ERR_INVALID_ARG;
  if (count == 0) return LRE_OK;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  WeightArgs W;
  for (int k = 0; k < 16; ++k) {
    W.dint[k] = k <= n ? shots * ipow(3, k) : 1;
    W.recip[k] = 1.0 / (double)W.dint[k];  // host IEEE division
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int64_t blocks = (count + 255) / 256;
  if (blocks > (int64_t)ctx->num_sms * 32) blocks = (int64_t)ctx->num_sms * 32;
  Launch L(ctx, "weight", s);
  weight_kernel<<<(unsigned)blocks, 256, 0, s>>>(S, n, first, count, W, theta);
  e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "weight kernel");
}
