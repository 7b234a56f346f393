// The 4^n-operator variant of step (i) (Sec. VI: the measurement operators
// cut from the 6^n Pauli eigenprojectors to 4^n).  Operator set read as the
// minimal informationally complete subset |0>, |1>, |+>, |+i> per qubit, whose
// frequencies are Pauli counts: |0>, |1> from the Z basis, |+> from the X
// basis (outcome 0), |+i> from the Y basis (outcome 0).  The design matrix is
// square and invertible (X = X_1^{(x)n}, X^T X = G^{(x)n} not diagonal), so
// Eq. (3) is the exact solution of X theta = p: with uniform shots N, in
// Pauli-expectation units t_P = 2^{n/2} theta_P,
//     t = R^{(x)n} u / N,   R = [[1, 1, 0, 0], [-1, -1, 2, 0], [-1, -1, 0, 2], [1, -1, 0, 0]]
// (rows I, X, Y, Z; columns |0>, |1>, |+>, |+i>), u_j the count of operator j.
// Kernels: a gather of the 4^n used counts (only a fraction (2/3)^n of the
// count matrix is read), integer Kronecker passes of two qubits (exact int64,
// |sums| <= N 3^n), the last pass dividing by N (correctly rounded).
#include <cuda_runtime.h>

#include "lre_internal.cuh"
#include "passes.cuh"

namespace lre {
namespace {

// u[j] = counts[b(j)][o(j)], digit j_q (qubit 1 first) -> (axis, outcome):
// 0 -> (Z, 0), 1 -> (Z, 1), 2 -> (X, 0), 3 -> (Y, 0).
template <typename InT>
__global__ void ic4_gather(const InT *__restrict__ counts, int n, int64_t *__restrict__ u) {
  const int64_t P = 1ll << (2 * n), d = 1ll << n;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P; j += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = 0, o = 0;
    for (int q = n - 1; q >= 0; --q) {
      const int dq = (int)((j >> (2 * q)) & 3);
      b = 3 * b + (dq < 2 ? 2 : dq - 2);
      o = 2 * o + (dq == 1 ? 1 : 0);
    }
    u[j] = (int64_t)counts[b * d + o];
  }
}

__device__ __forceinline__ void r4(const int64_t (&x)[4], int64_t (&y)[4]) {
  const int64_t z = x[0] + x[1];
  y[0] = z;
  y[1] = 2 * x[2] - z;
  y[2] = 2 * x[3] - z;
  y[3] = x[0] - x[1];
}

// One or two qubits (t, t+1) of R^{(x)n}: thread per (hi, lo), hi the
// digits before t, lo the m = n - t - J digits after.  LAST: write
// theta = S / N instead of the sums.
template <int J, bool LAST>
__global__ void ic4_pass(const int64_t *__restrict__ in, void *__restrict__ out, int n, int t, int64_t shots,
                         double recip) {
  const int m = n - t - J;
  const int64_t lo_n = 1ll << (2 * m), items = (1ll << (2 * t)) * lo_n;
  constexpr int K = J == 2 ? 16 : 4;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t hi = it >> (2 * m), lo = it & (lo_n - 1);
    const int64_t base = (hi << (2 * (m + J))) + lo;
    int64_t v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = in[base + ((int64_t)k << (2 * m))];
    if constexpr (J == 2) {
      // k = 4 d1 + d2: R on d2 for each d1, then on d1 for each d2
#pragma unroll
      for (int d1 = 0; d1 < 4; ++d1) {
        int64_t x[4] = {v[4 * d1], v[4 * d1 + 1], v[4 * d1 + 2], v[4 * d1 + 3]}, y[4];
        r4(x, y);
#pragma unroll
        for (int d2 = 0; d2 < 4; ++d2) v[4 * d1 + d2] = y[d2];
      }
#pragma unroll
      for (int d2 = 0; d2 < 4; ++d2) {
        int64_t x[4] = {v[d2], v[4 + d2], v[8 + d2], v[12 + d2]}, y[4];
        r4(x, y);
#pragma unroll
        for (int d1 = 0; d1 < 4; ++d1) v[4 * d1 + d2] = y[d1];
      }
    } else {
      int64_t x[4] = {v[0], v[1], v[2], v[3]}, y[4];
      r4(x, y);
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = y[k];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = base + ((int64_t)k << (2 * m));
      if constexpr (LAST)
        static_cast<double *>(out)[o] = passes::div_int_rn(v[k], shots, recip);
      else
        static_cast<int64_t *>(out)[o] = v[k];
    }
  }
}

}  // namespace
}  // namespace lre

using namespace lre;

extern "C" lre_status lre_estimate_ic4(lre_ctx *ctx, const void *counts, lre_count_kind kind, int64_t shots_uniform,
                                       int n, double *theta, lre_c64 *rho, lre_stream stream) {
  if (!ctx || !counts || !theta || shots_uniform <= 0) return LRE_ERR_INVALID_ARG;
  if (n < 1) return LRE_ERR_INVALID_ARG;
  if (n > 14) return LRE_ERR_UNSUPPORTED;
  if (kind != LRE_COUNTS_I32 && kind != LRE_COUNTS_I16) return LRE_ERR_INVALID_ARG;
  if ((double)shots_uniform * (double)ipow(3, n) >= 9007199254740992.0) return LRE_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t vec = (((size_t)8 << (2 * n)) + 255) & ~(size_t)255;
  const size_t asmb = rho ? assemble_workspace_bytes(n) : 0;
  lre_status st = ensure_workspace(ctx, (2 * vec > asmb ? 2 * vec : asmb));
  if (st != LRE_OK) return st;
  int64_t *A = static_cast<int64_t *>(ctx->ws);
  int64_t *Bv = reinterpret_cast<int64_t *>(static_cast<char *>(ctx->ws) + vec);
  const int grid = ctx->num_sms * 8;
  {
    Launch L(ctx, "ic4_gather", s);
    if (kind == LRE_COUNTS_I16)
      ic4_gather<int16_t><<<grid, 256, 0, s>>>(static_cast<const int16_t *>(counts), n, A);
    else
      ic4_gather<int32_t><<<grid, 256, 0, s>>>(static_cast<const int32_t *>(counts), n, A);
  }
  const double recip = 1.0 / (double)shots_uniform;  // host IEEE division
  int64_t *cur = A, *nxt = Bv;
  for (int t = 0; t < n;) {
    const int J = (n - t) >= 2 ? 2 : 1;
    const bool last = (t + J == n);
    void *out = last ? static_cast<void *>(theta) : static_cast<void *>(nxt);
    Launch L(ctx, last ? "ic4_last" : "ic4_pass", s);
    if (J == 2 && last)
      ic4_pass<2, true><<<grid, 256, 0, s>>>(cur, out, n, t, shots_uniform, recip);
    else if (J == 2)
      ic4_pass<2, false><<<grid, 256, 0, s>>>(cur, out, n, t, shots_uniform, recip);
    else if (last)
      ic4_pass<1, true><<<grid, 256, 0, s>>>(cur, out, n, t, shots_uniform, recip);
    else
      ic4_pass<1, false><<<grid, 256, 0, s>>>(cur, out, n, t, shots_uniform, recip);
    t += J;
    int64_t *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "4^n-operator passes");
  return rho ? assemble_run(ctx, theta, n, rho, ctx->ws, s) : LRE_OK;
}
