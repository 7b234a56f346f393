// Step (ii) of the LRE (arXiv:1602.08604 Eq. 4): rho = sum_i theta_i Omega_i
//   = (1/2^n) sum_P t_P P, evaluated as a butterfly over qubits.
//
// Per qubit the map from the Pauli letter coefficients (I, X, Y, Z) to the
// 2x2 block entries (row bit r, column bit c) is
//     (0,0) = (I + Z)/2   (0,1) = (X - iY)/2   (1,0) = (X + iY)/2   (1,1) = (I - Z)/2
// so rho = M^{(x)n} t.  The paper instead sums, for each output element, the
// 2^n strings sharing its nonzero pattern (Sec. IV, the 2^n x-mask groups);
// the butterfly reaches the same sums in O(n 4^n).  Passes transform J <= 2
// qubits each, lowest qubit first, in FP64; the last pass rounds once to
// complex64 and writes rho row-major.
//
// Layout after t qubits are done: [P_hi in 4^(n-t)][R_lo in 2^t][C_lo in 2^t]
// (complex128), so the final layout (t = n) is rho[R][C].
#include <cuda_runtime.h>

#include "lre_internal.cuh"

namespace lre {
namespace {

struct AsmParams {
  const void *in;
  void *out;
  int t;          // qubits already transformed
  int n;
  int64_t items;  // 4^(n-t-J) * 4^t
};

__device__ __forceinline__ void m_qubit(double2 vI, double2 vX, double2 vY, double2 vZ, double2 &o00,
                                        double2 &o01, double2 &o10, double2 &o11) {
  o00 = make_double2(0.5 * (vI.x + vZ.x), 0.5 * (vI.y + vZ.y));
  o11 = make_double2(0.5 * (vI.x - vZ.x), 0.5 * (vI.y - vZ.y));
  // -i*vY = (vY.y, -vY.x);  +i*vY = (-vY.y, vY.x)
  o01 = make_double2(0.5 * (vX.x + vY.y), 0.5 * (vX.y - vY.x));
  o10 = make_double2(0.5 * (vX.x - vY.y), 0.5 * (vX.y + vY.x));
}

template <int J, bool FIRST, bool LAST>
__global__ void __launch_bounds__(256) assemble_pass(AsmParams P) {
  constexpr int NP = 1 << (2 * J);
  const int t = P.t;
  const int tp = t + J;
  const int64_t L4 = 1ll << (2 * t);  // 4^t
  for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < P.items;
       item += (int64_t)gridDim.x * blockDim.x) {
    const int64_t L = item & (L4 - 1);
    const int64_t Pp = item >> (2 * t);
    const int64_t R_lo = L >> t, C_lo = L & ((1ll << t) - 1);
    double2 v[NP];
    const int64_t ibase = Pp * NP * L4 + L;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      if constexpr (FIRST) {
        v[p] = make_double2(__ldg(static_cast<const double *>(P.in) + ibase + p * L4), 0.0);
      } else {
        v[p] = __ldg(static_cast<const double2 *>(P.in) + ibase + p * L4);
      }
    }
    // digit 0 (qubit t): index p = p1*4 + p0 -> u0 = 2 r0 + c0
#pragma unroll
    for (int h = 0; h < NP / 4; ++h) {
      double2 a, b, c, d;
      m_qubit(v[4 * h + 0], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3], a, b, c, d);
      v[4 * h + 0] = a; v[4 * h + 1] = b; v[4 * h + 2] = c; v[4 * h + 3] = d;
    }
    if constexpr (J == 2) {
#pragma unroll
      for (int u0 = 0; u0 < 4; ++u0) {
        double2 a, b, c, d;
        m_qubit(v[u0], v[4 + u0], v[8 + u0], v[12 + u0], a, b, c, d);
        v[u0] = a; v[4 + u0] = b; v[8 + u0] = c; v[12 + u0] = d;
      }
    }
    // v[u1*4 + u0] with u_q = 2 r_q + c_q  ->  rj, cj
    const int64_t W = 1ll << tp;
    const int64_t obase = Pp * W * W;
#pragma unroll
    for (int u = 0; u < NP; ++u) {
      int rj, cj;
      if constexpr (J == 1) {
        rj = u >> 1;
        cj = u & 1;
      } else {
        const int u0 = u & 3, u1 = u >> 2;
        rj = ((u1 >> 1) << 1) | (u0 >> 1);
        cj = ((u1 & 1) << 1) | (u0 & 1);
      }
      const int64_t R = ((int64_t)rj << t) | R_lo;
      const int64_t Cc = ((int64_t)cj << t) | C_lo;
      const int64_t o = obase + R * W + Cc;
      if constexpr (LAST) {
        static_cast<float2 *>(P.out)[o] = make_float2((float)v[u].x, (float)v[u].y);
      } else {
        static_cast<double2 *>(P.out)[o] = v[u];
      }
    }
  }
}

template <int J>
void launch(bool first, bool last, const AsmParams &p, int grid, cudaStream_t s) {
  if (first && last) assemble_pass<J, true, true><<<grid, 256, 0, s>>>(p);
  else if (first) assemble_pass<J, true, false><<<grid, 256, 0, s>>>(p);
  else if (last) assemble_pass<J, false, true><<<grid, 256, 0, s>>>(p);
  else assemble_pass<J, false, false><<<grid, 256, 0, s>>>(p);
}

}  // namespace

size_t assemble_workspace_bytes(int n) {
  const size_t one = ((size_t)1 << (2 * n)) * sizeof(double2);
  return 2 * ((one + 255) & ~(size_t)255);
}

lre_status assemble_run(lre_ctx *ctx, const double *theta, int n, lre_c64 *rho, void *ws,
                        cudaStream_t s) {
  const size_t one = (((size_t)1 << (2 * n)) * sizeof(double2) + 255) & ~(size_t)255;
  char *bufs[2] = {static_cast<char *>(ws), static_cast<char *>(ws) + one};
  const void *in = theta;
  int t = 0, k = 0;
  while (t < n) {
    const int J = (n - t) >= 2 ? 2 : 1;
    const bool first = (t == 0), last = (t + J == n);
    AsmParams p;
    p.in = in;
    p.out = last ? static_cast<void *>(rho) : static_cast<void *>(bufs[k & 1]);
    p.t = t;
    p.n = n;
    p.items = (1ll << (2 * (n - t - J))) << (2 * t);
    int64_t blocks = (p.items + 255) / 256;
    const int64_t cap = (int64_t)ctx->num_sms * 32;
    if (blocks > cap) blocks = cap;
    {
      Launch L(ctx, last ? "assemble_last" : "assemble_pass", s);
      if (J == 2) launch<2>(first, last, p, (int)blocks, s);
      else launch<1>(first, last, p, (int)blocks, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "assemble pass launch");
    in = p.out;
    t += J;
    ++k;
  }
  return LRE_OK;
}

}  // namespace lre
