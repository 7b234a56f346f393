// Step (ii) of the LRE (arXiv:1602.08604 Eq. 4): rho = sum_i theta_i Omega_i
//   = (1/2^n) sum_P t_P P, evaluated as a butterfly over qubits.
//
// Per qubit the map from the Pauli letter coefficients (I, X, Y, Z) to the
// 2x2 block entries (row bit r, column bit c) is
//     (0,0) = I + Z   (0,1) = X - iY   (1,0) = X + iY   (1,1) = I - Z
// (times 1/2), so rho = 2^-n M^{(x)n} t.  The paper instead sums, for each
// output element, the 2^n strings sharing its nonzero pattern (Sec. IV, the
// 2^n x-mask groups); the butterfly reaches the same sums in O(n 4^n).
//
// Two number types run the same passes:
//   * FP64 (lre_assemble on an arbitrary theta): FP64 butterflies with the
//     1/2 per qubit, rounded once to complex64 at the end;
//   * exact int64 (lre_estimate with uniform shots): the fold hands over
//     T_i = S_i 3^(n-k_i) = t_i N 3^n, integers; the butterflies are exact
//     integer adds and the last pass scales by 1/(2^n N 3^n) once.  GB300's
//     FP64 rate is far below its integer rate, and this path is also exact
//     until that single scaling.
//
// Layout after t qubits are done: [P_hi in 4^(n-t)][R_lo in 2^t][C_lo in 2^t],
// so the final layout (t = n) is rho[R][C].  For n >= 10 the passes are
// shared-memory tiled (6 qubits, then 4 at a time); smaller n and the
// leftover qubits use register passes of 1-2 qubits (passes.cuh).  From the
// tiled first pass on, each block of an intermediate is Hermitian and only
// its upper half by the low six bits (herm_upper) is stored and read, which
// cuts the intermediates' traffic by about 40 %; the last pass writes rho
// whole.
#include <cuda_runtime.h>

#include "lre_internal.cuh"
#include "passes.cuh"

namespace lre {
namespace {

using namespace passes;

// Register pass over J <= 2 qubits: one thread per (P', R_lo, C_lo).
// The entries of rho the Hermitian-half passes left out (herm_stored false),
// as the conjugates of their mirrors, one 64 x 64 block (A, B) at a time:
// the stored entries of block (B, A) that mirror its missing ones -- source
// row c from column 8 (c / 8 + 1) on, whole sectors -- go through shared
// memory and come out conjugated and transposed.  Blocks (A, B) and (B, A)
// read and write disjoint entries, so no two CTAs touch the same place.
__global__ void __launch_bounds__(256) assemble_mirror(float2 *__restrict__ rho, int64_t d) {
  __shared__ float2 tile[56][65];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nb = d >> 6;
  for (int64_t blk = blockIdx.x; blk < nb * nb; blk += gridDim.x) {
    const int64_t A = blk / nb, B = blk - A * nb;
    // warp w takes source rows c = w + 8 i (columns 8 (i + 1) .. 63) and target
    // rows r = 8 + w + 8 i (columns 0 .. 8 (i + 1) - 1): every bound is known
    // at compile time, so all fourteen loads of a thread are in flight at once
    const float2 *src = rho + (B * 64) * d + A * 64;  // block (B, A)
    float2 v[7][2];
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 8 * (i + 1) + lane + 32 * h;
        if (j < 64) v[i][h] = src[(int64_t)(warp + 8 * i) * d + j];
      }
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 8 * (i + 1) + lane + 32 * h;
        if (j < 64) tile[warp + 8 * i][j] = v[i][h];
      }
    __syncthreads();
    float2 *dst = rho + (A * 64) * d + B * 64;        // block (A, B)
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = 8 + warp + 8 * i, c = lane + 32 * h;
        if (c < 8 * (i + 1)) {
          const float2 z = tile[c][r];
          dst[(int64_t)r * d + c] = make_float2(z.x, -z.y);
        }
      }
    __syncthreads();
  }
}

template <class Num, int J, bool FIRST, bool LAST, bool HERM>
__global__ void __launch_bounds__(256) assemble_pass(AsmParams P) {
  for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < P.items;
       item += (int64_t)gridDim.x * blockDim.x)
    asm_item<Num, J, FIRST, LAST, HERM>(P, item);
}

// ---------------------------------------------------------------------------
// Shared-memory tiled passes (n >= 10): a 6-qubit first pass over contiguous
// blocks of 4096 coefficients (asm_low6_block in passes.cuh, shared with the
// batched kernel), then 4-qubit passes over 16-column strips.  Each thread
// holds 16 complex values (two qubits) per round; rounds exchange through
// shared memory (one padding element per 16: at most 4 wavefronts per
// 16-byte warp access).
// ---------------------------------------------------------------------------
constexpr int TILE_SMEM = ASM_TILE_SMEM;

// First pass: qubits 0..5 of each block of 4096 coefficients ->
// [R_lo 64][C_lo 64] per block (its stored part, herm_stored).
template <class Num>
__global__ void __launch_bounds__(256) assemble_low6(const typename Num::In *__restrict__ in,
                                                    typename Num::V *__restrict__ out, int64_t blocks) {
  using V = typename Num::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V *S = reinterpret_cast<V *>(smem_raw);  // 4096 + 256 padded entries
  for (int64_t blk = blockIdx.x; blk < blocks; blk += gridDim.x)
    asm_low6_block<Num, false, true>(in, out, blk, S, LastScale{0.f, 0.f});
}

// 4-qubit pass over qubits t..t+3 (t >= 6): unit = (P', R_lo, 16 consecutive
// C_lo).  Input [P'][p 256][R_lo][C_lo]; output [P'][R'][C'] with
// R' = (rJ << t) | R_lo, C' = (cJ << t) | C_lo.  Only the stored part is
// read and written (herm_stored): a strip whose 16 columns all lie outside it
// is skipped, a straddling strip is computed whole (its other columns read and
// write places nobody reads), and the last pass writes the stored entries of
// rho only (assemble_mirror fills the rest).
template <class Num, bool LAST>
__global__ void __launch_bounds__(256) assemble_high4(const typename Num::V *__restrict__ in,
                                                     void *__restrict__ out, int t, int64_t units,
                                                     LastScale scale) {
  using V = typename Num::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V *S = reinterpret_cast<V *>(smem_raw);
  const int tid = threadIdx.x;
  const int64_t side = 1ll << t;        // 2^t
  const int64_t L4 = side * side;       // 4^t
  const int64_t per_p = L4 / 16;        // units per P'
  const int64_t W = side << 4;          // 2^(t+4)
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t Pp = u / per_p;
    const int64_t L0 = (u - Pp * per_p) * 16;  // first L of the strip
    const int64_t R_lo = L0 >> t, C0 = L0 & (side - 1);
    if ((C0 & 63) + 15 < ((R_lo & 63) & ~7)) continue;  // no column of the strip is stored
    const V *src = in + Pp * 256 * L4 + L0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int e = tid + 256 * k;  // e = p * 16 + l
      S[pad16(e)] = src[(int64_t)(e >> 4) * L4 + (e & 15)];
    }
    __syncthreads();
    const int l = tid & 15, h = tid >> 4;
    V v[16];
    // round 1: digits 0,1 of p (p = d0 + 4 d1 + 16 (d2 + 4 d3))
#pragma unroll
    for (int w = 0; w < 16; ++w) v[w] = S[pad16(((w | (h << 4)) << 4) | l)];
    m2(v);
#pragma unroll
    for (int w = 0; w < 16; ++w) S[pad16(((w | (h << 4)) << 4) | l)] = v[w];
    __syncthreads();
    // round 2: digits 2,3 for fixed (u0,u1) = h
#pragma unroll
    for (int w = 0; w < 16; ++w) v[w] = S[pad16(((h | (w << 4)) << 4) | l)];
    m2(v);
    const int r0 = (h >> 1) & 1, c0 = h & 1, r1 = (h >> 3) & 1, c1 = (h >> 2) & 1;
#pragma unroll
    for (int w = 0; w < 16; ++w) {
      const int r2 = (w >> 1) & 1, c2 = w & 1, r3 = (w >> 3) & 1, c3 = (w >> 2) & 1;
      const int64_t rJ = r0 | (r1 << 1) | (r2 << 2) | (r3 << 3);
      const int64_t cJ = c0 | (c1 << 1) | (c2 << 2) | (c3 << 3);
      const int64_t Rp = (rJ << t) | R_lo, Cp = (cJ << t) | (C0 + l);
      const int64_t o = Pp * W * W + Rp * W + Cp;
      if constexpr (LAST) {
        if (herm_stored(R_lo, C0 + l)) static_cast<float2 *>(out)[o] = to_c64(v[w], scale);
      } else {
        static_cast<V *>(out)[o] = v[w];
      }
    }
    __syncthreads();
  }
}

// herm: the pass runs after the tiled first pass, on the stored half only
template <class Num, int J>
void launch_reg(bool first, bool last, bool herm, const AsmParams &p, int grid, cudaStream_t s) {
  if (first && last) assemble_pass<Num, J, true, true, false><<<grid, 256, 0, s>>>(p);
  else if (first) assemble_pass<Num, J, true, false, false><<<grid, 256, 0, s>>>(p);
  else if (last && herm) assemble_pass<Num, J, false, true, true><<<grid, 256, 0, s>>>(p);
  else if (last) assemble_pass<Num, J, false, true, false><<<grid, 256, 0, s>>>(p);
  else if (herm) assemble_pass<Num, J, false, false, true><<<grid, 256, 0, s>>>(p);
  else assemble_pass<Num, J, false, false, false><<<grid, 256, 0, s>>>(p);
}

template <class Num>
lre_status run_passes(lre_ctx *ctx, const typename Num::In *in0, int n, lre_c64 *rho, void *ws,
                      LastScale scale, cudaStream_t s) {
  using V = typename Num::V;
  const size_t one = (((size_t)1 << (2 * n)) * sizeof(V) + 255) & ~(size_t)255;
  char *bufs[2] = {static_cast<char *>(ws), static_cast<char *>(ws) + one};
  const void *in = in0;
  int t = 0, k = 0;
  if (n >= 10) {
    const int64_t blocks = 1ll << (2 * (n - 6));
    int grid = ctx->num_sms * 4;
    if (grid > blocks) grid = (int)blocks;
    {
      Launch L(ctx, "assemble_low6", s);
      cudaFuncSetAttribute(assemble_low6<Num>, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_SMEM);
      assemble_low6<Num><<<grid, 256, TILE_SMEM, s>>>(in0, reinterpret_cast<V *>(bufs[0]), blocks);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "assemble_low6 launch");
    in = bufs[0];
    t = 6;
    k = 1;
    while (n - t >= 4) {
      const bool last = (t + 4 == n);
      const int64_t units = (1ll << (2 * (n - t - 4))) * ((1ll << (2 * t)) / 16);
      int g = ctx->num_sms * 4;
      if (g > units) g = (int)units;
      void *out = last ? static_cast<void *>(rho) : static_cast<void *>(bufs[k & 1]);
      {
        Launch L(ctx, last ? "assemble_high4_last" : "assemble_high4", s);
        if (last) {
          cudaFuncSetAttribute(assemble_high4<Num, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_SMEM);
          assemble_high4<Num, true><<<g, 256, TILE_SMEM, s>>>(static_cast<const V *>(in), out, t, units, scale);
        } else {
          cudaFuncSetAttribute(assemble_high4<Num, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_SMEM);
          assemble_high4<Num, false><<<g, 256, TILE_SMEM, s>>>(static_cast<const V *>(in), out, t, units, scale);
        }
      }
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(ctx, e, "assemble_high4 launch");
      in = out;
      t += 4;
      ++k;
    }
  }
  while (t < n) {
    const int J = (n - t) >= 2 ? 2 : 1;
    const bool first = (t == 0), last = (t + J == n);
    AsmParams p;
    p.in = in;
    p.out = last ? static_cast<void *>(rho) : static_cast<void *>(bufs[k & 1]);
    p.t = t;
    p.n = n;
    p.items = (1ll << (2 * (n - t - J))) << (2 * t);
    p.scale = scale;
    int64_t blocks = (p.items + 255) / 256;
    const int64_t cap = (int64_t)ctx->num_sms * 32;
    if (blocks > cap) blocks = cap;
    {
      Launch L(ctx, last ? "assemble_last" : "assemble_pass", s);
      const bool herm = n >= 10;  // after the tiled first pass: the stored part only
      if (J == 2) launch_reg<Num, 2>(first, last, herm, p, (int)blocks, s);
      else launch_reg<Num, 1>(first, last, herm, p, (int)blocks, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "assemble pass launch");
    in = p.out;
    t += J;
    ++k;
  }
  if (n >= 10) {  // the Hermitian-half passes wrote the stored entries of rho only
    const int64_t nb = 1ll << (n - 6);
    int64_t g = (int64_t)ctx->num_sms * 8;
    if (g > nb * nb) g = nb * nb;
    {
      Launch L(ctx, "assemble_mirror", s);
      assemble_mirror<<<(int)g, 256, 0, s>>>(reinterpret_cast<float2 *>(rho), 1ll << n);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "assemble_mirror launch");
  }
  return LRE_OK;
}

}  // namespace

size_t assemble_workspace_bytes(int n) {
  const size_t one = ((size_t)1 << (2 * n)) * 16;  // complex128 or int64 pair
  return 2 * ((one + 255) & ~(size_t)255);
}

LastScaleArgs int_assembly_scale(int n, int64_t shots) {
  // 1 / (2^n N 3^n) split into two floats
  const double scale = 1.0 / ((double)(1ll << n) * (double)shots * (double)ipow(3, n));
  LastScaleArgs ls;
  ls.sh = (float)scale;
  ls.sl = (float)(scale - (double)ls.sh);
  return ls;
}

// Load every kernel assemble_run may launch into the current device's
// memory now (under lazy module loading a kernel's code is otherwise loaded,
// and its device memory taken, at its first launch).
lre_status assemble_preload() {
  const void *kernels[] = {
      reinterpret_cast<const void *>(assemble_low6<NumF64>),
      reinterpret_cast<const void *>(assemble_high4<NumF64, true>),
      reinterpret_cast<const void *>(assemble_high4<NumF64, false>),
      reinterpret_cast<const void *>(assemble_mirror),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 1, true, true, false>),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 1, true, false, false>),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 1, false, true, false>),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 1, false, false, false>),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 1, false, true, true>),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 1, false, false, true>),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 2, true, true, false>),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 2, true, false, false>),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 2, false, true, false>),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 2, false, false, false>),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 2, false, true, true>),
      reinterpret_cast<const void *>(assemble_pass<NumF64, 2, false, false, true>)};
  for (const void *k : kernels) {
    cudaFuncAttributes attr;
    if (cudaFuncGetAttributes(&attr, k) != cudaSuccess) return LRE_ERR_CUDA;
  }
  return LRE_OK;
}

lre_status assemble_run(lre_ctx *ctx, const double *theta, int n, lre_c64 *rho, void *ws,
                        cudaStream_t s) {
  return run_passes<NumF64>(ctx, theta, n, rho, ws, LastScale{0.f, 0.f}, s);
}

lre_status assemble_int_run(lre_ctx *ctx, const int64_t *T, int n, int64_t shots, lre_c64 *rho,
                            void *ws, cudaStream_t s) {
  const LastScaleArgs a = int_assembly_scale(n, shots);
  return run_passes<NumI64>(ctx, reinterpret_cast<const long long *>(T), n, rho, ws, LastScale{a.sh, a.sl}, s);
}

}  // namespace lre
