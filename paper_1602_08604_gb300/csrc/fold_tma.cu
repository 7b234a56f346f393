// TMA-staged form of the fold passes after the first (Sec. III, Eq. 3): the
// same contraction as fold_item, one thread per output column, but the
// inputs of 32 consecutive columns arrive as one 5-D TMA box in shared
// memory instead of 3^J 2^J separate global loads per thread.
//
// A pass reads X[ah][al][oh][ol][c] (al in 3^J, ol in 2^J, c in C) and writes
// Y[ah][oh][pl][c].  A task is (ah, oh, 32 consecutive c): its box
// {32 c, 2^J ol, 1 oh, 3^J al, 1 ah} is 27 x 8 x 32 int32 = 27 KB for J = 3.
// Each warp runs its own task list with two buffers, so one box is always in
// flight per warp while the other is contracted (about 110 KB in flight per
// SM with four warps); lane l owns column c0 + l, reads its 3^J 2^J inputs
// from shared memory (consecutive lanes, consecutive words: no bank
// conflicts) and writes its 4^J outputs with the shared epilogue
// (fold_emit), coalesced across the warp.
#include <cuda_runtime.h>

#include <cudaTypedefs.h>

#include "lre_internal.cuh"
#include "passes.cuh"
#include "sm103.cuh"

namespace lre {
namespace {

using namespace passes;

constexpr int TC = 32;  // columns per task

// warps per CTA: four for J = 3 (a 27 KB box each, two buffers: 221 KB), 16
// for the smaller boxes of J <= 2, whose passes carry more arithmetic per byte
// (the final division of every coefficient)
template <int J>
__host__ __device__ constexpr int tma_warps() {
  return J == 3 ? 4 : 16;
}

// box bytes per task: int32 values, or split planes (2 + 1 bytes per value)
template <int J, bool PLANES = false>
__host__ __device__ constexpr int box_bytes() {
  return (J == 1 ? 3 : J == 2 ? 9 : 27) * (1 << J) * TC * (PLANES ? 3 : 4);
}

// PLANES: the input is split planes (map: the uint16 low halves, map_hi: the
// int8 high parts, one box of each per task on the same barrier).
template <int J, typename AccT, int MODE, bool PLANES>
__global__ void __launch_bounds__(tma_warps<J>() * 32, 1) fold_tma(const __grid_constant__ CUtensorMap map,
                                                                    const __grid_constant__ CUtensorMap map_hi,
                                                                    GenParams P) {
  constexpr int TMA_WARPS = tma_warps<J>();
  constexpr int NA = (J == 1) ? 3 : (J == 2) ? 9 : 27;
  constexpr int NO = 1 << J;
  constexpr int NP = 1 << (2 * J);
  constexpr int BOX = box_bytes<J, PLANES>();
  constexpr int BOX_LO = NA * NO * TC * 2;  // PLANES: the uint16 box, then the int8 box
  static_assert(!PLANES || BOX_LO % 128 == 0, "TMA destinations stay 128-byte aligned");
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((128u - (sm103::smem_addr(smem_raw) & 127u)) & 127u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t *buf = smem + warp * 2 * BOX;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + TMA_WARPS * 2 * BOX) + warp * 2;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + TMA_WARPS * 2 * BOX + TMA_WARPS * 16);
  __shared__ DivTables tab;
  if constexpr (MODE == M_FINAL_U) load_div_tables(P, tab);
  if (threadIdx.x == 0) *abort_flag = 0;
  if (lane == 0) {
    sm103::mbar_init(&bar[0], 1);
    sm103::mbar_init(&bar[1], 1);
    sm103::fence_barrier_init();
  }
  __syncthreads();

  const int64_t cblocks = P.C / TC;
  const int64_t tasks = P.items / TC;  // items = 3^(r-J) 2^(r-J) C
  const int64_t stride = (int64_t)gridDim.x * TMA_WARPS;
  const int64_t first = (int64_t)blockIdx.x * TMA_WARPS + warp;
  // PLANES: both boxes of every task are loaded (neighbouring tasks then run
  // in step and share the 256-byte L2 lines of both planes), but the high
  // plane holds values only where one of a task's letters can need it; the
  // others take the low 16 bits as int16
  auto with_hi = [&](int64_t task) {
    return PLANES && planes_hi_needed((task % cblocks) * TC, P.hi_from, P.hi_letters);
  };
  auto issue = [&](int64_t task, int b) {
    const int64_t ahoh = task / cblocks, cb = task - ahoh * cblocks;
    const int64_t ah = ahoh / P.n_oh, oh = ahoh - ah * P.n_oh;
    sm103::mbar_arrive_expect_tx(&bar[b], BOX);
    sm103::tma_load_5d(buf + b * BOX, &map, (int)(cb * TC), 0, (int)oh, 0, (int)ah, &bar[b]);
    if constexpr (PLANES)
      sm103::tma_load_5d(buf + b * BOX + BOX_LO, &map_hi, (int)(cb * TC), 0, (int)oh, 0, (int)ah, &bar[b]);
  };
  if (lane == 0 && first < tasks) issue(first, 0);
  int64_t i = 0;
  for (int64_t task = first; task < tasks; task += stride, ++i) {
    const int b = (int)(i & 1);
    const int64_t next = task + stride;
    if (next < tasks) {
      // the other buffer was read (generic proxy) in the previous iteration
      __syncwarp();
      sm103::fence_proxy_async_smem();
      if (lane == 0) issue(next, b ^ 1);
    }
    if (!sm103::mbar_wait(&bar[b], (uint32_t)((i >> 1) & 1), abort_flag)) {
      *abort_flag = 1;
      latch(P.status, LRE_ERR_TIMEOUT);
      break;
    }
    const int32_t *S = reinterpret_cast<const int32_t *>(buf + b * BOX);
    const unsigned short *SL = reinterpret_cast<const unsigned short *>(buf + b * BOX);
    const signed char *SH = reinterpret_cast<const signed char *>(buf + b * BOX + BOX_LO);
    const bool hi = with_hi(task);
    AccT acc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = 0;
#pragma unroll
    for (int al = 0; al < NA; ++al) {
      AccT v[NO];
#pragma unroll
      for (int ol = 0; ol < NO; ++ol) {
        const int idx = (al * NO + ol) * TC + lane;
        if constexpr (PLANES)
          v[ol] = hi ? (AccT)(int32_t)(((uint32_t)(int32_t)SH[idx] << 16) | (uint32_t)SL[idx])
                     : (AccT)(int16_t)SL[idx];
        else
          v[ol] = (AccT)S[idx];
      }
      wht<J>(v);
#pragma unroll
      for (int m = 0; m < NO; ++m) acc[block_pauli(al, m, J)] += v[m];
    }
    const int64_t ahoh = task / cblocks, cb = task - ahoh * cblocks;
    fold_emit<J, AccT, MODE>(P, acc, ahoh, cb * TC + lane, MODE == M_FINAL_U ? &tab : nullptr);
  }
  // no TMA may still write into shared memory when the CTA exits
  if (lane == 0) {
    for (int64_t q = i; q < i + 2; ++q) {
      const int64_t t = first + q * stride;
      if (t >= tasks) break;
      if (q == i && *abort_flag == 0) continue;  // loop ended normally: nothing outstanding
      for (uint32_t it = 0; it < sm103::kSpinLimit; ++it)
        if (sm103::mbar_try_wait(&bar[q & 1], (uint32_t)((q >> 1) & 1))) break;
    }
  }
  __syncwarp();
}

template <int J, typename AccT, int MODE, bool PLANES = false>
lre_status launch(lre_ctx *ctx, const CUtensorMap &map, const CUtensorMap &map_hi, const GenParams &P,
                  cudaStream_t s) {
  constexpr int TMA_WARPS = tma_warps<J>();
  constexpr int smem = TMA_WARPS * 2 * box_bytes<J, PLANES>() + TMA_WARPS * 16 + 16 + 128;
  auto k = fold_tma<J, AccT, MODE, PLANES>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int64_t tasks = P.items / TC;
  int64_t grid = (tasks + TMA_WARPS - 1) / TMA_WARPS;
  const int64_t cap = (int64_t)ctx->num_sms * (smem <= 110 * 1024 ? 2 : 1);
  if (grid > cap) grid = cap;
  k<<<(unsigned)grid, TMA_WARPS * 32, smem, s>>>(map, map_hi, P);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "TMA fold pass launch");
}

}  // namespace

lre_status passes::tma_pass(lre_ctx *ctx, const GenParams &P, int J, int in_t, int acc_t, int mode, bool weight,
                            cudaStream_t s) {
  if ((in_t != T_I32 && in_t != T_I24P) || J < 1 || J > 3 || P.C % TC != 0 || weight) return LRE_ERR_UNSUPPORTED;
  // final passes (the correctly rounded division of every coefficient) are
  // ALU-bound and run faster in the register-load kernel at full occupancy
  if (mode != M_STORE && mode != M_PARITY) return LRE_ERR_UNSUPPORTED;
  if (acc_t != T_I32 && acc_t != T_I64) return LRE_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(P.in) & 15) != 0) return LRE_ERR_UNSUPPORTED;
  const bool planes = in_t == T_I24P;
  if (planes && (J != 3 || mode != M_STORE || acc_t != T_I32)) return LRE_ERR_UNSUPPORTED;
  const int NA = J == 1 ? 3 : J == 2 ? 9 : 27, NO = 1 << J;
  const int64_t n_ah = ipow(3, P.r - J);
  // X[ah][al][oh][ol][c], innermost first
  const uint64_t dims[5] = {(uint64_t)P.C, (uint64_t)NO, (uint64_t)P.n_oh, (uint64_t)NA, (uint64_t)n_ah};
  const uint32_t box[5] = {TC, (uint32_t)NO, 1, (uint32_t)NA, 1};
  auto strides_of = [&](uint64_t e, uint64_t *st) {
    st[0] = (uint64_t)P.C * e;
    st[1] = (uint64_t)P.C * NO * e;
    st[2] = (uint64_t)P.C * NO * P.n_oh * e;
    st[3] = (uint64_t)P.C * NO * P.n_oh * NA * e;
  };
  CUtensorMap map, map_hi;
  uint64_t strides[4];
  if (planes) {
    const uint64_t elems = (uint64_t)P.C * NO * P.n_oh * NA * n_ah;
    strides_of(2, strides);
    if (!encode_tensor_map(&map, CU_TENSOR_MAP_DATA_TYPE_UINT16, P.in, 5, dims, strides, box))
      return LRE_ERR_UNSUPPORTED;
    strides_of(1, strides);
    if (!encode_tensor_map(&map_hi, CU_TENSOR_MAP_DATA_TYPE_UINT8, static_cast<const char *>(P.in) + elems * 2, 5,
                           dims, strides, box))
      return LRE_ERR_UNSUPPORTED;
    Launch L(ctx, "fold_tma", s);
    return launch<3, int32_t, M_STORE, true>(ctx, map, map_hi, P, s);
  }
  strides_of(4, strides);
  if (!encode_tensor_map_i32(&map, P.in, 5, dims, strides, box)) return LRE_ERR_UNSUPPORTED;
  map_hi = map;
  Launch L(ctx, "fold_tma", s);
  const bool i64 = acc_t == T_I64;
#define LRE_TMA_CASE(JJ)                                                                                  \
  if (J == JJ) {                                                                                          \
    if (mode == M_STORE)                                                                                  \
      return i64 ? launch<JJ, int64_t, M_STORE>(ctx, map, map_hi, P, s)                                   \
                 : launch<JJ, int32_t, M_STORE>(ctx, map, map_hi, P, s);                                  \
    return i64 ? launch<JJ, int64_t, M_PARITY>(ctx, map, map_hi, P, s)                                    \
               : launch<JJ, int32_t, M_PARITY>(ctx, map, map_hi, P, s);                                   \
  }
  LRE_TMA_CASE(1)
  LRE_TMA_CASE(2)
  LRE_TMA_CASE(3)
#undef LRE_TMA_CASE
  return LRE_ERR_UNSUPPORTED;
}

}  // namespace lre
