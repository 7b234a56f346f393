// Step (i) of the LRE (arXiv:1602.08604 Sec. III, Eq. 3): per-basis counts ->
// Pauli coefficients, as an atomic-free, mode-blocked Kronecker fold.
//
// With the diagonal X^T X of Sec. III the estimate of Pauli string P (support
// mask m, k identity letters) is
//     t_P = 1/(N 3^k) * sum_{bases a compatible with P} sum_o c_a(o) (-1)^{o.m}.
// Per qubit this is one fixed 4x6 integer map T from (axis a_q, outcome o_q)
// to the Pauli letter p_q:
//     I <- sum over all six;  X <- c(X,0)-c(X,1);  Y <- c(Y,0)-c(Y,1);  Z <- ...
// which factors as a 2-point Walsh-Hadamard butterfly over o_q (the parity
// transform, the paper's "nonzero matrix") followed by a ternary fold over
// a_q (the paper's "locations": I sums the three axes, X/Y/Z keep one).
// The whole step is T^{(x)n} applied to the [3^n][2^n] count tensor.  Passes
// apply it to a block of qubits at a time; every pass reads its input once
// and writes a tensor 2/3 smaller per contracted qubit.
//
// Tensor view before a pass with r qubits still to contract and C = 4^(n-r)
// coefficient columns already produced:
//     X[ah][al][oh][ol][c],   al in 3^J, ol in 2^J (the J qubits of the pass)
// and after it
//     Y[ah][oh][pl][c],       pl in 4^J,
// so the last pass leaves theta in the canonical order of Eq. (5).
//
// Which kernel runs which pass (fold_run):
//   first pass, int16 counts of at most 2047 shots: fold_first6_mma
//     (fold_mma.cu, tensor cores; split-plane partials when the next pass is
//     TMA-staged), or its records-fed form for lre_estimate_host;
//   first pass otherwise: fold_first6_pipe below (TMA pipeline on the ALU),
//     fold_first6 (register kernel, test hook) or the fused variant;
//   later store/parity passes: fold_tma (fold_tma.cu, TMA-staged) where the
//     columns allow, else fold_generic below;
//   the final pass: fold_generic with the divisor tables in shared memory
//     (the correctly rounded division in passes.cuh is ALU/FP64-bound).
#include <cuda_runtime.h>

#include <cudaTypedefs.h>

#include <vector>

#include "lre_internal.cuh"
#include "passes.cuh"
#include "sm103.cuh"

namespace lre {
namespace {

using namespace passes;

// ---------------------------------------------------------------------------
// Two-level first pass over the raw counts: 6 qubits per tile.
//   tile = (ah, oh): 729 basis rows x 64 consecutive outcomes.
//   level A (registers): 216 work items (alB in 27, olB in 8); each reads 27
//     rows x 8 outcomes (one 16 B vector per row for int16) and contracts the
//     three lowest qubits to 64 partial sums.
//   level B (shared memory): 64 work items (one per level-A Pauli digit
//     triple); each contracts the 27 x 8 level-A results over the next three
//     qubits and writes 64 int32 outputs.
// ---------------------------------------------------------------------------
constexpr int P1_THREADS = 256;
constexpr int P1_ZSTRIDE = 217;  // odd stride: conflict-free level-B reads

template <typename InT>
__device__ __forceinline__ void load_row8(const InT *p, int32_t (&v)[8]);

template <>
__device__ __forceinline__ void load_row8<int16_t>(const int16_t *p, int32_t (&v)[8]) {
  uint4 u = __ldcs(reinterpret_cast<const uint4 *>(p));
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = (int32_t)(int16_t)(w[k] & 0xffffu);
    v[2 * k + 1] = ((int32_t)w[k]) >> 16;
  }
}

template <>
__device__ __forceinline__ void load_row8<int32_t>(const int32_t *p, int32_t (&v)[8]) {
  int4 a = __ldcs(reinterpret_cast<const int4 *>(p));
  int4 b = __ldcs(reinterpret_cast<const int4 *>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

template <typename InT>
__global__ void __launch_bounds__(P1_THREADS, 2)
    fold_first6(const InT *__restrict__ counts, int32_t *__restrict__ out, int n,
                int64_t num_tiles) {
  extern __shared__ int32_t Z[];  // [64][P1_ZSTRIDE]
  const int t = threadIdx.x;
  const int64_t d = 1ll << n;
  const int64_t n_oh = d >> 6;
  for (int64_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
    const int64_t ah = tile / n_oh, oh = tile - ah * n_oh;
    if (t < 216) {
      const int alB = t >> 3, olB = t & 7;
      const InT *base = counts + (ah * 729 + alB * 27) * d + oh * 64 + olB * 8;
      int32_t acc[64];
#pragma unroll
      for (int p = 0; p < 64; ++p) acc[p] = 0;
#pragma unroll
      for (int alA = 0; alA < 27; ++alA) {
        int32_t v[8];
        load_row8<InT>(base + alA * d, v);
        wht<3>(v);
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[block_pauli(alA, m, 3)] += v[m];
      }
#pragma unroll
      for (int p = 0; p < 64; ++p) Z[p * P1_ZSTRIDE + t] = acc[p];
    }
    __syncthreads();
    if (t < 64) {
      int32_t acc[64];
#pragma unroll
      for (int p = 0; p < 64; ++p) acc[p] = 0;
      const int32_t *z = Z + t * P1_ZSTRIDE;
#pragma unroll
      for (int alB = 0; alB < 27; ++alB) {
        int32_t v[8];
#pragma unroll
        for (int olB = 0; olB < 8; ++olB) v[olB] = z[alB * 8 + olB];
        wht<3>(v);
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[block_pauli(alB, m, 3)] += v[m];
      }
      int32_t *o = out + tile * 4096 + t;
#pragma unroll
      for (int p = 0; p < 64; ++p) __stcs(o + p * 64, acc[p]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The same first pass as a warp-specialised TMA pipeline (the ALU first pass
// wherever the tensor-core one, fold_mma.cu, does not apply).
//   warp 0      producer: one 2D TMA load per sub-tile (81 rows x 64
//               outcomes = the two top ternary digits of the tile fixed) into
//               a ring of R shared-memory slots, completion on mbarriers.
//   warps 1..5  level A: one sub-tile per warp, lane = (a3, olB) for 24
//               lanes, 27 rows x 8 outcomes from shared memory -> 64 partial
//               sums -> exchange buffer Z[tile parity].
//   warps 6..7  level B: one thread per level-A Pauli triple, 27 x 8
//               partials -> 64 outputs -> HBM.
//   warps 8..9  (fused variant only) the second pass, see FUSE_* below.
// Loads never sit in registers, so up to R sub-tiles (R x 10.4 KB for int16)
// are in flight per SM while the ALU warps work.  Every wait is bounded; a
// timed-out wait latches LRE_ERR_TIMEOUT and the CTA drains and exits.
// ---------------------------------------------------------------------------
constexpr int PIPE_A_WARPS = 5;
constexpr int PIPE_THREADS = 32 * (1 + PIPE_A_WARPS + 2);
constexpr int SUB_ROWS = 81;
constexpr int Z_WORDS = 64 * P1_ZSTRIDE;

// Ring slots are owned by level-A warps (RW per warp): every wait is then at
// most one barrier phase ahead of the last completed one, which is what the
// parity test of mbarrier.try_wait.parity can tell apart.
template <typename InT>
struct PipeCfg {
  static constexpr int RW = sizeof(InT) == 2 ? 2 : 1;  // slots per level-A warp
  static constexpr int R = PIPE_A_WARPS * RW;           // ring slots
  static constexpr int SUB_BYTES = SUB_ROWS * 64 * (int)sizeof(InT);
  static constexpr int RING_BYTES = R * SUB_BYTES;
  static constexpr int Z_OFF = RING_BYTES;
  static constexpr int BAR_OFF = Z_OFF + 2 * Z_WORDS * 4;
  static constexpr int SMEM = BAR_OFF + (2 * R + 4) * 8 + 16 + 1024;  // + alignment slack
};

// Fused first + second pass (6 + 3 qubits): first-pass tiles are processed
// group-major, a group being the 27 x 8 tiles (qubits 6..8 of the a-digits
// and o-bits) that one second-pass column reads; tile outputs go to a ring of
// FUSE_RING group slots that stays in L2 and is read back by 32-column jobs
// of two extra warps per CTA once the group's tile counter is complete.
constexpr int FUSE_RING = 8;
constexpr int FUSE_JOBS = 4096 / 32;  // second-pass jobs per group
constexpr int FUSE_THREADS = PIPE_THREADS + 64;

struct FuseState {  // zeroed before each launch; counters only grow
  unsigned int job_next;
  unsigned int tiles_done[FUSE_RING];
  unsigned int jobs_done[FUSE_RING];
};

struct PipeArgs {
  int32_t *out;      // first pass: [tiles][4096]; fused: second-pass output [groups][64][4096]
  int32_t *scratch;  // fused: [FUSE_RING][216][4096]
  FuseState *fs;     // fused
  int fuse;
  int n;
  int64_t tile_begin, tile_end, row_base;
  int *status;
};

__device__ __forceinline__ void tile_coords(int fuse, int64_t q, int64_t n_oh, int64_t &ah, int64_t &oh) {
  if (!fuse) {
    ah = q / n_oh;
    oh = q - ah * n_oh;
    return;
  }
  const int64_t G = q / 216, k = q - G * 216, n_goh = n_oh >> 3;
  const int64_t gah = G / n_goh, goh = G - gah * n_goh;
  ah = gah * 27 + k / 8;
  oh = goh * 8 + (k & 7);
}

// Wait (bounded by time) until *p >= target; acquire ordering.
__device__ __forceinline__ bool poll_at_least(unsigned int *p, unsigned int target, volatile int *abort) {
  const uint64_t t0 = sm103::globaltimer();
  for (uint32_t it = 0;; ++it) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    if (v >= target) return true;
    if ((it & 63u) == 63u) {
      if (*abort || sm103::globaltimer() - t0 > sm103::kWaitNs) return false;
      __nanosleep(64);
    }
  }
}

template <typename InT>
__device__ __forceinline__ void lds_row8(const InT *p, int32_t (&v)[8]);

template <>
__device__ __forceinline__ void lds_row8<int16_t>(const int16_t *p, int32_t (&v)[8]) {
  const uint4 u = *reinterpret_cast<const uint4 *>(p);
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = (int32_t)(int16_t)(w[k] & 0xffffu);
    v[2 * k + 1] = ((int32_t)w[k]) >> 16;
  }
}

template <>
__device__ __forceinline__ void lds_row8<int32_t>(const int32_t *p, int32_t (&v)[8]) {
  const int4 a = reinterpret_cast<const int4 *>(p)[0];
  const int4 b = reinterpret_cast<const int4 *>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

template <typename InT, bool FUSE>
__global__ void __launch_bounds__(FUSE ? FUSE_THREADS : PIPE_THREADS, 1)
    fold_first6_pipe(const __grid_constant__ CUtensorMap tmap, PipeArgs A) {
  int32_t *__restrict__ out = A.out;
  const int n = A.n;
  const int64_t tile_begin = A.tile_begin, tile_end = A.tile_end, row_base = A.row_base;
  int *status = A.status;
  using Cfg = PipeCfg<InT>;
  constexpr int R = Cfg::R;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // TMA destinations must be 128-byte aligned: align the base explicitly
  uint8_t *smem = smem_raw + ((1024u - (sm103::smem_addr(smem_raw) & 1023u)) & 1023u);
  InT *ring = reinterpret_cast<InT *>(smem);
  int32_t *Z = reinterpret_cast<int32_t *>(smem + Cfg::Z_OFF);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + Cfg::BAR_OFF);
  uint64_t *empty = full + R;
  uint64_t *zfull = empty + R;
  uint64_t *zempty = zfull + 2;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(zempty + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_oh = (1ll << n) >> 6;
  if (threadIdx.x == 0) {
    for (int i = 0; i < R; ++i) {
      sm103::mbar_init(&full[i], 1);
      sm103::mbar_init(&empty[i], 32);
    }
    for (int b = 0; b < 2; ++b) {
      sm103::mbar_init(&zfull[b], 9 * 32);
      sm103::mbar_init(&zempty[b], 64);
    }
    *abort_flag = 0;
    sm103::fence_barrier_init();
  }
  __syncthreads();
  auto give_up = [&]() {
    *abort_flag = 1;
    latch(status, LRE_ERR_TIMEOUT);
  };

  if (warp == 0) {
    if (lane == 0) {
      // sub-tile g goes to warp g % NA, its j-th item (j = g / NA), slot
      // w*RW + j % RW, fill f = j / RW of that slot
      int64_t g = 0;
      for (int64_t tile = tile_begin + blockIdx.x; tile < tile_end && !*abort_flag; tile += gridDim.x) {
        int64_t ah, oh;
        tile_coords(FUSE ? 1 : 0, tile, n_oh, ah, oh);
        for (int s = 0; s < 9; ++s, ++g) {
          const int w = (int)(g % PIPE_A_WARPS);
          const int64_t j = g / PIPE_A_WARPS;
          const int slot = w * Cfg::RW + (int)(j % Cfg::RW);
          const int64_t f = j / Cfg::RW;
          if (f > 0 && !sm103::mbar_wait(&empty[slot], (uint32_t)((f - 1) & 1), abort_flag)) {
            give_up();
            break;
          }
          sm103::mbar_arrive_expect_tx(&full[slot], Cfg::SUB_BYTES);
          sm103::tma_load_2d(ring + (size_t)slot * (Cfg::SUB_BYTES / sizeof(InT)), &tmap, (int)(oh * 64),
                             (int)(ah * 729 + s * SUB_ROWS - row_base), &full[slot]);
        }
      }
      // drain: every issued load must land before the CTA may exit; only the
      // last fill of each slot can still be in flight
      for (int slot = 0; slot < R; ++slot) {
        const int w = slot / Cfg::RW, r = slot % Cfg::RW;
        // number of items of warp w issued: ceil((g - w) / NA); fills of this slot:
        const int64_t items = g > w ? (g - w + PIPE_A_WARPS - 1) / PIPE_A_WARPS : 0;
        const int64_t fills = items > r ? (items - r + Cfg::RW - 1) / Cfg::RW : 0;
        if (fills == 0) continue;
        for (uint32_t it = 0; it < sm103::kSpinLimit; ++it)
          if (sm103::mbar_try_wait(&full[slot], (uint32_t)((fills - 1) & 1))) break;
      }
    }
  } else if (warp <= PIPE_A_WARPS) {
    const int wa = warp - 1;
    for (int64_t j = 0;; ++j) {
      const int64_t g = wa + PIPE_A_WARPS * j;
      const int64_t lt = g / 9;
      const int s = (int)(g - lt * 9);
      const int64_t tile = tile_begin + blockIdx.x + lt * gridDim.x;
      if (tile >= tile_end) break;
      const int slot = wa * Cfg::RW + (int)(j % Cfg::RW);
      if (!sm103::mbar_wait(&full[slot], (uint32_t)((j / Cfg::RW) & 1), abort_flag)) {
        give_up();
        break;
      }
      const int zb = (int)(lt & 1);
      if (lt >= 2 && !sm103::mbar_wait(&zempty[zb], (uint32_t)(((lt >> 1) - 1) & 1), abort_flag)) {
        give_up();
        break;
      }
      if (lane < 24) {
        const int a3 = lane >> 3, olB = lane & 7;
        const InT *src = ring + (size_t)slot * (Cfg::SUB_BYTES / sizeof(InT)) + a3 * 27 * 64 + olB * 8;
        int32_t acc[64];
#pragma unroll
        for (int p = 0; p < 64; ++p) acc[p] = 0;
#pragma unroll
        for (int alA = 0; alA < 27; ++alA) {
          int32_t v[8];
          lds_row8<InT>(src + alA * 64, v);
          wht<3>(v);
#pragma unroll
          for (int m = 0; m < 8; ++m) acc[block_pauli(alA, m, 3)] += v[m];
        }
        int32_t *z = Z + zb * Z_WORDS + s * 24 + lane;
#pragma unroll
        for (int p = 0; p < 64; ++p) z[p * P1_ZSTRIDE] = acc[p];
      }
      sm103::mbar_arrive(&empty[slot]);
      sm103::mbar_arrive(&zfull[zb]);
    }
  } else if (warp < PIPE_A_WARPS + 3) {
    const int tb = threadIdx.x - 32 * (PIPE_A_WARPS + 1);  // 0..63
    for (int64_t lt = 0;; ++lt) {
      const int64_t tile = tile_begin + blockIdx.x + lt * gridDim.x;
      if (tile >= tile_end) break;
      const int zb = (int)(lt & 1);
      if (!sm103::mbar_wait(&zfull[zb], (uint32_t)((lt >> 1) & 1), abort_flag)) {
        give_up();
        break;
      }
      int32_t *dst = out + tile * 4096;
      int slot = 0;
      if constexpr (FUSE) {
        // ring slot of this tile's group; wait until the slot's previous group
        // has been read by all of its second-pass jobs
        const int64_t G = tile / 216;
        slot = (int)(G % FUSE_RING);
        const uint32_t need = (uint32_t)(FUSE_JOBS * (G / FUSE_RING));
        if (need && !poll_at_least(&A.fs->jobs_done[slot], need, abort_flag)) {
          give_up();
          break;
        }
        dst = A.scratch + ((int64_t)slot * 216 + (tile - G * 216)) * 4096;
      }
      const int32_t *z = Z + zb * Z_WORDS + tb * P1_ZSTRIDE;
      int32_t acc[64];
#pragma unroll
      for (int p = 0; p < 64; ++p) acc[p] = 0;
#pragma unroll
      for (int alB = 0; alB < 27; ++alB) {
        int32_t v[8];
#pragma unroll
        for (int olB = 0; olB < 8; ++olB) v[olB] = z[alB * 8 + olB];
        wht<3>(v);
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[block_pauli(alB, m, 3)] += v[m];
      }
      sm103::mbar_arrive(&zempty[zb]);
      int32_t *o = dst + tb;
      if constexpr (FUSE) {
#pragma unroll
        for (int p = 0; p < 64; ++p) o[p * 64] = acc[p];  // stays in L2 for the second pass
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(&A.fs->tiles_done[slot], 1u);  // one count per level-B warp
      } else {
#pragma unroll
        for (int p = 0; p < 64; ++p) __stcs(o + p * 64, acc[p]);
      }
    }
  } else if (FUSE) {
    // second pass (qubits 6..8) over finished groups, one 32-column job per
    // warp: input the group's 216 tile outputs (27 a-digit x 8 o-bit
    // combinations) from L2, output [G][64][4096] like fold_generic<3>.
    const int64_t total_jobs = (int64_t)((tile_end - tile_begin) / 216) * FUSE_JOBS;
    for (;;) {
      uint32_t jj = 0;
      if (lane == 0) jj = atomicAdd(&A.fs->job_next, 1u);
      const int64_t j = __shfl_sync(0xffffffffu, jj, 0);
      if (j >= total_jobs || *abort_flag) break;
      const int64_t G = j / FUSE_JOBS;
      const int chunk = (int)(j - G * FUSE_JOBS);
      const int slot = (int)(G % FUSE_RING);
      if (!poll_at_least(&A.fs->tiles_done[slot], (uint32_t)(2 * 216 * (G / FUSE_RING + 1)), abort_flag)) {
        give_up();
        break;
      }
      const int32_t *src = A.scratch + (int64_t)slot * 216 * 4096 + chunk * 32 + lane;
      int32_t acc[64];
#pragma unroll
      for (int p = 0; p < 64; ++p) acc[p] = 0;
#pragma unroll
      for (int al2 = 0; al2 < 27; ++al2) {
        int32_t v[8];
#pragma unroll
        for (int ol2 = 0; ol2 < 8; ++ol2) v[ol2] = __ldcg(src + (al2 * 8 + ol2) * 4096);
        wht<3>(v);
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[block_pauli(al2, m, 3)] += v[m];
      }
      int32_t *o = A.out + (G - tile_begin / 216) * 64 * 4096 + chunk * 32 + lane;
#pragma unroll
      for (int p = 0; p < 64; ++p) __stcs(o + p * 4096, acc[p]);
      __syncwarp();
      // the 216 consumed 128-byte lines are dead: drop them from L2 unwritten
      const int32_t *line0 = A.scratch + (int64_t)slot * 216 * 4096 + chunk * 32;
      for (int r = lane; r < 216; r += 32)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(line0 + r * 4096) : "memory");
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicAdd(&A.fs->jobs_done[slot], 1u);
    }
  }
}

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

// TMA map over rows [0, rows) of a [rows][2^n] count matrix, box 81 x 64.
bool make_count_map(CUtensorMap *map, const void *base, lre_count_kind kind, int n, int64_t rows,
                    uint32_t box_rows = SUB_ROWS) {
  EncodeTiled enc = encode_fn();
  if (!enc) return false;
  const size_t es = kind == LRE_COUNTS_I16 ? 2 : 4;
  const cuuint64_t dims[2] = {(cuuint64_t)1 << n, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {((cuuint64_t)1 << n) * es};
  const cuuint32_t box[2] = {64, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, kind == LRE_COUNTS_I16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_INT32,
                   2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// Generic pass: one thread per (ah, oh, c) column, J <= 3 qubits in registers.
// ---------------------------------------------------------------------------
// Generic pass: one thread per (ah, oh, c) column, J <= 3 qubits in registers.
template <int J, typename InT, typename AccT, int MODE, bool WEIGHT>
__global__ void __launch_bounds__(256) fold_generic(GenParams P) {
  __shared__ DivTables tab;  // uniform-shot final pass: divisor tables per k
  if constexpr (MODE == M_FINAL_U) {
    load_div_tables(P, tab);
    __syncthreads();
  }
  for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < P.items;
       item += (int64_t)gridDim.x * blockDim.x)
    fold_item<J, InT, AccT, MODE, WEIGHT>(P, item, MODE == M_FINAL_U ? &tab : nullptr);
}

using GenKernel = void (*)(GenParams);

template <int J, typename InT, typename AccT, bool WEIGHT>
GenKernel pick_mode(int mode) {
  switch (mode) {
    case M_STORE: return fold_generic<J, InT, AccT, M_STORE, WEIGHT>;
    case M_FINAL_U:
      if constexpr (!WEIGHT && !std::is_same<AccT, double>::value)
        return fold_generic<J, InT, AccT, M_FINAL_U, WEIGHT>;
      return nullptr;
    case M_FINAL_W:
      if constexpr (std::is_same<AccT, double>::value) return fold_generic<J, InT, AccT, M_FINAL_W, WEIGHT>;
      return nullptr;
    case M_PARITY:
      if constexpr (!WEIGHT && !std::is_same<AccT, double>::value)
        return fold_generic<J, InT, AccT, M_PARITY, WEIGHT>;
      return nullptr;
  }
  return nullptr;
}

template <int J>
GenKernel pick_types(int in_t, int acc_t, int mode, bool weight) {
  if (weight) {  // first pass of the per-basis-weighted path
    if (in_t == T_I16) return pick_mode<J, int16_t, double, true>(mode);
    if (in_t == T_I32) return pick_mode<J, int32_t, double, true>(mode);
    return nullptr;
  }
  if (acc_t == T_F64) {
    if (in_t == T_F64 && J <= 2) return pick_mode<(J <= 2 ? J : 2), double, double, false>(mode);
    return nullptr;
  }
  if (acc_t == T_I32) {
    if (in_t == T_I16) return pick_mode<J, int16_t, int32_t, false>(mode);
    if (in_t == T_I32) return pick_mode<J, int32_t, int32_t, false>(mode);
    return nullptr;
  }
  if (acc_t == T_I64) {
    if (in_t == T_I16) return pick_mode<J, int16_t, int64_t, false>(mode);
    if (in_t == T_I32) return pick_mode<J, int32_t, int64_t, false>(mode);
    if (in_t == T_I64) return pick_mode<J, int64_t, int64_t, false>(mode);
  }
  return nullptr;
}

GenKernel pick_generic(int J, int in_t, int acc_t, int mode, bool weight) {
  switch (J) {
    case 1: return pick_types<1>(in_t, acc_t, mode, weight);
    case 2: return pick_types<2>(in_t, acc_t, mode, weight);
    case 3: return pick_types<3>(in_t, acc_t, mode, weight);
  }
  return nullptr;
}

int type_size(int t) { return t == T_I16 ? 2 : (t == T_I32 ? 4 : 8); }

struct PassPlan {
  bool first6;  // a tiled first pass: six qubits (J = 6), or seven (J = 7, the raw tensor-core pass)
  bool fused9;  // first pass fused with the second through L2 (6 + 3 qubits)
  int J, r, in_t, acc_t, mode;
  bool weight;
  int64_t C;
  size_t out_bytes;  // non-final passes only
};

// Build the pass schedule.  shots_bound: an upper bound on every basis' total
// count (decides int32 vs int64 partial sums); weighted: FP64 path; first7:
// the caller runs the raw tensor-core first pass, which may fold seven qubits.
std::vector<PassPlan> make_plan(int n, lre_count_kind kind, bool weighted, bool parity,
                                int64_t shots_bound, bool aligned16, int variant, bool first7 = false) {
  std::vector<PassPlan> plan;
  int r = n, t = 0;
  int64_t C = 1;
  int in_t = (kind == LRE_COUNTS_I16) ? T_I16 : T_I32;
  auto fits32 = [&](int tt) {
    return shots_bound > 0 && (double)ipow(3, tt) * (double)shots_bound < 2147483647.0;
  };
  if (!weighted && r > 9 && aligned16 && fits32(9) && variant >= 2) {
    PassPlan p{};
    p.first6 = true;
    p.fused9 = true;
    p.J = 9;
    p.r = r;
    p.in_t = in_t;
    p.acc_t = T_I32;
    p.mode = M_STORE;
    p.C = C;
    p.out_bytes = (size_t)ipow(6, r - 9) * ((size_t)1 << 18) * 4;
    plan.push_back(p);
    r -= 9;
    t += 9;
    C <<= 18;
    in_t = T_I32;
  } else if (first7 && !weighted && kind == LRE_COUNTS_I16 && r > 7 && aligned16 && fits32(7)) {
    PassPlan p{};
    p.first6 = true;
    p.J = 7;
    p.r = r;
    p.in_t = in_t;
    p.acc_t = T_I32;
    p.mode = M_STORE;
    p.C = C;
    p.out_bytes = (size_t)ipow(6, r - 7) * 16384 * 4;
    plan.push_back(p);
    r -= 7;
    t += 7;
    C *= 16384;
    in_t = T_I32;
  } else if (!weighted && n >= 6 && r > 6 && aligned16 && fits32(6)) {
    PassPlan p{};
    p.first6 = true;
    p.J = 6;
    p.r = r;
    p.in_t = in_t;
    p.acc_t = T_I32;
    p.mode = M_STORE;
    p.C = C;
    p.out_bytes = (size_t)ipow(6, r - 6) * 4096 * 4;
    plan.push_back(p);
    r -= 6;
    t += 6;
    C *= 4096;
    in_t = T_I32;
  }
  while (r > 0) {
    const int jmax = weighted ? 2 : 3;
    const int J = r < jmax ? r : jmax;
    const bool last = (J == r);
    t += J;
    PassPlan p{};
    p.first6 = false;
    p.J = J;
    p.r = r;
    p.in_t = in_t;
    p.weight = weighted && (in_t != T_F64);
    p.acc_t = weighted ? T_F64 : (fits32(t) ? T_I32 : T_I64);
    p.mode = last ? (parity ? M_PARITY : (weighted ? M_FINAL_W : M_FINAL_U)) : M_STORE;
    p.C = C;
    p.out_bytes = last ? 0 : (size_t)ipow(6, r - J) * (size_t)ipow(4, J) * C * type_size(p.acc_t);
    plan.push_back(p);
    in_t = p.acc_t;
    r -= J;
    C *= ipow(4, J);
  }
  return plan;
}

void plan_buffers(const std::vector<PassPlan> &plan, size_t &bufA, size_t &bufB) {
  bufA = bufB = 0;
  for (size_t k = 0; k < plan.size(); ++k) {
    size_t &b = (k % 2 == 0) ? bufA : bufB;
    if (plan[k].out_bytes > b) b = plan[k].out_bytes;
  }
}

size_t round_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

bool encode_tensor_map_i32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                           const uint64_t *strides, const uint32_t *box) {
  return encode_tensor_map(map, CU_TENSOR_MAP_DATA_TYPE_INT32, base, rank, dims, strides, box);
}

bool encode_tensor_map(CUtensorMap *map, CUtensorMapDataType type, const void *base, int rank,
                       const uint64_t *dims, const uint64_t *strides, const uint32_t *box) {
  EncodeTiled enc = encode_fn();
  if (!enc || rank < 1 || rank > 5) return false;
  cuuint64_t d[5], st[4];
  cuuint32_t bx[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    bx[i] = box[i];
    es[i] = 1;
    if (i + 1 < rank) st[i] = strides[i];
  }
  CUresult r = enc(map, type, rank, const_cast<void *>(base), d, st, bx, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// the ring and counters of whichever fused pass runs (ALU or tensor-core)
size_t fuse_scratch_bytes() {
  const size_t alu = (size_t)FUSE_RING * 216 * 4096 * 4, mma = mma_fused9_scratch_bytes();
  return round_up(alu > mma ? alu : mma);
}
size_t fuse_counter_bytes() {
  const size_t alu = sizeof(FuseState), mma = mma_fused9_counter_bytes();
  return round_up(alu > mma ? alu : mma);
}

size_t fuse_bytes(const std::vector<PassPlan> &plan) {
  for (const auto &pp : plan)
    if (pp.fused9) return fuse_scratch_bytes() + fuse_counter_bytes();
  return 0;
}

size_t fold_workspace_bytes(int n, lre_count_kind kind, bool weighted, int64_t shots_bound, int variant) {
  size_t most = 0;
  for (int seven = 0; seven < 2; ++seven) {  // room for either first pass
    auto plan = make_plan(n, kind, weighted, false, shots_bound, true, variant, seven != 0);
    size_t a, b;
    plan_buffers(plan, a, b);
    size_t w = weighted ? round_up((size_t)ipow(3, n) * sizeof(double)) : 0;
    const size_t need = round_up(a) + round_up(b) + w + fuse_bytes(plan);
    if (need > most) most = need;
  }
  return most;
}

__global__ void inv_shots_kernel(const int64_t *shots, double *w, int64_t B, int *status) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = shots[b];
    if (s <= 0) latch(status, LRE_ERR_INVALID_ARG);
    w[b] = s > 0 ? 1.0 / (double)s : 0.0;
  }
}

namespace {

// Operand variant of the tensor-core first pass for this pass (0 raw int16,
// 1 biased int16, 3 int32 in two planes), or -1 when the ALU pass runs.
int tensor_variant(lre_ctx *ctx, const PassPlan &pp, const FoldArgs &a) {
  if (!pp.first6 || ctx->fold_path < 1 || !ctx->mma_operand || a.shots != nullptr || a.shots_uniform <= 0)
    return -1;
  int v = pp.in_t == T_I16 ? ctx->mma_biased : (pp.in_t == T_I32 && ctx->fold_path == 2 ? 3 : -1);
  if (pp.fused9 && v != 0) return -1;  // the fused first + second pass exists for the raw encoding
  if (pp.J == 7) v = v == 0 ? MMA_SEVEN : -1;  // and the seven-qubit pass
  return v >= 0 && a.shots_uniform <= mma_max_count(v) ? v : -1;
}

bool tensor_first_pass(lre_ctx *ctx, const PassPlan &pp, const FoldArgs &a) {
  return tensor_variant(ctx, pp, a) >= 0;
}

// The tensor-core first pass writes its partials (below 729 x shots, which
// must stay below 2^23) as split planes (3 bytes instead of 4) when the next
// pass is a TMA-staged store pass that reads them back.
bool use_planes(lre_ctx *ctx, const std::vector<PassPlan> &plan, const FoldArgs &a) {
  return !plan.empty() && !plan[0].fused9 && tensor_first_pass(ctx, plan[0], a) && plan.size() > 1 &&
         a.shots_uniform * (plan[0].J == 7 ? 2187 : 729) < (1ll << 23) && plan[1].mode == M_STORE &&
         plan[1].in_t == T_I32 && ctx->generic_tma && plan[1].C % 32 == 0;
}

// The schedule of a fold: the seven-qubit first pass where the raw
// tensor-core pass runs over a whole fold (stage 0, counts in memory),
// otherwise the six-qubit one (streamed folds always: their chunks are tile
// rows of the six-qubit pass).
std::vector<PassPlan> fold_plan(lre_ctx *ctx, const FoldArgs &a, bool weighted, bool parity, int64_t bound,
                                bool aligned16) {
  auto plan = make_plan(a.n, a.kind, weighted, parity, bound, aligned16, ctx->first_variant);
  if (ctx->first7 && a.stage == 0 && !a.rec_entries && !plan.empty() && plan[0].first6 && !plan[0].fused9 &&
      tensor_variant(ctx, plan[0], a) == 0) {
    auto p7 = make_plan(a.n, a.kind, weighted, parity, bound, aligned16, ctx->first_variant, true);
    if (!p7.empty() && p7[0].J == 7 && tensor_variant(ctx, p7[0], a) == MMA_SEVEN) return p7;
  }
  return plan;
}

}  // namespace

int64_t fold_split_rows(lre_ctx *ctx, const FoldArgs &a) {
  if (a.shots) return 0;
  const bool aligned16 = (reinterpret_cast<uintptr_t>(a.counts) & 15) == 0;
  auto plan = make_plan(a.n, a.kind, false, a.S != nullptr, a.shots_uniform, aligned16, ctx->first_variant);
  if (plan.empty() || !plan[0].first6 || plan[0].fused9) return 0;
  // the tensor-core and TMA-pipeline kernels take tile ranges; the register kernel does not
  return (tensor_first_pass(ctx, plan[0], a) || ctx->first_variant >= 1) ? 729 : 0;
}

bool fold_stage1_layout(lre_ctx *ctx, const FoldArgs &a, bool *planes, int64_t *elems) {
  if (a.shots || fold_split_rows(ctx, a) == 0) return false;
  const bool aligned16 = (reinterpret_cast<uintptr_t>(a.counts) & 15) == 0;
  auto plan = make_plan(a.n, a.kind, false, a.S != nullptr, a.shots_uniform, aligned16, ctx->first_variant);
  *elems = ipow(6, plan[0].r - 6) * 4096;
  *planes = use_planes(ctx, plan, a);
  return true;
}

bool fold_first_is_tensor(lre_ctx *ctx, const FoldArgs &a) {
  if (a.shots) return false;
  const bool aligned16 = (reinterpret_cast<uintptr_t>(a.counts) & 15) == 0;
  auto plan = make_plan(a.n, a.kind, false, a.S != nullptr, a.shots_uniform, aligned16, ctx->first_variant);
  return !plan.empty() && tensor_first_pass(ctx, plan[0], a);
}

lre_status fold_run(lre_ctx *ctx, const FoldArgs &a, void *ws, size_t ws_bytes, cudaStream_t s) {
  const bool weighted = a.shots != nullptr;
  const bool parity = a.S != nullptr;
  const bool aligned16 = (reinterpret_cast<uintptr_t>(a.counts) & 15) == 0;
  const int64_t bound = weighted ? 0 : a.shots_uniform;
  auto plan = fold_plan(ctx, a, weighted, parity, bound, aligned16);
  size_t bA, bB;
  plan_buffers(plan, bA, bB);
  char *p = static_cast<char *>(ws);
  void *bufA = p;
  void *bufB = p + round_up(bA);
  const size_t wbytes = weighted ? round_up((size_t)ipow(3, a.n) * 8) : 0;
  double *wgt = reinterpret_cast<double *>(p + round_up(bA) + round_up(bB));
  int32_t *fuse_scratch = reinterpret_cast<int32_t *>(p + round_up(bA) + round_up(bB) + wbytes);
  FuseState *fuse_state = reinterpret_cast<FuseState *>(reinterpret_cast<char *>(fuse_scratch) +
                                                         fuse_scratch_bytes());
  const size_t need = round_up(bA) + round_up(bB) + wbytes + fuse_bytes(plan);
  if (need > ws_bytes) return LRE_ERR_OOM;
  const int64_t B = ipow(3, a.n);
  if (weighted) {
    Launch L(ctx, "inv_shots", s);
    inv_shots_kernel<<<256, 256, 0, s>>>(a.shots, wgt, B, ctx->d_status);
  }
  const bool planes = use_planes(ctx, plan, a);
  const void *in = a.counts;
  size_t k_begin = 0, k_end = plan.size();
  if (a.stage != 0) {
    if (fold_split_rows(ctx, a) == 0) return LRE_ERR_UNSUPPORTED;
    if (a.stage == 1) {
      k_end = 1;
    } else {
      k_begin = 1;
      in = bufA;  // the first pass's output
    }
  }
  for (size_t k = k_begin; k < k_end; ++k) {
    const PassPlan &pp = plan[k];
    const int64_t all_tiles = pp.first6 ? (ipow(3, pp.r - 6) << (pp.r - 6)) : 0;
    const int64_t tile_begin = a.stage == 1 ? a.ah_begin << (pp.r - 6) : 0;
    const int64_t tile_end = a.stage == 1 ? a.ah_end << (pp.r - 6) : all_tiles;
    if (a.stage == 1 && (tile_begin < 0 || tile_end > all_tiles || tile_end < tile_begin)) return LRE_ERR_INVALID_ARG;
    if (a.stage == 1 && tile_end == tile_begin) return LRE_OK;
    void *out;
    if (pp.mode == M_STORE)
      out = (k % 2 == 0) ? bufA : bufB;
    else
      out = parity ? static_cast<void *>(a.S) : static_cast<void *>(a.theta);
    CUtensorMap tmap, tmap_tail;
    const bool tensor = tensor_first_pass(ctx, pp, a);
    if (tensor && a.rec_entries) {
      if (a.stage != 1) return LRE_ERR_INVALID_ARG;
      const int64_t elems = ipow(6, pp.r - 6) * 4096;
      int8_t *hi = planes ? static_cast<int8_t *>(out) + elems * 2 : nullptr;
      lre_status st = mma_first_pass_records(ctx, ctx->mma_operand, a.rec_entries, a.rec_offs, a.shots_uniform,
                                             static_cast<int32_t *>(out), hi, pp.r, tile_begin, tile_end, s);
      if (st != LRE_OK) return st;
    } else if (tensor && pp.fused9) {
      const int64_t rows = ipow(3, pp.r);
      if (!make_count_map(&tmap, in, LRE_COUNTS_I16, pp.r, rows, mma_box_rows(0, 0)) ||
          !make_count_map(&tmap_tail, in, LRE_COUNTS_I16, pp.r, rows, mma_box_rows(1, 0))) {
        ctx->last_error = "tensor map of the counts rejected";
        return LRE_ERR_CUDA;
      }
      lre_status st = mma_first_pass_fused9(ctx, tmap, tmap_tail, ctx->mma_operand, static_cast<int32_t *>(out),
                                            fuse_scratch, reinterpret_cast<unsigned *>(fuse_state), pp.r,
                                            a.shots_uniform, ctx->fused_consumers, ctx->fused_discard != 0, s);
      if (st != LRE_OK) return st;
    } else if (tensor) {
      const lre_count_kind mk = pp.in_t == T_I16 ? LRE_COUNTS_I16 : LRE_COUNTS_I32;
      const int64_t rows = (a.stage == 1 && a.rows_in > 0) ? a.rows_in : ipow(3, pp.r);
      const int tv = tensor_variant(ctx, pp, a);
      if (!make_count_map(&tmap, in, mk, pp.r, rows, mma_box_rows(0, tv)) ||
          !make_count_map(&tmap_tail, in, mk, pp.r, rows, mma_box_rows(1, tv))) {
        ctx->last_error = "tensor map of the counts rejected";
        return LRE_ERR_CUDA;
      }
      const int64_t elems = pp.J == 7 ? ipow(6, pp.r - 7) * 16384 : ipow(6, pp.r - 6) * 4096;
      int8_t *hi = planes ? static_cast<int8_t *>(out) + elems * 2 : nullptr;
      lre_status st = mma_first_pass(ctx, tmap, tmap_tail, ctx->mma_operand, static_cast<int32_t *>(out), hi,
                                     pp.r, tensor_variant(ctx, pp, a), a.shots_uniform, tile_begin, tile_end,
                                     a.stage == 1 ? a.row_base : 0, s);
      if (st != LRE_OK) return st;
    } else if (pp.first6 && (ctx->first_variant >= 1 || pp.fused9) &&
        make_count_map(&tmap, in, pp.in_t == T_I16 ? LRE_COUNTS_I16 : LRE_COUNTS_I32, pp.r,
                       (a.stage == 1 && a.rows_in > 0) ? a.rows_in : ipow(3, pp.r))) {
      const int64_t tiles = tile_end - tile_begin;
      int grid = ctx->num_sms;
      if ((int64_t)grid > tiles) grid = (int)tiles;
      PipeArgs A{};
      A.out = static_cast<int32_t *>(out);
      A.n = pp.r;
      A.tile_begin = tile_begin;
      A.tile_end = tile_end;
      A.row_base = a.stage == 1 ? a.row_base : 0;
      A.status = ctx->d_status;
      A.fuse = pp.fused9 ? 1 : 0;
      const int threads = pp.fused9 ? FUSE_THREADS : PIPE_THREADS;
      if (pp.fused9) {
        A.scratch = fuse_scratch;
        A.fs = fuse_state;
        cudaError_t e0 = cudaMemsetAsync(fuse_state, 0, sizeof(FuseState), s);
        if (e0 != cudaSuccess) return cuda_fail(ctx, e0, "fused pass state");
      }
      Launch L(ctx, pp.fused9 ? "fold_first9_fused" : "fold_first6", s);
      if (pp.in_t == T_I16) {
        constexpr int sm = PipeCfg<int16_t>::SMEM;
        auto k = pp.fused9 ? fold_first6_pipe<int16_t, true> : fold_first6_pipe<int16_t, false>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        k<<<grid, threads, sm, s>>>(tmap, A);
      } else {
        constexpr int sm = PipeCfg<int32_t>::SMEM;
        auto k = pp.fused9 ? fold_first6_pipe<int32_t, true> : fold_first6_pipe<int32_t, false>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        k<<<grid, threads, sm, s>>>(tmap, A);
      }
    } else if (pp.first6 && !pp.fused9) {
      const int64_t tiles = ipow(3, pp.r - 6) << (pp.r - 6);
      const size_t smem = 64 * P1_ZSTRIDE * sizeof(int32_t);
      int grid = ctx->num_sms * 2;
      if ((int64_t)grid > tiles) grid = (int)tiles;
      Launch L(ctx, "fold_first6_regs", s);
      if (pp.in_t == T_I16) {
        cudaFuncSetAttribute(fold_first6<int16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fold_first6<int16_t><<<grid, P1_THREADS, smem, s>>>(static_cast<const int16_t *>(in),
                                                            static_cast<int32_t *>(out), pp.r, tiles);
      } else {
        cudaFuncSetAttribute(fold_first6<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fold_first6<int32_t><<<grid, P1_THREADS, smem, s>>>(static_cast<const int32_t *>(in),
                                                            static_cast<int32_t *>(out), pp.r, tiles);
      }
    } else {
      GenKernel kern = pick_generic(pp.J, pp.in_t, pp.acc_t, pp.mode, pp.weight);
      if (!kern) return LRE_ERR_UNSUPPORTED;
      GenParams gp;
      gp.in = in;
      gp.out = out;
      gp.C = pp.C;
      gp.n_oh = 1ll << (pp.r - pp.J);
      gp.items = ipow(3, pp.r - pp.J) * gp.n_oh * pp.C;
      gp.r = pp.r;
      gp.n = a.n;
      gp.wgt = wgt;
      gp.shots = (double)a.shots_uniform;
      gp.total = a.shots_uniform * B;
      gp.T = a.T;
      for (int id = 0; id < 16; ++id) {  // id: number of identity letters
        const double p3 = (double)ipow(3, id <= a.n ? id : 0);
        gp.denom[id] = weighted ? p3 : (double)a.shots_uniform * p3;  // exact: < 2^53
        gp.recip[id] = 1.0 / gp.denom[id];                              // host IEEE division
        gp.dint[id] = weighted ? 0 : a.shots_uniform * ipow(3, id <= a.n ? id : 0);
        gp.up3[id] = id <= a.n ? ipow(3, a.n - id) : 0;
      }
      gp.status = ctx->d_status;
      gp.hi_from = planes_hi_from(a.shots_uniform);
      gp.hi_letters = plan[0].J == 7 ? 7 : 6;
      gp.top7 = plan[0].J == 7 ? 1 : 0;  // the seven-qubit first pass folded qubit n
      const int in_t = (planes && k == 1) ? (int)T_I24P : pp.in_t;
      lre_status tst = ctx->generic_tma ? tma_pass(ctx, gp, pp.J, in_t, pp.acc_t, pp.mode, pp.weight, s)
                                        : LRE_ERR_UNSUPPORTED;
      if (tst == LRE_ERR_UNSUPPORTED && in_t == T_I24P) {
        ctx->last_error = "split-plane partials need the TMA-staged second pass";
        return LRE_ERR_UNSUPPORTED;
      }
      if (tst == LRE_ERR_UNSUPPORTED) {
        int64_t blocks = (gp.items + 255) / 256;
        const int64_t cap = (int64_t)ctx->num_sms * 64;
        if (blocks > cap) blocks = cap;
        Launch L(ctx, pp.mode == M_STORE ? "fold_pass" : "fold_final", s);
        kern<<<(unsigned)blocks, 256, 0, s>>>(gp);
      } else if (tst != LRE_OK) {
        return tst;
      }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fold pass launch");
    in = out;
  }
  return LRE_OK;
}

}  // namespace lre

namespace lre {
namespace {
__global__ void debug_div_kernel(const int64_t *S, int64_t count, int64_t D, double y, double *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = passes::div_int_rn(S[i], D, y);
}
}  // namespace
}  // namespace lre

// Test hook (not part of include/lre.h; host only, no device work): the
// fold pass schedule for these arguments.  Per pass, 9 int64 at out + 9 k:
// first6, fused9, J, r, in_t, acc_t, mode, C, out_bytes (at most max_passes
// written).  variant: the first-pass variant (0..2), plus 256 when the raw
// tensor-core first pass runs (the seven-qubit pass may be planned).
// Returns the number of passes, or -1 for n outside 1..14.
extern "C" int lre_debug_fold_plan(int n, int kind, int weighted, int parity, int64_t shots_bound, int aligned16,
                                   int variant, int64_t *out, int max_passes) {
  using namespace lre;
  if (n < 1 || n > 14) return -1;
  const auto plan = make_plan(n, static_cast<lre_count_kind>(kind), weighted != 0, parity != 0, shots_bound,
                              aligned16 != 0, variant & 255, (variant & 256) != 0);
  for (int k = 0; out && k < (int)plan.size() && k < max_passes; ++k) {
    const PassPlan &p = plan[k];
    const int64_t v[9] = {p.first6, p.fused9, p.J, p.r, p.in_t, p.acc_t, p.mode, p.C, (int64_t)p.out_bytes};
    for (int f = 0; f < 9; ++f) out[9 * k + f] = v[f];
  }
  return (int)plan.size();
}

// Test hook (not part of include/lre.h): out[i] = the final pass's correctly
// rounded S[i] / D (device arrays of `count`), for 0 < D < 2^53.
extern "C" lre_status lre_debug_div(lre_ctx *ctx, const int64_t *S, int64_t count, int64_t D, double *out,
                                    lre_stream stream) {
  using namespace lre;
  if (!ctx || !S || !out || count <= 0 || D <= 0 || D >= (1ll << 53)) return LRE_ERR_INVALID_ARG;
  debug_div_kernel<<<256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(S, count, D, 1.0 / (double)D, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "debug division");
}

// Test hook (not part of include/lre.h): run only the 6-qubit first pass of
// step (i) over all tiles, variant 0 = register-only kernel, 1 = TMA
// pipeline.  out: device int32 [3^(n-6)][2^(n-6)][4096].
extern "C" lre_status lre_debug_first_pass(lre_ctx *ctx, const void *counts, lre_count_kind kind, int n,
                                           int32_t *out, int variant, lre_stream stream) {
  using namespace lre;
  if (!ctx || !counts || !out || n < 7 || n > 14) return LRE_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t tiles = ipow(3, n - 6) << (n - 6);
  if (variant == 1) {
    CUtensorMap tmap;
    if (!make_count_map(&tmap, counts, kind, n, ipow(3, n))) return LRE_ERR_CUDA;
    const int grid = (int)(tiles < ctx->num_sms ? tiles : ctx->num_sms);
    PipeArgs A{};
    A.out = out;
    A.n = n;
    A.tile_end = tiles;
    A.status = ctx->d_status;
    if (kind == LRE_COUNTS_I16) {
      constexpr int sm = PipeCfg<int16_t>::SMEM;
      cudaFuncSetAttribute(fold_first6_pipe<int16_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
      fold_first6_pipe<int16_t, false><<<grid, PIPE_THREADS, sm, s>>>(tmap, A);
    } else {
      constexpr int sm = PipeCfg<int32_t>::SMEM;
      cudaFuncSetAttribute(fold_first6_pipe<int32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
      fold_first6_pipe<int32_t, false><<<grid, PIPE_THREADS, sm, s>>>(tmap, A);
    }
  } else {
    const size_t smem = 64 * P1_ZSTRIDE * sizeof(int32_t);
    const int grid = (int)(tiles < 2 * ctx->num_sms ? tiles : 2 * ctx->num_sms);
    if (kind == LRE_COUNTS_I16) {
      cudaFuncSetAttribute(fold_first6<int16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      fold_first6<int16_t><<<grid, P1_THREADS, smem, s>>>(static_cast<const int16_t *>(counts), out, n, tiles);
    } else {
      cudaFuncSetAttribute(fold_first6<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      fold_first6<int32_t><<<grid, P1_THREADS, smem, s>>>(static_cast<const int32_t *>(counts), out, n, tiles);
    }
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "debug first pass");
}
