// Tensor-core form of the first fold pass (int16 counts below 1024).
//
// The level-A contraction of a sub-tile (81 basis rows x 64 outcomes, three
// qubits in the rows and three in the outcome octets) is the GEMM
//     D[plA][item] = sum_k Tt[plA][k] X[k][item],   k = (alA, olA), item = (a3, olB)
// with Tt the constant 64 x 216 matrix of the per-qubit map T (entries 0, +1,
// -1).  In the K-major canonical layout of the tensor-core operands a core
// matrix is 8 rows x 16 bytes; for X those 8 rows are the 8 outcome octets
// (olB) of one basis row and the 16 bytes are the octet's 8 counts (olA), i.e.
// a core matrix is exactly one 128-byte count row of the TMA tile.  So the
// tile feeds tcgen05.mma (kind::f16) where it landed: K-step stride
// (next alA) = 128 B, N-group stride (next a3) = 27 rows.
//
// Exactness: each count c < 1024 becomes the fp16 1024 + c by one OR per
// pair (0x6400 | c is the fp16 bit pattern of 1024 + c).  The bias adds
// 1024 * sum_k Tt[plA][k] to D, which is 1024 * 216 for plA = III and zero
// otherwise (a row of T sums to 6 for I and 0 for X, Y, Z); the level-B
// warps subtract it.  Every partial sum stays below 2^24, so FP32 accumulation
// in TMEM is exact and D is the same integer the ALU path computes.
//
// Roles (192 threads):
//   warp 0    TMA producer into a ring of R sub-tile slots (82 rows: one
//             zero row after each sub-tile so the padded 14th K-step reads
//             0 x 0); a slot is released by a tcgen05.commit as soon as the
//             MMAs reading it have completed
//   warps 2,3 convert the slots in place (even / odd sub-tiles)
//   warp 1    issues 14 MMAs per sub-tile (M=128 with rows 64..127 of A zero,
//             N=24, K=16) into the sub-tile's 24 columns of a whole-tile
//             accumulator in TMEM (216 columns, two tile buffers)
//   warps 4,5 level B straight from TMEM: thread plA (TMEM lane) reads its
//             216 columns eight at a time with tcgen05.ld, removes the bias,
//             contracts the next three qubits on the ALU and writes 64 outputs
// Every barrier has one in-order consumer, so parity waits cannot alias, and
// every wait is bounded by time.
#include <cuda_runtime.h>

#include <cudaTypedefs.h>

#include <vector>

#include "lre_internal.cuh"
#include "passes.cuh"
#include "sm103.cuh"

namespace lre {
namespace {

using namespace passes;

constexpr int MMA_THREADS = 192;
constexpr int MMA_R = 14;                     // ring slots (even: slot parity = converter)
constexpr int SLOT_ROWS = 82;                 // 81 + one zero row
constexpr int SLOT_BYTES = SLOT_ROWS * 128;   // int16 rows of 64 outcomes
constexpr int A_BYTES = 16 * 28 * 128;        // 128 x 224 fp16, core-matrix layout
constexpr int OFF_A = MMA_R * SLOT_BYTES;
constexpr int OFF_BAR = OFF_A + A_BYTES;
constexpr int MMA_SMEM = OFF_BAR + 64 * 8 + 1024;
constexpr int BIAS = 1024 * 216;
constexpr uint32_t TMEM_COLS = 512;           // two whole-tile accumulators of 216 columns
constexpr uint32_t TILE_COLS = 256;

__global__ void __launch_bounds__(MMA_THREADS, 1)
    fold_first6_mma(const __grid_constant__ CUtensorMap tmap, const uint4 *__restrict__ gA,
                    int32_t *__restrict__ out, int n, int64_t tiles, int *status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024u - (sm103::smem_addr(smem_raw) & 1023u)) & 1023u);
  uint8_t *ring = smem;
  uint8_t *Am = smem + OFF_A;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
  uint64_t *conv = full + MMA_R;
  uint64_t *empty = conv + MMA_R;
  uint64_t *tile_done = empty + MMA_R;
  uint64_t *tile_free = tile_done + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tile_free + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_oh = (1ll << n) >> 6;

  // constant operand A and the zero pad rows
  for (int i = threadIdx.x; i < A_BYTES / 16; i += MMA_THREADS) reinterpret_cast<uint4 *>(Am)[i] = gA[i];
  for (int i = threadIdx.x; i < MMA_R * 8; i += MMA_THREADS)
    reinterpret_cast<uint4 *>(ring + (i >> 3) * SLOT_BYTES + 81 * 128)[i & 7] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    for (int i = 0; i < MMA_R; ++i) {
      sm103::mbar_init(&full[i], 1);
      sm103::mbar_init(&conv[i], 32);
      sm103::mbar_init(&empty[i], 1);
    }
    for (int b = 0; b < 2; ++b) {
      sm103::mbar_init(&tile_done[b], 1);
      sm103::mbar_init(&tile_free[b], 64);
    }
    *abort_flag = 0;
    sm103::fence_barrier_init();
  }
  sm103::fence_proxy_async_smem();  // A and the pad rows are read by the tensor cores
  if (warp == 1) sm103::tmem_alloc(tmem_slot, TMEM_COLS);
  sm103::tc_fence_before();
  __syncthreads();
  sm103::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto give_up = [&]() {
    *abort_flag = 1;
    latch(status, LRE_ERR_TIMEOUT);
  };
  const int64_t my_tiles = tiles > blockIdx.x ? (tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t total = my_tiles * 9;  // sub-tiles of this CTA

  if (warp == 0) {
    if (lane == 0) {
      int64_t g = 0;
      for (; g < total && !*abort_flag; ++g) {
        const int64_t tile = blockIdx.x + (g / 9) * gridDim.x;
        const int s = (int)(g % 9);
        const int64_t ah = tile / n_oh, oh = tile - ah * n_oh;
        const int slot = (int)(g % MMA_R);
        if (g >= MMA_R && !sm103::mbar_wait(&empty[slot], (uint32_t)((g / MMA_R - 1) & 1), abort_flag)) {
          give_up();
          break;
        }
        sm103::mbar_arrive_expect_tx(&full[slot], 81 * 128);
        sm103::tma_load_2d(ring + slot * SLOT_BYTES, &tmap, (int)(oh * 64), (int)(ah * 729 + s * 81), &full[slot]);
      }
      for (int64_t q = g > MMA_R ? g - MMA_R : 0; q < g; ++q)  // drain in-flight loads
        for (uint32_t it = 0; it < sm103::kSpinLimit; ++it)
          if (sm103::mbar_try_wait(&full[q % MMA_R], (uint32_t)((q / MMA_R) & 1))) break;
    }
  } else if (warp == 2 || warp == 3) {
    // converters: warp 2 takes even sub-tiles, warp 3 odd ones (MMA_R even,
    // so each slot always belongs to the same converter)
    for (int64_t g = warp - 2; g < total; g += 2) {
      const int slot = (int)(g % MMA_R);
      if (!sm103::mbar_wait(&full[slot], (uint32_t)((g / MMA_R) & 1), abort_flag)) {
        give_up();
        break;
      }
      uint4 *rows = reinterpret_cast<uint4 *>(ring + slot * SLOT_BYTES);
      for (int k = lane; k < 81 * 8; k += 32) {  // counts -> fp16(1024 + c), in place
        uint4 v = rows[k];
        v.x |= 0x64006400u; v.y |= 0x64006400u; v.z |= 0x64006400u; v.w |= 0x64006400u;
        rows[k] = v;
      }
      sm103::fence_proxy_async_smem();
      sm103::mbar_arrive(&conv[slot]);
    }
  } else if (warp == 1) {
    const uint32_t idesc = sm103::umma_idesc_f16(128, 24);
    const uint32_t a_base = sm103::smem_addr(Am);
    int64_t g = 0;
    for (; g < total; ++g) {
      const int slot = (int)(g % MMA_R);
      const int64_t lt = g / 9;
      const int s = (int)(g - lt * 9);
      const int tb = (int)(lt & 1);
      if (!sm103::mbar_wait(&conv[slot], (uint32_t)((g / MMA_R) & 1), abort_flag)) {
        give_up();
        break;
      }
      if (s == 0 && lt >= 2 &&
          !sm103::mbar_wait(&tile_free[tb], (uint32_t)(((lt >> 1) - 1) & 1), abort_flag)) {
        give_up();
        break;
      }
      sm103::tc_fence_after();
      if (lane == 0) {
        const uint32_t b_base = sm103::smem_addr(ring + slot * SLOT_BYTES);
        const uint32_t d = tmem + tb * TILE_COLS + s * 24;
#pragma unroll 1
        for (int kk = 0; kk < 14; ++kk) {
          const uint64_t ad = sm103::umma_desc(a_base + kk * 256, 128, 28 * 128);
          const uint64_t bd = sm103::umma_desc(b_base + kk * 256, 128, 27 * 128);
          sm103::umma_f16(d, ad, bd, idesc, kk > 0);
        }
        sm103::umma_commit(&empty[slot]);                  // slot reusable when these finish
        if (s == 8) sm103::umma_commit(&tile_done[tb]);    // whole tile accumulated
      }
      __syncwarp();
    }
    // no MMA may still run when TMEM is released
    if (lane == 0 && g > 0) {
      const int64_t q = g - 1;
      for (uint32_t it = 0; it < sm103::kSpinLimit; ++it)
        if (sm103::mbar_try_wait(&empty[q % MMA_R], (uint32_t)((q / MMA_R) & 1))) break;
    }
  } else {
    // warps 4, 5: level B from TMEM lanes 0..63
    const int plA = (warp - 4) * 32 + lane;
    for (int64_t lt = 0; lt < my_tiles; ++lt) {
      const int tb = (int)(lt & 1);
      if (!sm103::mbar_wait(&tile_done[tb], (uint32_t)((lt >> 1) & 1), abort_flag)) {
        give_up();
        break;
      }
      sm103::tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)((warp - 4) * 32) << 16) + tb * TILE_COLS;
      int32_t acc[64];
#pragma unroll
      for (int p = 0; p < 64; ++p) acc[p] = 0;
#pragma unroll
      for (int alB = 0; alB < 27; ++alB) {
        uint32_t r[8];
        sm103::tmem_ld8(ta + alB * 8, r);
        sm103::tmem_ld_wait();
        int32_t v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (int32_t)__uint_as_float(r[i]) - (plA == 0 ? BIAS : 0);
        wht<3>(v);
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[block_pauli(alB, m, 3)] += v[m];
      }
      sm103::tc_fence_before();
      sm103::mbar_arrive(&tile_free[tb]);
      const int64_t tile = blockIdx.x + lt * gridDim.x;
      int32_t *o = out + tile * 4096 + plA;
#pragma unroll
      for (int p = 0; p < 64; ++p) __stcs(o + p * 64, acc[p]);
    }
  }
  sm103::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    sm103::tc_fence_after();
    sm103::tmem_dealloc(tmem, TMEM_COLS);
  }
}

// Tt as fp16 bits in the K-major core-matrix layout: row plA (0..127, rows
// 64.. zero), column k = alA*8 + olA (0..223, alA = 27 zero); core matrix
// (m-group, k-group) at (m-group * 28 + k-group) * 128 bytes.
std::vector<uint16_t> make_a_operand() {
  std::vector<uint16_t> A(A_BYTES / 2, 0);
  const uint16_t one = 0x3C00, mone = 0xBC00;
  for (int p = 0; p < 64; ++p)
    for (int al = 0; al < 27; ++al)
      for (int ol = 0; ol < 8; ++ol) {
        int v = 1;
        for (int q = 0, pp = p, aa = al; q < 3; ++q, pp >>= 2, aa /= 3) {
          const int letter = pp & 3, axis = aa % 3, o = (ol >> q) & 1;
          if (letter == 0) continue;            // I: +1
          if (letter != axis + 1) { v = 0; break; }
          if (o) v = -v;                        // matching axis: (-1)^o
        }
        if (v == 0) continue;
        const int k = al * 8 + ol;
        const size_t idx = ((size_t)(p >> 3) * 28 + (k >> 3)) * 64 + (p & 7) * 8 + (k & 7);
        A[idx] = v > 0 ? one : mone;
      }
  return A;
}

}  // namespace

size_t mma_operand_bytes() { return A_BYTES; }

// Launch the tensor-core first pass over all tiles of an n-qubit int16 count
// matrix; a_dev must hold the operand written by mma_operand_upload.
lre_status mma_first_pass(lre_ctx *ctx, const CUtensorMap &tmap, const void *a_dev, int32_t *out, int n,
                          cudaStream_t s) {
  const int64_t tiles = ipow(3, n - 6) << (n - 6);
  const int grid = (int)(tiles < ctx->num_sms ? tiles : ctx->num_sms);
  Launch L(ctx, "fold_first6_mma", s);
  cudaFuncSetAttribute(fold_first6_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, MMA_SMEM);
  fold_first6_mma<<<grid, MMA_THREADS, MMA_SMEM, s>>>(tmap, static_cast<const uint4 *>(a_dev), out, n, tiles,
                                                     ctx->d_status);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "tensor-core first pass launch");
}

lre_status mma_operand_upload(lre_ctx *ctx, void *a_dev, cudaStream_t s) {
  static const std::vector<uint16_t> A = make_a_operand();
  // pageable source: the copy is staged before the call returns
  cudaError_t e = cudaMemcpyAsync(a_dev, A.data(), A_BYTES, cudaMemcpyHostToDevice, s);
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "tensor-core operand upload");
}

}  // namespace lre
