// Shot records grouped by count tile, for the tensor-core first pass that
// builds its count tiles in shared memory straight from the records (step (i),
// Sec. III: the counts c_b(o) are only ever needed tile by tile).
//
// A tile row is 729 consecutive bases (the six lowest basis digits, al); its
// 2^(n-6) tiles are the outcome blocks oh (the outcome's bits above the six
// lowest).  tile_bucket_kernel takes one tile row per CTA and counting-sorts
// the row's 729 x N shot records into 16-bit entries (al << 6) | ol, ol = the
// outcome's six lowest bits, by bucket oh * 2 + (al >= 432) -- the tile and
// the half of its rows the first pass stages together -- with the start of
// every bucket in offs[tile row][bucket] (offsets within the tile row's
// 729 N entries; the last bucket ends at 729 N).  The order inside a bucket
// is irrelevant: the consumer only adds counts.
#include <cuda_runtime.h>

#include "lre_internal.cuh"

namespace lre {

namespace {

constexpr int BUCKET_THREADS = 512;
constexpr int BUCKET_WARPS = BUCKET_THREADS / 32;
constexpr int MAX_BUCKETS = 512;  // two per tile, n <= 14: one thread per bucket
static_assert(MAX_BUCKETS <= BUCKET_THREADS, "one thread per bucket in the scan");

// One tile row per CTA (grid-stride).  Every warp counts into its own copy of
// the bucket counters (no contention between warps), a scan turns the
// per-warp counts into per-warp cursors, and the scatter pass places each
// entry through its warp's cursor.  Records are read eight at a time (shots
// a multiple of 8, rows 16-byte aligned).
__global__ void __launch_bounds__(BUCKET_THREADS) tile_bucket_kernel(const uint16_t *__restrict__ rec,
                                                                     int64_t tile_rows, int64_t shots, int n,
                                                                     uint16_t *__restrict__ out,
                                                                     int32_t *__restrict__ offs, int *status) {
  extern __shared__ int32_t wcnt[];  // [BUCKET_WARPS][nb]
  const int nb = 2 << (n - 6);
  const uint32_t d = 1u << n;
  const int warp = threadIdx.x >> 5;
  int32_t *mine = wcnt + warp * nb;
  const int64_t tv = 729 * shots / 8;  // uint4 per tile row
  const float inv_shots = 1.0f / (float)shots;
  for (int64_t tr = blockIdx.x; tr < tile_rows; tr += gridDim.x) {
    const uint4 *r4 = reinterpret_cast<const uint4 *>(rec + tr * 729 * shots);
    uint16_t *o = out + tr * 729 * shots;
    for (int b = threadIdx.x; b < BUCKET_WARPS * nb; b += blockDim.x) wcnt[b] = 0;
    __syncthreads();
    bool bad = false;
    for (int pass = 0; pass < 2; ++pass) {
      for (int64_t q0 = threadIdx.x; q0 < tv; q0 += 4 * (int64_t)blockDim.x) {
        uint4 w4[4];  // four independent 16-byte loads in flight per thread
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t q = q0 + u * (int64_t)blockDim.x;
          w4[u] = q < tv ? __ldcs(r4 + q) : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t q = q0 + u * (int64_t)blockDim.x;
          if (q >= tv) continue;
          const uint32_t word[4] = {w4[u].x, w4[u].y, w4[u].z, w4[u].w};
          // basis row of these 8 records (shots is a multiple of 8): q * 8 / shots
          int al = (int)((float)(q * 8) * inv_shots);
          if ((int64_t)al * shots > q * 8) --al;
          else if ((int64_t)(al + 1) * shots <= q * 8) ++al;
          const uint32_t half = al >= 432 ? 1u : 0u;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint32_t v = (word[k >> 1] >> ((k & 1) * 16)) & 0xFFFFu;
            if (v >= d) {
              bad = true;
              continue;
            }
            const uint32_t key = (v >> 6) << 1 | half;
            if (pass == 0)
              atomicAdd(&mine[key], 1);
            else
              o[atomicAdd(&mine[key], 1)] = (uint16_t)((al << 6) | (v & 63u));
          }
        }
      }
      __syncthreads();
      if (pass == 0) {
        // per bucket (one thread each): the warps' counts -> their offsets
        // inside the bucket, then an exclusive scan of the bucket totals
        // across the CTA (warp shuffles, then the warps' sums)
        int32_t tot = 0;
        const int b = threadIdx.x;
        if (b < nb)
          for (int w = 0; w < BUCKET_WARPS; ++w) {
            const int32_t c = wcnt[w * nb + b];
            wcnt[w * nb + b] = tot;
            tot += c;
          }
        int32_t incl = tot;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
          const int32_t t = __shfl_up_sync(0xffffffffu, incl, o2);
          if (lane >= o2) incl += t;
        }
        __shared__ int32_t wsum[BUCKET_WARPS];
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int32_t before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        const int32_t start = before + incl - tot;  // exclusive
        if (b < nb) {
          offs[tr * nb + b] = start;
          for (int w = 0; w < BUCKET_WARPS; ++w) wcnt[w * nb + b] += start;
        }
        __syncthreads();
      }
    }
    if (bad) latch(status, LRE_ERR_INVALID_ARG);
  }
}

}  // namespace

lre_status tile_bucket_run(lre_ctx *ctx, const uint16_t *records, int64_t tile_rows, int64_t shots, int n,
                           uint16_t *entries, int32_t *offs, cudaStream_t s) {
  if (n < 7 || n > 14 || shots <= 0 || (int64_t)729 * shots >= (1ll << 31)) return LRE_ERR_UNSUPPORTED;
  static_assert(MAX_BUCKETS >= (2 << 8), "two buckets per tile at n = 14");
  if (tile_rows <= 0) return LRE_OK;
  if (shots % 8 != 0 || (reinterpret_cast<uintptr_t>(records) & 15) != 0) return LRE_ERR_UNSUPPORTED;
  int grid = ctx->num_sms * 2;
  if (grid > tile_rows) grid = (int)tile_rows;
  const size_t smem = (size_t)BUCKET_WARPS * (2 << (n - 6)) * sizeof(int32_t);
  Launch L(ctx, "tile_bucket", s);
  cudaFuncSetAttribute(tile_bucket_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  tile_bucket_kernel<<<grid, BUCKET_THREADS, smem, s>>>(records, tile_rows, shots, n, entries, offs, ctx->d_status);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "tile bucket launch");
}

}  // namespace lre
