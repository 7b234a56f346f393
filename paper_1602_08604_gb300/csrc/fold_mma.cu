// Tensor-core form of the first fold pass (int16 counts below 2048, or int32
// counts below 16384 as two planes).
//
// A tile is 729 basis rows x 64 outcomes: six qubits in the rows (alB: the
// high three, alA: the low three) and six in the outcomes (olB, olA).  Its
// level-A contraction is the GEMM
//     D[plA][(alB, olB)] = sum_k Tt[plA][k] X[(alB, olB)][k],   k = (alA, olA)
// with Tt the constant 64 x 216 matrix of the per-qubit map T (entries 0, +1,
// -1).  In the K-major canonical layout of the tensor-core operands a core
// matrix is 8 rows x 16 bytes; for X those 8 rows are the 8 outcome octets
// (olB) of one basis row and the 16 bytes the octet's 8 counts (olA), so a
// core matrix is exactly one 128-byte count row as TMA lands it: the K-step
// stride (next alA) is one row and the N-group stride (next alB) 27 rows, the
// same for every alB of the tile.  The tile therefore feeds two MMA chains in
// place, N = 128 (alB 0..15) and N = 96 (alB 16..27; alB 27 reads rows past
// the tile and lands in accumulator columns nobody reads).
//
// K = 216 is 13.5 K-steps of 16: the 14th step reads rows alA = 25, 26 against
// an operand column block that is zero for alA = 25, so no row outside an alB
// group enters a used column.
//
// Operand encodings (the variant V):
//   RAW      the int16 count c < 2048 is used unchanged as fp16 bits, which
//            encode exactly c * 2^-24 (subnormal below 1024, the first
//            binade above); D = S * 2^-24.
//   BIASED   a converter pass ORs 0x6400 into each count (c < 1024), giving
//            fp16(1024 + c); D = S + 1024 * rowsum(Tt) = S + 1024 * 216 for
//            plA = III and S otherwise.
//   RECORDS  RAW, with the count tiles built in shared memory from shot
//            records (below).
//   SPLIT    int32 counts c < 16384 (the 256-byte rows land as TMA brings
//            them, 216 rows per chunk, four chunks per tile): converter warps
//            rewrite each row in place as two 128-byte planes, the low plane
//            holding c mod 2048 as fp16 bits (c_lo * 2^-24, as RAW) and the
//            high plane fp16(c_hi * 2^-13) with c_hi = c >> 11, so that
//            c_lo * 2^-24 + c_hi * 2^-13 = c * 2^-24.  Each K-step issues one
//            MMA per plane (same Tt operand, B stride 256 bytes per row) into
//            the same accumulator: D = S * 2^-24 again.
// Every partial sum is an integer multiple of 2^-24 below 2^22 units (216
// counts of at most 16383), so FP32 accumulation in TMEM is exact and the
// level-B warps recover the same integer the ALU path computes.
//
// Range check: the encodings are exact only for counts in range, so the
// warps that do not build or convert (RAW: warps 2, 3) read every landed
// count, and the converter warps check what they convert; a count above the
// stated shots per basis (or negative) latches LRE_ERR_SHOTS_MISMATCH.  RAW:
// the check reads a slot while its MMAs run, and the slot is released once
// both are done; the converting variants' MMAs wait for the conversion.
//
// Roles (256 threads, 320 for SPLIT; one CTA per SM):
//   warp 0     TMA producer into a ring of 3 chunk slots (RAW/BIASED: one
//              chunk = 16 alB groups = 432 rows of 128 bytes; SPLIT: 8 alB
//              groups = 216 rows of 256 bytes); a slot is released by
//              tcgen05.commit once the MMAs reading it have completed
//   warp 1     issues the MMAs (M = 128, K = 16) of each chunk into the
//              tile's accumulator (224 columns; two tile buffers in 512)
//   warps 2,3  RAW: range check; BIASED: range check and convert in place
//              (half the rows each); SPLIT (with warps 8, 9): range check and
//              plane conversion, two rows per warp at a time
//   warps 4,5  level B of even tiles from TMEM lanes 0..63
//   warps 6,7  level B of odd tiles from TMEM lanes 64..127 (rows 64..127 of
//              the operand repeat Tt, so those lanes hold the same D)
// Level B: thread plA reads its 216 columns 32 at a time, contracts the next
// three qubits (alB, olB) on the ALU and writes 64 outputs.  Every barrier has
// in-order consumers only, so parity waits cannot alias, and every wait is
// bounded by time.
#include <cuda_runtime.h>

#include <cudaTypedefs.h>

#include <vector>

#include "lre_internal.cuh"
#include "passes.cuh"
#include "sm103.cuh"

namespace lre {
namespace {

using namespace passes;

enum : int { V_RAW = 0, V_BIASED = 1, V_RECORDS = 2, V_SPLIT = 3, V_RAW9 = 4, V_RAW7 = MMA_SEVEN };

// V_RAW7: the raw pass folding seven qubits: the six of the tile and the
// last one, qubit n (the top ternary digit of ah, the top bit of oh), so
// that CTAs working side by side still read neighbouring 128-byte count
// chunks (qubit 7, whose outcome is bit 0 of oh, would have them read every
// other chunk at a time: 256-byte L2 lines fetched twice as fast as used).
// Tiles come in groups of six, a supertile (AH, OH): the three axes a times
// the two outcomes o of qubit n, ah = AH + a 3^(n-7), oh = OH + o 2^(n-7), in
// the order (a, o) = (0,0), (0,1), (1,0), ... .  Every tile's level A and B
// run as in the six-qubit pass; then the level-B warps of lanes 0..63 (pair
// 0) add all six results into the letter I of qubit n, and those of lanes
// 64..127 (pair 1, the same values, since rows 64..127 of the operand repeat
// Tt) take D(a, 0) - D(a, 1) into the letter a + 1 (the outcome-1 tile
// converted with the opposite sign).  Both pairs read every tile, from the
// two TMEM tile buffers in turn.  The output is [3^(n-7)][2^(n-7)][16384],
// column pn * 4096 + plB * 64 + plA: four blocks where the six-qubit pass
// writes six, and the later passes (qubits 7..n-1) have one qubit less to
// fold; the final pass puts qubit n's letter back at the top of the index.
// Measured at n = 14 (1000 shots): the later passes drop from 5.4 to 4.2 ms,
// but this pass takes 28.3 ms against the six-qubit pass's 25.6-25.9: its
// CTAs end between 24.6 and 27.9 ms where the six-qubit pass's end within
// 0.2 ms (dealing supertiles out dynamically made it 30.4 ms), so the six
// qubit pass stays the default (lre_debug_set_first7 selects this one).

// V_RAW9: the raw pass fused with the second fold pass (three more qubits)
// through L2, in one cooperative launch whose CTAs take one of two roles.
// CTAs 0..np1-1 run the raw pass over the tiles in group-major order (a group
// = the 27 x 8 tiles one second-pass column reads: the low ternary digits of
// ah and the low bits of oh), counts streamed with an evict-first hint; their
// level-B warps write a tile's 4096 int32 partials into slot G mod F9_RING of
// a scratch ring (3.5 MB per group, small enough to stay in L2) and count the
// tile in tiles_done[slot].  The other CTAs run the second pass: each of their
// eight warps takes jobs (a group and 32 columns) cw, cw + W, ... in order,
// waits for the group's tiles, has TMA bring the job's 216 rows x 32 columns
// from the ring into its own shared-memory buffer (27 KB; eight loads in
// flight per SM), contracts al2, ol2, stores the 64 outputs, drops the
// consumed 128-byte lines from L2 without write-back and counts the job in
// jobs_done[slot], which the level-B warps wait for before reusing the slot.
// Every wait points at an earlier group and every warp takes its jobs in
// increasing order, so the smallest unfinished tile can always proceed; the
// cooperative launch makes every CTA resident.
constexpr int F9_RING = 16;
constexpr int F9_JOBS = 4096 / 32;             // second-pass jobs per group
constexpr int F9_WARPS = 8;                    // second-pass warps per CTA
constexpr int F9_BOX = 216 * 32 * 4;           // one job's rows: 216 x 32 int32

constexpr int MMA_THREADS = 256;
constexpr int MMA_R = 3;                       // ring slots of one chunk each
constexpr int CHUNK_ROWS = 432;                // 16 alB groups x 27 rows
constexpr int SLOT_BYTES = CHUNK_ROWS * 128;   // int16 rows of 64 outcomes
// SPLIT chunks: 8 alB groups (216 int32 rows, N = 64) three times, then alB
// 24..26 (81 rows, N = 32, whose padded alB = 27 reads rows 81..107).
// Measured: 216-row chunks in 3 slots (2.70 ms at n = 12) beat 108-row
// chunks in 6 slots (3.64 ms): the per-chunk fixed costs outweigh the
// extra loads in flight.
constexpr int SPLIT_ROWS = 216;
constexpr int SPLIT_TAIL = 81;
constexpr int SPLIT_CHUNKS = 4;                // 3 x 216 + 81 = 729 rows
constexpr int64_t SPLIT_MAX = 16383;           // SPLIT: largest count (216 c < 2^22)
static_assert(3 * SPLIT_ROWS + SPLIT_TAIL == 729, "chunks cover the tile");
static_assert(SPLIT_ROWS * 256 == SLOT_BYTES, "a SPLIT chunk fills one slot");
static_assert(4 * 27 <= SPLIT_ROWS, "padded alB group stays in the slot");

template <int V>
struct MmaCfg {
  static constexpr int CPT = V == V_SPLIT ? SPLIT_CHUNKS : 2;       // chunks per tile
  static constexpr int R = MMA_R;                                     // ring slots
  static constexpr int SLOT = SLOT_BYTES;
  static constexpr int THREADS = V == V_SPLIT ? 320 : 256;  // + converters
  static constexpr int CONV_WARPS = V == V_SPLIT ? 4 : 2;            // arrivals on conv: 32 each
};
constexpr int A_BYTES = 16 * 28 * 128;         // 128 x 224 fp16, core-matrix layout
constexpr int OFF_RING = A_BYTES;
constexpr int OFF_BAR = OFF_RING + MMA_R * SLOT_BYTES;
constexpr int MMA_SMEM = OFF_BAR + 32 * 8 + 1024;
constexpr int BIAS = 1024 * 216;
constexpr uint32_t TMEM_COLS = 512;            // two tile accumulators
constexpr uint32_t TILE_COLS = 256;
constexpr uint32_t BOX_BIG = 216, BOX_TAIL = 81;  // TMA boxes: 8 and 3 alB groups
static_assert(MMA_SMEM <= 232448, "shared memory of one CTA");
static_assert(F9_WARPS * (F9_BOX + 8) + 1024 <= MMA_SMEM, "second-pass buffers and barriers fit");
static_assert(2 * BOX_BIG <= CHUNK_ROWS && BOX_BIG + BOX_TAIL <= CHUNK_ROWS, "chunk fits its slot");
// the N = 96 chain reads alB = 27 (rows 729..755 of the tile): still inside the slot
static_assert(12 * 27 <= CHUNK_ROWS, "padded alB group stays in the slot");

__device__ __forceinline__ int32_t d_to_int(uint32_t bits, float scale, int32_t sub) {
  // x * scale is an integer of magnitude below 2^22; adding 1.5 * 2^23 puts it
  // in the low mantissa bits
  return __float_as_int(fmaf(__uint_as_float(bits), scale, 12582912.f)) - 0x4B400000 - sub;
}

// RECORDS: the count tiles are built in shared memory from shot records
// grouped by tile and chunk (records.cu: entries (al << 6) | ol per tile
// row, bucket starts in offs, bucket = oh * 2 + chunk) instead of being
// loaded by TMA: warps 0, 2 and 3 each own one ring slot; once the MMAs of
// the slot's previous chunk are done they clear it (only the cells that chunk
// set, when it was sparse), add the bucket's entries with packed 16-bit
// shared-memory atomics (eight loads in flight per lane), make the
// writes visible to the tensor cores (proxy fence) and arrive on the slot.
// Tile rows are numbered from tile_begin / 2^(n-6) in entries and offs.
// shots: the shots per basis (the range of every count).
template <int V>
__global__ void __launch_bounds__(MmaCfg<V>::THREADS, 1)
    fold_first6_mma(const __grid_constant__ CUtensorMap map_big, const __grid_constant__ CUtensorMap map_tail,
                    const __grid_constant__ CUtensorMap map_s, int np1, int f9_opts, const uint4 *__restrict__ gA,
                    int32_t *__restrict__ out, int8_t *__restrict__ out_hi, int n,
                    int64_t tile_begin, int64_t tile_end, const uint16_t *__restrict__ entries,
                    const int32_t *__restrict__ offs, int64_t shots, int64_t row_base, int32_t *__restrict__ scratch,
                    unsigned *__restrict__ f9, int *status) {
  constexpr bool BIASED = V == V_BIASED, RECORDS = V == V_RECORDS, SPLIT = V == V_SPLIT;
  constexpr bool RAWLIKE = V == V_RAW || V == V_RAW9 || V == V_RAW7, F9 = V == V_RAW9, SEVEN = V == V_RAW7;
  // F9 counters: f9[0] the next job, f9[1 + s] tiles done, f9[1 + F9_RING + s] jobs done (slot s)
  constexpr int CPT = MmaCfg<V>::CPT;
  constexpr int MR = MmaCfg<V>::R;          // ring slots
  constexpr int SLOT = MmaCfg<V>::SLOT;     // bytes per slot
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024u - (sm103::smem_addr(smem_raw) & 1023u)) & 1023u);
  uint8_t *Am = smem;
  uint8_t *ring = smem + OFF_RING;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
  uint64_t *conv = full + MR;
  uint64_t *empty = conv + MR;
  uint64_t *tile_done = empty + MR;
  uint64_t *tile_free = tile_done + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tile_free + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_oh = (1ll << n) >> 6;
  // F9: CTAs np1.. run the second pass; the first np1 share the tiles
  const bool consumer = F9 && (int)blockIdx.x >= np1;
  const int nP = F9 ? np1 : (int)gridDim.x;

  if (!consumer)
    for (int i = threadIdx.x; i < A_BYTES / 16; i += MmaCfg<V>::THREADS) reinterpret_cast<uint4 *>(Am)[i] = gA[i];
  if (threadIdx.x == 0) *abort_flag = 0;
  if (threadIdx.x == 0 && !consumer) {
    for (int i = 0; i < MR; ++i) {
      sm103::mbar_init(&full[i], 1);
      sm103::mbar_init(&conv[i], 32 * MmaCfg<V>::CONV_WARPS);
      // RAW: released by the MMAs' commit and by the two range-check warps,
      // which read the slot while the MMAs run
      sm103::mbar_init(&empty[i], RAWLIKE ? 3 : 1);
    }
    for (int b = 0; b < 2; ++b) {
      sm103::mbar_init(&tile_done[b], 1);
      sm103::mbar_init(&tile_free[b], SEVEN ? 128 : 64);  // SEVEN: both pairs read every tile
    }
    sm103::fence_barrier_init();
  }
  sm103::fence_proxy_async_smem();  // A is read by the tensor cores
  if (warp == 1 && !consumer) sm103::tmem_alloc(tmem_slot, TMEM_COLS);
  sm103::tc_fence_before();
  __syncthreads();
  sm103::tc_fence_after();
  const uint32_t tmem = consumer ? 0u : *tmem_slot;
  auto give_up = [&]() {
    *abort_flag = 1;
    latch(status, LRE_ERR_TIMEOUT);
  };
  const int64_t tiles = tile_end - tile_begin;
  // units of work dealt out over the CTAs in turn: tiles, or SEVEN supertiles of six
  const int64_t units = SEVEN ? tiles / 6 : tiles;
  const int64_t my_units = (!consumer && units > blockIdx.x) ? (units - blockIdx.x + nP - 1) / nP : 0;
  const int64_t my_tiles = SEVEN ? 6 * my_units : my_units;
  const int64_t total = my_tiles * CPT;  // chunks of this CTA
  // SEVEN: the level-B work of every tile is done twice (both pairs), so it
  // is kept off warp 1's sub-partition (warp % 4 == 1, whose MMA issue sets
  // the pace): level B on warps 4, 6 (TMEM lanes 0..31 / 64..95) and 3, 7
  // (lanes 96..127), the range check on warps 2 and 5
  const bool conv_warp = SPLIT   ? (warp == 2 || warp == 3 || warp == 8 || warp == 9)
                         : SEVEN ? (warp == 2 || warp == 5)
                                 : (warp == 2 || warp == 3);
  const bool levelb_warp = SEVEN ? (warp == 3 || warp == 4 || warp == 6 || warp == 7) : (warp >= 4 && warp < 8);

  if (consumer) {
    // second pass (qubits 7..9): warp cw takes jobs cw, cw + W, ...; a job is
    // a group and 32 of its 4096 columns, output [G][64][4096] as the unfused
    // second pass writes it.  The ring slot is released as soon as the job's
    // copy has landed, and the next job's copy is in flight while this job's
    // outputs are stored.
    uint8_t *buf = smem + warp * F9_BOX;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + F9_WARPS * F9_BOX) + warp;
    if (lane == 0) {
      sm103::mbar_init(bar, 1);
      sm103::fence_barrier_init();
    }
    __syncwarp();
    const int64_t total_jobs = tiles / 216 * F9_JOBS;
    const int64_t W = (int64_t)(gridDim.x - np1) * F9_WARPS;
    const bool discard = (f9_opts & 1) != 0;
    // lane 0 waits for job j's group, then has TMA bring the job's rows into buf
    auto fetch = [&](int64_t j) -> bool {
      int ok = 1;
      if (lane == 0) {
        const int64_t G = j / F9_JOBS;
        const int slot = (int)(G % F9_RING);
        ok = sm103::poll_geq(f9 + 1 + slot, (unsigned)(2 * 216 * (G / F9_RING + 1)), abort_flag);
        if (ok) {
          // the tiles' generic-proxy stores, acquired above, before the async-proxy
          // read; this buffer's last generic reads before the copy overwrites it
          sm103::fence_proxy_async_global();
          sm103::fence_proxy_async_smem();
          sm103::mbar_arrive_expect_tx(bar, F9_BOX);
          sm103::tma_load_2d(buf, &map_s, (int)(j % F9_JOBS) * 32, slot * 216, bar);
        }
      }
      return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };
    int64_t j = (int64_t)(blockIdx.x - np1) * F9_WARPS + warp;
    bool inflight = false;
    if (j < total_jobs) {
      inflight = fetch(j);
      if (!inflight) give_up();
    }
    uint32_t phase = 0;
    while (inflight) {
      inflight = false;
      if (!sm103::mbar_wait(bar, phase, abort_flag)) {
        give_up();
        for (uint32_t it = 0; it < sm103::kSpinLimit; ++it)  // the copy in flight lands first
          if (sm103::mbar_try_wait(bar, phase)) break;
        break;
      }
      phase ^= 1u;
      const int64_t G = j / F9_JOBS;
      const int chunk = (int)(j % F9_JOBS);
      const int slot = (int)(G % F9_RING);
      if (discard) {
        // the 216 consumed 128-byte lines are dead: drop them from L2 unwritten,
        // ordered before the count that lets the slot be rewritten
        const int32_t *line0 = scratch + (int64_t)slot * 216 * 4096 + chunk * 32;
        for (int r = lane; r < 216; r += 32)
          asm volatile("discard.global.L2 [%0], 128;" ::"l"(line0 + r * 4096) : "memory");
        __threadfence();
      }
      __syncwarp();
      if (lane == 0) atomicAdd(f9 + 1 + F9_RING + slot, 1u);  // the copy has landed: slot reusable
      const int32_t *src = reinterpret_cast<const int32_t *>(buf) + lane;
      int32_t acc[64];
#pragma unroll
      for (int p = 0; p < 64; ++p) acc[p] = 0;
#pragma unroll
      for (int al2 = 0; al2 < 27; ++al2) {  // unrolled: the Pauli digits index registers
        int32_t v[8];
#pragma unroll
        for (int ol2 = 0; ol2 < 8; ++ol2) v[ol2] = src[(al2 * 8 + ol2) * 32];
        wht<3>(v);
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[block_pauli(al2, m, 3)] += v[m];
      }
      __syncwarp();  // buf fully read before the next copy overwrites it
      const int64_t jn = j + W;
      if (jn < total_jobs) {
        inflight = fetch(jn);
        if (!inflight) give_up();
      }
      int32_t *o = out + G * 64 * 4096 + chunk * 32 + lane;
#pragma unroll
      for (int p = 0; p < 64; ++p) __stcs(o + p * 4096, acc[p]);
      j = jn;
    }
  } else if (RECORDS && (warp == 0 || warp == 2 || warp == 3)) {
    const int bw = warp == 0 ? 0 : warp - 1;  // builder of chunks g = bw (mod 3): always slot bw
    const int64_t tr0 = tile_begin / n_oh;
    const int64_t row_entries = 729 * shots;
    const int nb = (int)(2 * n_oh);  // buckets per tile row: (oh, chunk)
    constexpr int32_t SPARSE = 2048;  // re-zero only the touched cells below this many entries
    uint4 *slot4 = reinterpret_cast<uint4 *>(ring + bw * SLOT);
    uint32_t *slot32 = reinterpret_cast<uint32_t *>(ring + bw * SLOT);
    const uint16_t *pent = nullptr;  // the slot's previous chunk: its entries and row base
    int32_t pe0 = 0, pe1 = -1;
    int pbase = 0;
    for (int64_t g = bw; g < total; g += MR) {
      const int64_t tile = tile_begin + blockIdx.x + (g >> 1) * nP;
      const int c = (int)(g & 1);
      const int64_t ah = tile / n_oh, oh = tile - ah * n_oh;
      if (g >= MR && !sm103::mbar_wait(&empty[bw], (uint32_t)((g / MR - 1) & 1), abort_flag)) {
        give_up();
        break;
      }
      if (pent && pe1 - pe0 <= SPARSE) {  // zero the cells the previous chunk set
        for (int32_t e = pe0 + lane; e < pe1; e += 32 * 8) {
          uint32_t v[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = e + 32 * k < pe1 ? (uint32_t)__ldcs(pent + e + 32 * k) : 0xFFFFFFFFu;
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (v[k] != 0xFFFFFFFFu) slot32[((uint32_t)((int)(v[k] >> 6) - pbase) * 64 + (v[k] & 63u)) >> 1] = 0u;
        }
      } else {
        for (int k = lane; k < CHUNK_ROWS * 8; k += 32) slot4[k] = make_uint4(0, 0, 0, 0);
      }
      __syncwarp();
      const uint16_t *ent = entries + (ah - tr0) * row_entries;
      const int32_t *of = offs + (ah - tr0) * nb;
      const int bk = (int)(oh * 2 + c);
      const int32_t e0 = of[bk], e1 = bk + 1 < nb ? of[bk + 1] : (int32_t)row_entries;
      const int base = c * 432;
      for (int32_t e = e0 + lane; e < e1; e += 32 * 8) {
        uint32_t v[8];  // eight independent loads in flight per lane, then their adds
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = e + 32 * k < e1 ? (uint32_t)__ldcs(ent + e + 32 * k) : 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (v[k] != 0xFFFFFFFFu) {
            const uint32_t idx = (uint32_t)((int)(v[k] >> 6) - base) * 64 + (v[k] & 63u);
            atomicAdd(&slot32[idx >> 1], 1u << ((idx & 1u) << 4));
          }
      }
      sm103::fence_proxy_async_smem();  // the tensor cores read what this warp wrote
      __syncwarp();
      if (lane == 0) sm103::mbar_arrive(&full[bw]);
      pent = ent;
      pe0 = e0;
      pe1 = e1;
      pbase = base;
    }
  } else if (warp == 0) {
    if (lane == 0) {
      int64_t g = 0;
      for (; g < total && !*abort_flag; ++g) {
        const int64_t tile = tile_begin + blockIdx.x + (g / CPT) * nP;
        const int c = (int)(g % CPT);
        int64_t ah, oh;
        if constexpr (F9) {  // group-major: group G = (gah, goh), k = (al2, ol2)
          const int64_t G = tile / 216, k = tile - G * 216, n_goh = n_oh >> 3;
          const int64_t gah = G / n_goh, goh = G - gah * n_goh;
          ah = gah * 27 + k / 8;
          oh = goh * 8 + (k & 7);
        } else if constexpr (SEVEN) {  // supertile st = (AH, OH), tile t6 = (a, o) of qubit n
          const int64_t lt = g / CPT, st = blockIdx.x + (lt / 6) * nP, n_oh2 = n_oh >> 1;
          const int t6 = (int)(lt % 6);
          const int64_t AH = st / n_oh2, OH = st - AH * n_oh2;
          ah = AH + (t6 >> 1) * (units / n_oh2);  // units / 2^(n-7) = 3^(n-7)
          oh = OH + (t6 & 1) * n_oh2;
        } else {
          ah = tile / n_oh;
          oh = tile - ah * n_oh;
        }
        const int slot = (int)(g % MR);
        if (g >= MR && !sm103::mbar_wait(&empty[slot], (uint32_t)((g / MR - 1) & 1), abort_flag)) {
          give_up();
          break;
        }
        uint8_t *dst = ring + slot * SLOT;
        const int x = (int)(oh * 64);
        if constexpr (SPLIT) {  // one box of int32 rows: 216, or 81 for alB 24..26
          const int y = (int)(ah * 729 + c * SPLIT_ROWS - row_base);
          sm103::mbar_arrive_expect_tx(&full[slot], (c < SPLIT_CHUNKS - 1 ? SPLIT_ROWS : SPLIT_TAIL) * 256);
          sm103::tma_load_2d(dst, c < SPLIT_CHUNKS - 1 ? &map_big : &map_tail, x, y, &full[slot]);
        } else {
          const int y = (int)(ah * 729 + c * 432 - row_base);
          sm103::mbar_arrive_expect_tx(&full[slot], (BOX_BIG + (c ? BOX_TAIL : BOX_BIG)) * 128);
          if constexpr (F9) {  // counts are read once: keep the scratch ring in L2 instead
            const uint64_t pol = sm103::l2_evict_first();
            sm103::tma_load_2d_hint(dst, &map_big, x, y, &full[slot], pol);
            sm103::tma_load_2d_hint(dst + BOX_BIG * 128, c == 0 ? &map_big : &map_tail, x, y + (int)BOX_BIG,
                                    &full[slot], pol);
          } else {
            sm103::tma_load_2d(dst, &map_big, x, y, &full[slot]);
            if (c == 0)
              sm103::tma_load_2d(dst + BOX_BIG * 128, &map_big, x, y + (int)BOX_BIG, &full[slot]);
            else
              sm103::tma_load_2d(dst + BOX_BIG * 128, &map_tail, x, y + (int)BOX_BIG, &full[slot]);
          }
        }
      }
      for (int64_t q = g > MR ? g - MR : 0; q < g; ++q)  // drain in-flight loads
        for (uint32_t it = 0; it < sm103::kSpinLimit; ++it)
          if (sm103::mbar_try_wait(&full[q % MR], (uint32_t)((q / MR) & 1))) break;
    }
  } else if (warp == 1) {
    const uint32_t a_base = sm103::smem_addr(Am);
    int64_t g = 0;
    for (; g < total; ++g) {
      const int slot = (int)(g % MR);
      const int64_t lt = g / CPT;
      const int c = (int)(g % CPT);
      const int tb = (int)(lt & 1);
      if (c == 0 && lt >= 2 &&
          !sm103::mbar_wait(&tile_free[tb], (uint32_t)(((lt >> 1) - 1) & 1), abort_flag)) {
        give_up();
        break;
      }
      if (!sm103::mbar_wait((RECORDS || RAWLIKE) ? &full[slot] : &conv[slot], (uint32_t)((g / MR) & 1),
                            abort_flag)) {
        give_up();
        break;
      }
      sm103::tc_fence_after();
      if (lane == 0) {
        const uint32_t b_base = sm103::smem_addr(ring + slot * SLOT);
        if constexpr (SPLIT) {
          const uint32_t d = tmem + tb * TILE_COLS + c * 64;
          const uint32_t idesc = sm103::umma_idesc_f16(128, c < SPLIT_CHUNKS - 1 ? 64 : 32);
#pragma unroll 1
          for (int kk = 0; kk < 14; ++kk) {
            const int brow = kk < 13 ? 2 * kk : 25;
            const uint64_t ad = sm103::umma_desc(a_base + kk * 256, 128, 28 * 128);
#pragma unroll
            for (int pl = 0; pl < 2; ++pl) {  // low plane, then high plane of the same rows
              const uint64_t bd = sm103::umma_desc(b_base + brow * 256 + pl * 128, 256, 27 * 256);
              sm103::umma_f16(d, ad, bd, idesc, kk > 0 || pl > 0);
            }
          }
        } else {
          const uint32_t d = tmem + tb * TILE_COLS + c * 128;
          const uint32_t idesc = sm103::umma_idesc_f16(128, c ? 96 : 128);
#pragma unroll 1
          for (int kk = 0; kk < 14; ++kk) {
            const int brow = kk < 13 ? 2 * kk : 25;
            const uint64_t ad = sm103::umma_desc(a_base + kk * 256, 128, 28 * 128);
            const uint64_t bd = sm103::umma_desc(b_base + brow * 128, 128, 27 * 128);
            sm103::umma_f16(d, ad, bd, idesc, kk > 0);
          }
        }
        sm103::umma_commit(&empty[slot]);                       // slot reusable when these finish
        if (c == CPT - 1) sm103::umma_commit(&tile_done[tb]);   // whole tile accumulated
      }
      __syncwarp();
    }
    // no MMA may still run when TMEM is released
    if (lane == 0 && g > 0) {
      const int64_t q = g - 1;
      for (uint32_t it = 0; it < sm103::kSpinLimit; ++it)
        if (sm103::mbar_try_wait(&empty[q % MR], (uint32_t)((q / MR) & 1))) break;
    }
  } else if (conv_warp) {
    // range check of every landed count (and the BIASED / SPLIT conversion)
    uint32_t mx = 0;  // SPLIT: largest count as unsigned; else the two 16-bit halves' maxima
    for (int64_t g = 0; g < total; ++g) {
      const int slot = (int)(g % MR);
      const int c = (int)(g % CPT);
      if (!sm103::mbar_wait(&full[slot], (uint32_t)((g / MR) & 1), abort_flag)) {
        give_up();
        break;
      }
      uint8_t *base = ring + slot * SLOT;
      if constexpr (SPLIT) {
        const int rows = c < SPLIT_CHUNKS - 1 ? SPLIT_ROWS : SPLIT_TAIL;
        const int cw = warp < 4 ? warp - 2 : warp - 6;  // 0..3
        const int q = lane & 15;                        // 16 bytes (4 counts) of a 256-byte row
        for (int r0 = 2 * cw; r0 < rows; r0 += 8) {    // two rows per warp at a time
          const int row = r0 + (lane >> 4);
          const bool act = row < rows;
          uint4 v = make_uint4(0, 0, 0, 0);
          if (act) v = *reinterpret_cast<const uint4 *>(base + row * 256 + q * 16);
          __syncwarp();  // the whole row is read before any lane rewrites it
          if (act) {
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
            uint32_t lo[4], hi[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              mx = max(mx, w[k]);
              lo[k] = w[k] & 0x7FFu;                 // fp16 bits of c_lo * 2^-24
              const uint32_t h = w[k] >> 11;
              // fp16 bits of h * 2^-13: the float exponent of h lowered by 13,
              // rebiased from 127 to 15, mantissa cut to 10 bits (exact, h < 2048)
              hi[k] = h ? (__float_as_uint((float)h) >> 13) - (125u << 10) : 0u;
            }
            *reinterpret_cast<uint2 *>(base + row * 256 + q * 8) =
                make_uint2(lo[0] | (lo[1] << 16), lo[2] | (lo[3] << 16));
            *reinterpret_cast<uint2 *>(base + row * 256 + 128 + q * 8) =
                make_uint2(hi[0] | (hi[1] << 16), hi[2] | (hi[3] << 16));
          }
        }
      } else {
        const int rows = c ? (int)(BOX_BIG + BOX_TAIL) : (int)(2 * BOX_BIG);
        uint4 *v4 = reinterpret_cast<uint4 *>(base);
#pragma unroll 4
        for (int k = (SEVEN ? (warp == 5) : warp - 2) * 32 + lane; k < rows * 8; k += 64) {
          uint4 v = v4[k];
          mx = __vmaxu2(__vmaxu2(mx, v.x), __vmaxu2(v.y, __vmaxu2(v.z, v.w)));
          if constexpr (BIASED) {  // counts -> fp16(1024 + c)
            v.x |= 0x64006400u; v.y |= 0x64006400u; v.z |= 0x64006400u; v.w |= 0x64006400u;
            v4[k] = v;
          }
        }
      }
      if constexpr (RAWLIKE) {  // done reading: one arrival per warp on the slot's release
        __syncwarp();
        if (lane == 0) sm103::mbar_arrive(&empty[slot]);
      } else {
        sm103::fence_proxy_async_smem();
        sm103::mbar_arrive(&conv[slot]);
      }
    }
    // a count above the shots per basis (a negative one reads as a large
    // unsigned value) is outside the encoding's exact range
    const uint32_t top = SPLIT ? mx : max(mx & 0xFFFFu, mx >> 16);
    const int64_t lim = BIASED ? (shots < 1023 ? shots : 1023) : shots;
    if ((int64_t)top > lim) latch(status, LRE_ERR_SHOTS_MISMATCH);
  } else if (levelb_warp) {
    // warps 4,5: even tiles, TMEM lanes 0..63; warps 6,7: odd tiles, lanes 64..127
    // (SEVEN: pair 0 = warps 4, 3 and pair 1 = warps 6, 7, every tile)
    const int pair = SEVEN ? (warp == 6 || warp == 7) : (warp - 4) >> 1;
    const int quarter = warp & 3;
    const int plA = (quarter & 1) * 32 + lane;
    const int hi_from = planes_hi_from(shots);  // split planes: identities from which the high plane counts
    const float scale = BIASED ? 1.f : 16777216.f;
    const int32_t sub = BIASED && plA == 0 ? BIAS : 0;
    int pend = -1;  // F9: ring slot of this warp's last tile, written but not yet counted
    // F9: make this warp's ring stores visible (TMA reads them back, through
    // the async proxy) and count the tile; two warps per tile
    auto publish = [&](int slot) {
      sm103::fence_proxy_async_global();
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicAdd(f9 + 1 + slot, 1u);
    };
    int32_t acc[64];  // SEVEN: carried over the tiles one output block gathers
    // SEVEN: both pairs take every tile, from the buffers in turn; otherwise
    // pair b takes the tiles of buffer b
    for (int64_t lt = SEVEN ? 0 : pair; lt < my_tiles; lt += SEVEN ? 1 : 2) {
      const int tb = SEVEN ? (int)(lt & 1) : pair;
      if (!sm103::mbar_wait(&tile_done[tb], (uint32_t)((lt >> 1) & 1), abort_flag)) {
        give_up();
        break;
      }
      sm103::tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + tb * TILE_COLS;
      // SEVEN: tile t6 = (a, o) of its supertile; pair 0 gathers all six
      // (letter I), pair 1 the two of one axis, the o = 1 tile negated
      const int t6 = SEVEN ? (int)(lt % 6) : 0;
      const bool fresh = !SEVEN || (pair == 0 ? t6 == 0 : (t6 & 1) == 0);
      const bool flush = !SEVEN || (pair == 0 ? t6 == 5 : (t6 & 1) == 1);
      const float sc = (SEVEN && pair == 1 && (t6 & 1)) ? -scale : scale;
      if (fresh) {
#pragma unroll
        for (int p = 0; p < 64; ++p) acc[p] = 0;
      }
      // columns 32 grp .. 32 grp + 31 hold alB = 4 grp .. 4 grp + 3; the load of
      // the next 32 columns is in flight while these are contracted
      uint32_t r[2][32];
      sm103::tmem_ld32(ta, r[0]);
#pragma unroll
      for (int grp = 0; grp < 7; ++grp) {
        sm103::tmem_ld_wait(r[grp & 1]);
        if (grp < 6) sm103::tmem_ld32(ta + (grp + 1) * 32, r[(grp + 1) & 1]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int alB = grp * 4 + j;
          if (alB < 27) {
            int32_t v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = d_to_int(r[grp & 1][j * 8 + i], sc, sub);
            wht<3>(v);
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[block_pauli(alB, m, 3)] += v[m];
          }
        }
      }
      sm103::tc_fence_before();
      sm103::mbar_arrive(&tile_free[tb]);
      if (!flush) continue;
      const int64_t tile = tile_begin + blockIdx.x + lt * nP;
      // first element of this output block, and its column within the row
      // of letters (the split planes' run bound depends on it)
      const int blk = pair == 0 ? 0 : (t6 >> 1) + 1;
      const int64_t row = SEVEN ? ((int64_t)blockIdx.x + (lt / 6) * nP) * 16384 + blk * 4096 : tile * 4096;
      const int col = SEVEN ? blk * 4096 : 0;
      if constexpr (F9) {
        // the previous tile's stores have had this tile's work to complete:
        // count it now, so that its fence does not wait on them
        if (pend >= 0) publish(pend);
        pend = -1;
        // into the group's ring slot, once that slot's previous group has been
        // read by all of its second-pass jobs
        const int64_t G = tile / 216, k = tile - G * 216;
        const int slot = (int)(G % F9_RING);
        const unsigned need = (unsigned)(F9_JOBS * (G / F9_RING));
        if (need && !sm103::poll_geq(f9 + 1 + F9_RING + slot, need, abort_flag)) {
          give_up();
          break;
        }
        int32_t *o = scratch + ((int64_t)slot * 216 + k) * 4096 + plA;
#pragma unroll
        for (int p = 0; p < 64; ++p) o[p * 64] = acc[p];  // stays in L2 for the second pass
        pend = slot;
      } else if (out_hi) {  // split planes: low 16 bits, then the (signed) bits above
        unsigned short *lo = reinterpret_cast<unsigned short *>(out) + row + plA;
        signed char *hi = reinterpret_cast<signed char *>(out_hi) + row + plA;
        bool bad = false;  // a partial the planes cannot hold: a row above its shots
#pragma unroll
        for (int p = 0; p < 64; ++p) {
          __stcs(lo + p * 64, (unsigned short)(acc[p] & 0xFFFF));
          if (planes_hi_needed(col + p * 64 + (quarter & 1) * 32, hi_from, SEVEN ? 7 : 6)) {  // warp-uniform
            __stcs(hi + p * 64, (signed char)(acc[p] >> 16));
            bad |= acc[p] >= (1 << 23) || acc[p] < -(1 << 23);
          } else {
            bad |= acc[p] != (int32_t)(int16_t)acc[p];
          }
        }
        if (bad) latch(status, LRE_ERR_SHOTS_MISMATCH);
      } else {
        int32_t *o = out + row + plA;
#pragma unroll
        for (int p = 0; p < 64; ++p) __stcs(o + p * 64, acc[p]);
      }
    }
    if (F9 && pend >= 0) publish(pend);
  }
  sm103::tc_fence_before();
  __syncthreads();
  if (warp == 1 && !consumer) {
    sm103::tc_fence_after();
    sm103::tmem_dealloc(tmem, TMEM_COLS);
  }
}

// Tt as fp16 bits in the K-major core-matrix layout: row m (0..127) holds
// plA = m mod 64; column k = j*8 + olA over K-groups j = 0..27, where groups
// 0..25 are alA = j, group 26 is zero (it meets alA = 25 a second time in the
// last K-step) and group 27 is alA = 26.  Core matrix (m-group, j) sits at
// (m-group * 28 + j) * 128 bytes.
std::vector<uint16_t> make_a_operand() {
  std::vector<uint16_t> A(A_BYTES / 2, 0);
  const uint16_t one = 0x3C00, mone = 0xBC00;
  for (int m = 0; m < 128; ++m)
    for (int j = 0; j < 28; ++j) {
      if (j == 26) continue;
      const int al = j < 26 ? j : 26;
      for (int ol = 0; ol < 8; ++ol) {
        int v = 1;
        for (int q = 0, pp = m & 63, aa = al; q < 3; ++q, pp >>= 2, aa /= 3) {
          const int letter = pp & 3, axis = aa % 3, o = (ol >> q) & 1;
          if (letter == 0) continue;            // I: +1
          if (letter != axis + 1) { v = 0; break; }
          if (o) v = -v;                        // matching axis: (-1)^o
        }
        if (v == 0) continue;
        const size_t idx = ((size_t)(m >> 3) * 28 + j) * 64 + (m & 7) * 8 + ol;
        A[idx] = v > 0 ? one : mone;
      }
    }
  return A;
}

}  // namespace

size_t mma_operand_bytes() { return A_BYTES; }
uint32_t mma_box_rows(int which, int variant) {
  if (variant == 3) return which ? SPLIT_TAIL : SPLIT_ROWS;
  return which ? BOX_TAIL : BOX_BIG;
}
int64_t mma_max_count(int variant) { return variant == 1 ? 1023 : (variant == 3 ? SPLIT_MAX : 2047); }

// Launch the tensor-core first pass over tiles [tile_begin, tile_end) of an
// n-qubit count matrix (tile = ah * 2^(n-6) + oh): variant 0 (RAW) or 1
// (BIASED) for int16 counts, 3 (SPLIT) for int32 counts; variant 5 (RAW,
// seven qubits folded, n >= 8) over all tiles only, output
// [3^(n-7)][2^(n-7)][16384].  out_hi == nullptr: int32 partials at out;
// otherwise split planes, the low 16 bits at out (as uint16) and the bits
// above at out_hi (int8), exact while every partial is below 2^23 in
// magnitude (729 x shots, 2187 x shots for variant 5).  map_big / map_tail are tensor maps
// of the counts (int16, or int32 for SPLIT) with boxes of 216 / 81 rows x 64
// outcomes, whose row 0 is basis row_base; a_dev holds the operand written by
// mma_operand_upload; shots is the shots per basis, at most
// mma_max_count(variant): a count above it latches LRE_ERR_SHOTS_MISMATCH.
lre_status mma_first_pass(lre_ctx *ctx, const CUtensorMap &map_big, const CUtensorMap &map_tail, const void *a_dev,
                          int32_t *out, int8_t *out_hi, int n, int variant, int64_t shots, int64_t tile_begin,
                          int64_t tile_end, int64_t row_base, cudaStream_t s) {
  const int64_t tiles = tile_end - tile_begin;
  if (tiles <= 0) return LRE_OK;
  if (shots <= 0 || shots > mma_max_count(variant) ||
      (variant != 0 && variant != 1 && variant != 3 && variant != V_RAW7))
    return LRE_ERR_UNSUPPORTED;
  const bool seven = variant == V_RAW7;
  if (seven && (n < 8 || tile_begin != 0 || row_base != 0 || tiles != (ipow(3, n - 6) << (n - 6))))
    return LRE_ERR_UNSUPPORTED;
  const int64_t units = seven ? tiles / 6 : tiles;
  const int ctas = ctx->first_grid > 0 ? ctx->first_grid : ctx->num_sms;
  const int grid = (int)(units < ctas ? units : ctas);
  Launch L(ctx, variant == 3 ? "fold_first6_mma_split" : (seven ? "fold_first7_mma" : "fold_first6_mma"), s);
  auto kern = variant == 3 ? fold_first6_mma<V_SPLIT>
                           : (variant == 1 ? fold_first6_mma<V_BIASED>
                                           : (seven ? fold_first6_mma<V_RAW7> : fold_first6_mma<V_RAW>));
  const int threads = variant == 3 ? MmaCfg<V_SPLIT>::THREADS : MMA_THREADS;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, MMA_SMEM);
  kern<<<grid, threads, MMA_SMEM, s>>>(map_big, map_tail, map_tail, grid, 0, static_cast<const uint4 *>(a_dev), out,
                                       out_hi, n, tile_begin, tile_end, nullptr, nullptr, shots, row_base, nullptr,
                                       nullptr, ctx->d_status);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "tensor-core first pass launch");
}

// The raw pass fused with the second fold pass (V_RAW9) over all tiles of an
// n-qubit int16 count matrix (n >= 10): out receives the second pass's
// output [groups][64][4096] int32; scratch is the L2 ring (F9_RING x 216 x
// 4096 int32) and f9 its 1 + 2 F9_RING counters, zeroed here.  consumers:
// the CTAs that run the second pass (0: a sixth of the SMs); discard: drop
// each consumed ring line from L2 without write-back (one fence per job).
// One CTA per SM, launched cooperatively, since the two roles wait on each
// other.
lre_status mma_first_pass_fused9(lre_ctx *ctx, const CUtensorMap &map_big, const CUtensorMap &map_tail,
                                 const void *a_dev, int32_t *out, int32_t *scratch, unsigned *f9, int n,
                                 int64_t shots, int consumers, bool discard, cudaStream_t s) {
  const int64_t tiles = ipow(3, n - 6) << (n - 6);
  if (n < 10 || shots <= 0 || shots > mma_max_count(0) || tiles % 216 != 0) return LRE_ERR_UNSUPPORTED;
  const int grid = ctx->num_sms;
  const int q = consumers > 0 ? consumers : grid / 6;
  if (q < 1 || q >= grid) return LRE_ERR_INVALID_ARG;
  CUtensorMap map_s;
  const uint64_t dims[2] = {4096, (uint64_t)F9_RING * 216};
  const uint64_t strides[1] = {4096 * 4};
  const uint32_t box[2] = {32, 216};
  if (!encode_tensor_map_i32(&map_s, scratch, 2, dims, strides, box)) {
    ctx->last_error = "tensor map of the fused pass's ring rejected";
    return LRE_ERR_CUDA;
  }
  cudaError_t e = cudaMemsetAsync(f9, 0, (1 + 2 * F9_RING) * sizeof(unsigned), s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fused pass counters");
  Launch L(ctx, "fold_first9_mma", s);
  auto kern = fold_first6_mma<V_RAW9>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, MMA_SMEM);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(MmaCfg<V_RAW9>::THREADS);
  cfg.dynamicSmemBytes = MMA_SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const uint4 *a4 = static_cast<const uint4 *>(a_dev);
  int8_t *no_hi = nullptr;
  const uint16_t *no_ent = nullptr;
  const int32_t *no_offs = nullptr;
  const int np1 = grid - q;
  const int64_t t0 = 0, r0 = 0;
  const int opts = discard ? 1 : 0;
  e = cudaLaunchKernelEx(&cfg, kern, map_big, map_tail, map_s, np1, opts, a4, out, no_hi, n, t0, tiles, no_ent,
                         no_offs, shots, r0, scratch, f9, ctx->d_status);
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "fused tensor-core pass launch");
}
size_t mma_fused9_scratch_bytes() { return (size_t)F9_RING * 216 * 4096 * 4; }
size_t mma_fused9_counter_bytes() { return (1 + 2 * F9_RING) * sizeof(unsigned); }

// The same pass over tiles [tile_begin, tile_end) whose counts come from shot
// records grouped by tile (tile_bucket_run over the tile rows from
// tile_begin / 2^(n-6) on); every count must be at most 2047.
lre_status mma_first_pass_records(lre_ctx *ctx, const void *a_dev, const uint16_t *entries, const int32_t *offs,
                                  int64_t shots, int32_t *out, int8_t *out_hi, int n, int64_t tile_begin,
                                  int64_t tile_end, cudaStream_t s) {
  const int64_t tiles = tile_end - tile_begin;
  if (tiles <= 0) return LRE_OK;
  if (shots > mma_max_count(0)) return LRE_ERR_UNSUPPORTED;
  const int grid = (int)(tiles < ctx->num_sms ? tiles : ctx->num_sms);
  CUtensorMap unused{};
  Launch L(ctx, "fold_first6_mma_records", s);
  auto kern = fold_first6_mma<V_RECORDS>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, MMA_SMEM);
  kern<<<grid, MMA_THREADS, MMA_SMEM, s>>>(unused, unused, unused, grid, 0, static_cast<const uint4 *>(a_dev), out,
                                           out_hi, n, tile_begin, tile_end, entries, offs, shots, 0, nullptr,
                                           nullptr, ctx->d_status);
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
