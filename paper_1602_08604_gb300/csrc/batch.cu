// Batched LRE: many small tomography instances (each n <= 9, its own shot
// count) in ONE persistent kernel launch.
//
// Every instance has the pass list of lre_estimate with uniform shots: the
// fold passes of step (i) (Sec. III, Eq. 3; at most JMAX qubits per pass in
// registers, int32 partial sums, the last pass dividing by N 3^k and handing
// the exact integers T = S 3^(n-k) on) and the exact-integer assembly passes
// of step (ii) (Eq. 4).  All passes of all instances form one list ordered
// pass-major (the first pass of every instance, then the second, ...), cut
// into work units of a tuned number of items.  Each CTA of the persistent
// grid claims units from a device counter; a unit first waits (bounded by
// time) until every unit of its instance's previous pass has finished, then
// runs.  The pass-major order means a CTA only ever waits on units claimed
// before its own, so with every CTA resident the launch always completes.
//
// The "schedule" (JMAX, CTAs per SM, items per unit of the count-reading
// first passes and of the other passes) is picked by lre_batch_tune, which
// times the candidates on the caller's batch and keeps the fastest in the
// context.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "lre_internal.cuh"
#include "passes.cuh"
#include "sm103.cuh"

namespace lre {
namespace {

using namespace passes;

// pass bodies a unit can run
enum : int {
  C_FOLD = 0,    // + (J-1)*8 + first*4 + (in_i16 ? 0 : 2) + (final ? 1 : 0): J in 1..3 -> 0..23
                 //   (no final pass of three qubits: codes 17, 19, 21, 23 are never planned)
  C_ASM = 32,    // + (J-1)*4 + first*2 + last: J in 1..2 -> 32..39
  C_ASM6 = 48,   // + last: the first six assembly qubits of one 4096-coefficient block per unit
};

struct BPhase {
  int code;
  int inst;         // the instance the pass belongs to (host bookkeeping)
  int dep;          // index of the phase this one waits for (-1: none)
  unsigned dep_units;
  int per_unit;     // items per work unit: a multiple of 256 (each thread takes every 256th), or 1 (a
                    // shared-memory block)
  int64_t unit_begin, units, items;
  GenParams g;
  AsmParams a;
};

struct BatchState {
  unsigned long long next_unit;
  int abort;
};

template <int JMAX>
__device__ __forceinline__ void run_item(const BPhase &P, int64_t item) {
  switch (P.code) {
    case C_FOLD + 0: fold_item<1, int16_t, int32_t, M_STORE, false, true, false>(P.g, item); break;
    case C_FOLD + 1: fold_item<1, int16_t, int64_t, M_FINAL_U, false, true, false>(P.g, item); break;
    case C_FOLD + 2: fold_item<1, int32_t, int32_t, M_STORE, false, true, false>(P.g, item); break;
    case C_FOLD + 3: fold_item<1, int32_t, int64_t, M_FINAL_U, false, true, false>(P.g, item); break;
    case C_FOLD + 4: fold_item<1, int16_t, int32_t, M_STORE, false, false, true>(P.g, item); break;
    case C_FOLD + 5: fold_item<1, int16_t, int64_t, M_FINAL_U, false, false, true>(P.g, item); break;
    case C_FOLD + 6: fold_item<1, int32_t, int32_t, M_STORE, false, false, true>(P.g, item); break;
    case C_FOLD + 7: fold_item<1, int32_t, int64_t, M_FINAL_U, false, false, true>(P.g, item); break;
    case C_FOLD + 8: fold_item<2, int16_t, int32_t, M_STORE, false, true, false>(P.g, item); break;
    case C_FOLD + 9: fold_item<2, int16_t, int64_t, M_FINAL_U, false, true, false>(P.g, item); break;
    case C_FOLD + 10: fold_item<2, int32_t, int32_t, M_STORE, false, true, false>(P.g, item); break;
    case C_FOLD + 11: fold_item<2, int32_t, int64_t, M_FINAL_U, false, true, false>(P.g, item); break;
    case C_FOLD + 12: fold_item<2, int16_t, int32_t, M_STORE, false, false, true>(P.g, item); break;
    case C_FOLD + 13: fold_item<2, int16_t, int64_t, M_FINAL_U, false, false, true>(P.g, item); break;
    case C_FOLD + 14: fold_item<2, int32_t, int32_t, M_STORE, false, false, true>(P.g, item); break;
    case C_FOLD + 15: fold_item<2, int32_t, int64_t, M_FINAL_U, false, false, true>(P.g, item); break;
    case C_FOLD + 16:
      if constexpr (JMAX >= 3) fold_item<3, int16_t, int32_t, M_STORE, false, true, false>(P.g, item);
      break;
    case C_FOLD + 18:
      if constexpr (JMAX >= 3) fold_item<3, int32_t, int32_t, M_STORE, false, true, false>(P.g, item);
      break;
    case C_FOLD + 20:
      if constexpr (JMAX >= 3) fold_item<3, int16_t, int32_t, M_STORE, false, false, true>(P.g, item);
      break;
    case C_FOLD + 22:
      if constexpr (JMAX >= 3) fold_item<3, int32_t, int32_t, M_STORE, false, false, true>(P.g, item);
      break;
    case C_ASM + 0: asm_item<NumI64, 1, false, false>(P.a, item); break;
    case C_ASM + 1: asm_item<NumI64, 1, false, true>(P.a, item); break;
    case C_ASM + 2: asm_item<NumI64, 1, true, false>(P.a, item); break;
    case C_ASM + 3: asm_item<NumI64, 1, true, true>(P.a, item); break;
    case C_ASM + 4: asm_item<NumI64, 2, false, false>(P.a, item); break;
    case C_ASM + 5: asm_item<NumI64, 2, false, true>(P.a, item); break;
    case C_ASM + 6: asm_item<NumI64, 2, true, false>(P.a, item); break;
    case C_ASM + 7: asm_item<NumI64, 2, true, true>(P.a, item); break;
    default: break;
  }
}

// Count-reading first fold pass (C == 1, store mode) with its rows staged
// through shared memory: a thread's items (first, first + 256, ...) read NA
// rows of 2^J counts each.  Instead of the register form's few row loads
// in flight next to its 4^J accumulators, each thread keeps STAGE_ROWS rows
// in flight as cp.async copies into its own shared-memory slots (no
// registers held), one commit group per row, the pipeline running across
// its items; each item's 4^J partials, contiguous because C == 1, leave as
// 16-byte stores (the register form's scalar stores put 4 bytes into 32
// separate sectors per warp instruction, which is what held this pass back).
// Slot layout [slot][16-byte half][thread]: a warp's 16-byte reads of one
// half are contiguous.
constexpr int STAGE_ROWS = 8;

template <int J, typename InT>
__device__ __forceinline__ void first_pass_staged(const BPhase &P, int64_t first, int count, unsigned char *stage) {
  constexpr int NA = J == 2 ? 9 : 27;
  constexpr int NO = 1 << J;
  constexpr int NP = 1 << (2 * J);
  constexpr int ROWB = NO * (int)sizeof(InT);  // 8, 16 or 32 bytes
  constexpr int HALVES = ROWB > 16 ? 2 : 1;
  constexpr int PIECE = ROWB > 16 ? 16 : ROWB;
  const GenParams &g = P.g;
  const InT *in = static_cast<const InT *>(g.in);
  const int t = threadIdx.x;
  const int total = count * NA;                   // rows of this thread, in item order
  // issue cursor: row `nf` of the stream, item `ni`, basis digit `nal`, and the
  // item's first row (one division per item, not per row)
  int nf = 0, ni = 0, nal = 0;
  const InT *nrow = nullptr;
  auto item_row0 = [&](int it) {
    const int64_t item = first + (int64_t)it * 256;
    const int64_t ah = item / g.n_oh, oh = item - ah * g.n_oh;
    return in + ((ah * NA) << g.r) + oh * NO;
  };
  if (total > 0) nrow = item_row0(0);
  auto issue = [&]() {  // the next row of the stream into its slot, then one commit group
    if (nf < total) {
      const InT *src = nrow + ((int64_t)nal << g.r);
#pragma unroll
      for (int h = 0; h < HALVES; ++h) {
        unsigned char *dst = stage + (((nf % STAGE_ROWS) * HALVES + h) * 256 + t) * PIECE;
        if constexpr (PIECE == 16)
          sm103::cp_async16(dst, reinterpret_cast<const unsigned char *>(src) + h * 16);
        else
          sm103::cp_async8(dst, src);
      }
      if (++nal == NA) {
        nal = 0;
        if (++ni < count) nrow = item_row0(ni);
      }
    }
    ++nf;
    sm103::cp_async_commit();  // empty past the end: keeps one group per row
  };
  for (int f = 0; f < STAGE_ROWS; ++f) issue();
  for (int it = 0; it < count; ++it) {
    int32_t acc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = 0;
#pragma unroll
    for (int al = 0; al < NA; ++al) {
      const int f = it * NA + al;
      sm103::cp_async_wait<STAGE_ROWS - 1>();  // row f has landed
      uint32_t w[ROWB / 4 > 0 ? ROWB / 4 : 1];
#pragma unroll
      for (int h = 0; h < HALVES; ++h) {
        const unsigned char *src = stage + (((f % STAGE_ROWS) * HALVES + h) * 256 + t) * PIECE;
        if constexpr (PIECE == 16) {
          const uint4 q = *reinterpret_cast<const uint4 *>(src);
          w[h * 4 + 0] = q.x; w[h * 4 + 1] = q.y; w[h * 4 + 2] = q.z; w[h * 4 + 3] = q.w;
        } else {
          const uint2 q = *reinterpret_cast<const uint2 *>(src);
          w[0] = q.x; w[1] = q.y;
        }
      }
      issue();  // row f + STAGE_ROWS, into the slot just read
      int32_t v[NO];
#pragma unroll
      for (int k = 0; k < NO; ++k) {
        if constexpr (sizeof(InT) == 2)
          v[k] = (int32_t)(int16_t)(uint16_t)(w[k >> 1] >> (16 * (k & 1)));
        else
          v[k] = (int32_t)w[k];
      }
      wht<J>(v);
#pragma unroll
      for (int m = 0; m < NO; ++m) acc[block_pauli(al, m, J)] += v[m];
    }
    int4 *o = reinterpret_cast<int4 *>(static_cast<int32_t *>(g.out) + (first + (int64_t)it * 256) * NP);
#pragma unroll
    for (int q = 0; q < NP / 4; ++q) o[q] = make_int4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
  }
  sm103::cp_async_wait<0>();
}

// Bytes of shared staging the staged first pass needs.
constexpr int STAGE_BYTES = STAGE_ROWS * 256 * 32;
static_assert(STAGE_BYTES <= ASM_TILE_SMEM, "the staging fits the assembly tile");

// Codes of the count-reading first passes (store mode, J >= 2) that run staged.
__host__ __device__ constexpr bool staged_code(int code) {
  return code == C_FOLD + 12 || code == C_FOLD + 14 || code == C_FOLD + 20 || code == C_FOLD + 22;
}

constexpr int BATCH_SMEM_PHASES = 4096;  // phase starts cached in shared memory up to this many

// Last phase with unit_begin <= u (binary search over the phase starts).
__device__ __forceinline__ int find_phase(const int64_t *begin, int nph, int64_t u) {
  int lo = 0, hi = nph - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begin[mid] <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int JMAX>
__global__ void __launch_bounds__(256, 2) batch_kernel(const BPhase *__restrict__ ph, const int64_t *__restrict__ gbegin,
                                                   int nph, unsigned *__restrict__ done, BatchState *st,
                                                   int64_t total_units, int tile_bytes, uint64_t wait_ns,
                                                   int *status) {
  // dynamic shared memory: [assembly tile (tile_bytes)][phase starts]
  extern __shared__ __align__(16) unsigned char bsmem[];
  int64_t *sbegin = reinterpret_cast<int64_t *>(bsmem + tile_bytes);
  NumI64::V *tile = reinterpret_cast<NumI64::V *>(bsmem);
  __shared__ int64_t s_unit;
  __shared__ int s_phase, s_ok;
  volatile int *abort = &st->abort;
  const bool cached = nph <= BATCH_SMEM_PHASES;
  if (cached)
    for (int k = threadIdx.x; k < nph; k += blockDim.x) sbegin[k] = gbegin[k];
  __syncthreads();
  const int64_t *begin = cached ? sbegin : gbegin;
  unsigned long long u = 0;
  if (threadIdx.x == 0) u = atomicAdd(&st->next_unit, 1ull);
  for (;;) {
    if (threadIdx.x == 0) {
      int p = -1, ok = 1;
      if ((int64_t)u < total_units && !*abort) {
        p = find_phase(begin, nph, (int64_t)u);
        const int dep = ph[p].dep;
        if (dep >= 0) {
          const unsigned need = ph[p].dep_units;
          const uint64_t t0 = sm103::globaltimer();
          for (uint32_t it = 0;; ++it) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(done + dep) : "memory");
            if (v >= need) break;
            if ((it & 63u) == 63u) {
              if (*abort || sm103::globaltimer() - t0 > wait_ns) {
                ok = 0;
                break;
              }
              __nanosleep(64);
            }
          }
        }
      }
      s_unit = (int64_t)u;
      s_phase = p;
      s_ok = ok;
    }
    __syncthreads();
    const int p = s_phase;
    if (p < 0) break;
    if (!s_ok) {
      if (threadIdx.x == 0) {
        *abort = 1;
        latch(status, LRE_ERR_TIMEOUT);
      }
      break;
    }
    // claim the next unit now: the atomic's round trip overlaps this unit's
    // work.  Every wait still points at a smaller unit than the waiter's own
    // (dependencies are earlier phases, a CTA's next unit is larger than its
    // current one), so the smallest unfinished unit always runs.
    if (threadIdx.x == 0) u = atomicAdd(&st->next_unit, 1ull);
    const BPhase &P = ph[p];
    if (P.code >= C_ASM6) {  // uniform across the CTA: every thread takes part in the block
      const int64_t blk = s_unit - P.unit_begin;
      const auto *in = static_cast<const long long *>(P.a.in);
      if (P.code == C_ASM6 + 1)
        asm_low6_block<NumI64, true>(in, P.a.out, blk, tile, P.a.scale);
      else
        asm_low6_block<NumI64, false>(in, P.a.out, blk, tile, P.a.scale);
    } else if (staged_code(P.code) && tile_bytes >= STAGE_BYTES &&
               ((reinterpret_cast<uintptr_t>(P.g.in) | reinterpret_cast<uintptr_t>(P.g.out)) & 15) == 0) {
      const int64_t first = (s_unit - P.unit_begin) * P.per_unit + threadIdx.x;
      const int64_t left = P.items > first ? (P.items - first + 255) / 256 : 0;
      const int count = (int)(left < P.per_unit / 256 ? left : P.per_unit / 256);
      unsigned char *stage = bsmem;
      if (count > 0) {
        switch (P.code) {
          case C_FOLD + 12: first_pass_staged<2, int16_t>(P, first, count, stage); break;
          case C_FOLD + 14: first_pass_staged<2, int32_t>(P, first, count, stage); break;
          case C_FOLD + 20:
            if constexpr (JMAX >= 3) first_pass_staged<3, int16_t>(P, first, count, stage);
            break;
          default:
            if constexpr (JMAX >= 3) first_pass_staged<3, int32_t>(P, first, count, stage);
            break;
        }
      }
    } else {
      const int64_t first = (s_unit - P.unit_begin) * P.per_unit + threadIdx.x;
      for (int k = 0; k < P.per_unit; k += 256) {
        const int64_t item = first + k;
        if (item < P.items) run_item<JMAX>(P, item);
      }
    }
    // publish the unit: the CTA barrier orders every thread's writes before
    // thread 0's device-scope fence, which orders them before the counter
    // the dependent units acquire (the usual grid-barrier pattern)
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(done + p, 1u);
    }
  }
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Plan {
  std::vector<BPhase> phases;
  size_t ws_bytes = 0;
  int64_t total_units = 0;
};

// Per-instance pass lists, workspace offsets relative to `base`, then the
// pass-major global order.
Plan build_plan(const lre_instance *inst, int count, int jmax, int first_unit, int unit, char *base) {
  std::vector<std::vector<BPhase>> per(count);
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    const lre_instance &I = inst[i];
    const int n = I.n;
    // fold passes
    int r = n, t = 0;
    int64_t C = 1;
    bool in16 = I.kind == LRE_COUNTS_I16;
    const void *in = I.counts;
    size_t bufA = 0, bufB = 0;
    struct P0 {
      int J, r;
      int64_t C;
      bool in16, last;
    };
    std::vector<P0> fp;
    while (r > 0) {
      // the final pass contracts at most two qubits: its int64 sums and FP64
      // quotients for three would need about 180 registers per thread, which
      // would leave one CTA per SM for every pass of the launch
      int J = std::min(r, jmax);
      if (r == 3 && J == 3) J = 2;
      fp.push_back({J, r, C, in16, J == r});
      const size_t ob = fp.back().last ? 0 : (size_t)ipow(6, r - J) * (size_t)ipow(4, J) * C * 4;
      if (fp.size() % 2) bufA = std::max(bufA, ob);
      else bufB = std::max(bufB, ob);
      t += J;
      r -= J;
      C *= ipow(4, J);
      in16 = false;
    }
    char *A = base + off;
    off += up256(bufA);
    char *Bf = base + off;
    off += up256(bufB);
    int64_t *T = nullptr;
    char *ab[2] = {nullptr, nullptr};
    if (I.rho) {
      T = reinterpret_cast<int64_t *>(base + off);
      off += up256((size_t)8 << (2 * n));
      ab[0] = base + off;
      off += up256((size_t)16 << (2 * n));
      ab[1] = base + off;
      off += up256((size_t)16 << (2 * n));
    }
    for (size_t k = 0; k < fp.size(); ++k) {
      BPhase b{};
      const P0 &q = fp[k];
      b.code = C_FOLD + (q.J - 1) * 8 + (k == 0 ? 4 : 0) + (q.in16 ? 0 : 2) + (q.last ? 1 : 0);
      GenParams &g = b.g;
      g.in = in;
      g.out = q.last ? static_cast<void *>(I.theta) : static_cast<void *>(k % 2 == 0 ? A : Bf);
      g.C = q.C;
      g.n_oh = 1ll << (q.r - q.J);
      g.items = ipow(3, q.r - q.J) * g.n_oh * q.C;
      g.r = q.r;
      g.n = n;
      g.shots = (double)I.shots;
      g.total = I.shots * ipow(3, n);
      g.T = T;
      for (int kk = 0; kk < 16; ++kk) {
        const double p3 = (double)ipow(3, kk <= n ? kk : 0);
        g.denom[kk] = (double)I.shots * p3;
        g.recip[kk] = 1.0 / g.denom[kk];
        g.dint[kk] = I.shots * ipow(3, kk <= n ? kk : 0);
        g.up3[kk] = kk <= n ? ipow(3, n - kk) : 0;
      }
      b.items = g.items;
      // a unit's claim, dependency wait and publish cost about as much as
      // moving a few hundred items' data: larger units amortise them (the
      // count-reading first passes and the rest are tuned separately)
      b.per_unit = k == 0 ? first_unit : unit;
      per[i].push_back(b);
      in = g.out;
    }
    if (I.rho) {
      const LastScaleArgs sc = int_assembly_scale(n, I.shots);
      int tt = 0, kk = 0;
      const void *ain = T;
      if (n >= 6) {
        // the first six qubits of each 4096-coefficient block in shared memory
        const bool last = n == 6;
        BPhase b{};
        b.code = C_ASM6 + (last ? 1 : 0);
        AsmParams &a = b.a;
        a.in = ain;
        a.out = last ? static_cast<void *>(I.rho) : static_cast<void *>(ab[0]);
        a.t = 0;
        a.n = n;
        a.items = 1ll << (2 * (n - 6));  // blocks
        a.scale = LastScale{sc.sh, sc.sl};
        b.items = a.items;
        b.per_unit = 1;
        per[i].push_back(b);
        ain = a.out;
        tt = 6;
        kk = 1;
      }
      while (tt < n) {
        const int J = (n - tt) >= 2 ? 2 : 1;
        const bool first = tt == 0, last = tt + J == n;
        BPhase b{};
        b.code = C_ASM + (J - 1) * 4 + (first ? 2 : 0) + (last ? 1 : 0);
        AsmParams &a = b.a;
        a.in = ain;
        a.out = last ? static_cast<void *>(I.rho) : static_cast<void *>(ab[kk & 1]);
        a.t = tt;
        a.n = n;
        a.items = (1ll << (2 * (n - tt - J))) << (2 * tt);
        a.scale = LastScale{sc.sh, sc.sl};
        b.items = a.items;
        b.per_unit = unit;
        per[i].push_back(b);
        ain = a.out;
        tt += J;
        ++kk;
      }
    }
  }
  Plan plan;
  plan.ws_bytes = off;
  size_t maxp = 0;
  for (auto &v : per) maxp = std::max(maxp, v.size());
  std::vector<int> last_index(count, -1);
  int64_t u = 0;
  for (size_t k = 0; k < maxp; ++k) {
    for (int i = 0; i < count; ++i) {
      if (k >= per[i].size()) continue;
      BPhase b = per[i][k];
      b.inst = i;
      b.units = (b.items + b.per_unit - 1) / b.per_unit;
      b.unit_begin = u;
      u += b.units;
      b.dep = last_index[i];
      b.dep_units = b.dep >= 0 ? (unsigned)plan.phases[b.dep].units : 0;
      last_index[i] = (int)plan.phases.size();
      plan.phases.push_back(b);
    }
  }
  plan.total_units = u;
  return plan;
}

lre_status validate(const lre_instance *inst, int count) {
  if (!inst || count <= 0) return LRE_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const lre_instance &I = inst[i];
    if (!I.counts || !I.theta || I.shots <= 0) return LRE_ERR_INVALID_ARG;
    if (I.kind != LRE_COUNTS_I16 && I.kind != LRE_COUNTS_I32) return LRE_ERR_INVALID_ARG;
    if (I.n < 1) return LRE_ERR_INVALID_ARG;
    if (I.n > 9) return LRE_ERR_UNSUPPORTED;
    if ((double)I.shots * (double)ipow(3, I.n) >= 2147483647.0) return LRE_ERR_UNSUPPORTED;  // int32 partials
  }
  return LRE_OK;
}

}  // namespace

lre_status batch_run(lre_ctx *ctx, const lre_instance *inst, int count, cudaStream_t s) {
  lre_status st = validate(inst, count);
  if (st != LRE_OK) return st;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "capture status");
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  const int jmax = ctx->batch_jmax;
  // A plan depends only on the descriptors and the schedule: an earlier call
  // with the same ones left its pass table in a device buffer (kept until
  // lre_destroy), so repeated and captured launches skip the host-side plan.
  const int sched[4] = {jmax, ctx->batch_first_unit, ctx->batch_unit, ctx->batch_stall_phase};
  std::vector<char> key(sizeof(lre_instance) * (size_t)count + sizeof(sched));
  std::copy(reinterpret_cast<const char *>(inst), reinterpret_cast<const char *>(inst + count), key.begin());
  std::copy(reinterpret_cast<const char *>(sched), reinterpret_cast<const char *>(sched + 4),
            key.begin() + sizeof(lre_instance) * (size_t)count);
  const lre_batch_entry *hit = nullptr;
  for (const auto &en : ctx->batch_cache)
    if (en.ws == ctx->ws && en.key == key) {
      hit = &en;
      break;
    }
  lre_batch_entry local;  // the plan of this call when it is not cached
  if (!hit) {
    if (capturing) {
      ctx->last_error = "lre_batch_run under stream capture: run the same batch once uncaptured first";
      return LRE_ERR_UNSUPPORTED;
    }
    // layout: [BatchState][done counters][phase table][instance workspaces]
    Plan probe = build_plan(inst, count, jmax, ctx->batch_first_unit, ctx->batch_unit, nullptr);
    const size_t nph = probe.phases.size();
    const size_t head = up256(sizeof(BatchState)) + up256(nph * sizeof(unsigned)) +
                        up256(nph * (sizeof(BPhase) + sizeof(int64_t)));
    if ((st = ensure_workspace(ctx, head + probe.ws_bytes)) != LRE_OK) return st;
    char *w = static_cast<char *>(ctx->ws);
    Plan plan = build_plan(inst, count, jmax, ctx->batch_first_unit, ctx->batch_unit, w + head);
    for (auto &b : plan.phases) b.g.status = ctx->d_status;
    if (ctx->batch_stall_phase >= 0)  // test hook: one more unit than exists, so the wait runs out
      for (size_t k = (size_t)ctx->batch_stall_phase; k < nph; ++k)
        if (plan.phases[k].dep >= 0) {
          plan.phases[k].dep_units += 1;
          break;
        }
    std::vector<char> tab(nph * (sizeof(BPhase) + sizeof(int64_t)));
    std::copy(reinterpret_cast<const char *>(plan.phases.data()),
              reinterpret_cast<const char *>(plan.phases.data()) + nph * sizeof(BPhase), tab.data());
    bool any_block = false;
    for (size_t k = 0; k < nph; ++k) {
      reinterpret_cast<int64_t *>(tab.data() + nph * sizeof(BPhase))[k] = plan.phases[k].unit_begin;
      any_block = any_block || plan.phases[k].code >= C_ASM6 || staged_code(plan.phases[k].code);
    }
    local.key = std::move(key);
    local.ws = ctx->ws;
    local.nph = nph;
    local.head = head;
    local.ws_bytes = probe.ws_bytes;
    local.total_units = plan.total_units;
    local.tile_bytes = any_block ? ASM_TILE_SMEM : 0;
    constexpr size_t kMaxPlans = 64;
    cudaError_t e = cudaSuccess;
    void *t = nullptr;
    if (ctx->batch_cache.size() < kMaxPlans && cudaMalloc(&t, tab.size()) == cudaSuccess) {
      local.table = t;
      e = cudaMemcpyAsync(t, tab.data(), tab.size(), cudaMemcpyHostToDevice, s);  // pageable: staged now
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // tab dies with this call
      ctx->batch_cache.push_back(local);
      hit = &ctx->batch_cache.back();
    } else {
      cudaGetLastError();
      // no room to keep it: the table goes into this call's workspace
      char *dph = w + up256(sizeof(BatchState)) + up256(nph * sizeof(unsigned));
      e = cudaMemcpyAsync(dph, tab.data(), tab.size(), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      local.table = dph;
      hit = &local;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch plan upload");
  }
  const size_t nph = hit->nph;
  char *w = static_cast<char *>(ctx->ws);
  BatchState *bs = reinterpret_cast<BatchState *>(w);
  unsigned *done = reinterpret_cast<unsigned *>(w + up256(sizeof(BatchState)));
  const BPhase *table = static_cast<const BPhase *>(hit->table);
  cudaError_t e = cudaMemsetAsync(w, 0, up256(sizeof(BatchState)) + up256(nph * sizeof(unsigned)), s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch state reset");
  int &occ = ctx->batch_occupancy[jmax >= 3 ? 1 : 0];  // queried once, outside any capture
  if (occ == 0) {
    // with the largest phase-start cache: every CTA of the grid must be resident
    const size_t sm_max = ASM_TILE_SMEM + BATCH_SMEM_PHASES * sizeof(int64_t);
    if (jmax >= 3) {
      cudaFuncSetAttribute(batch_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_max);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel<3>, 256, sm_max);
    } else {
      cudaFuncSetAttribute(batch_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_max);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel<2>, 256, sm_max);
    }
  }
  const int per_sm = std::max(1, std::min(occ, ctx->batch_ctas_per_sm));
  const int grid = ctx->num_sms * per_sm;  // every CTA resident: waits always resolve
  const int64_t *starts = reinterpret_cast<const int64_t *>(table + nph);
  const int tile_bytes = hit->tile_bytes;
  const int64_t total_units = hit->total_units;
  const size_t smem = tile_bytes + (nph <= (size_t)BATCH_SMEM_PHASES ? nph * sizeof(int64_t) : 0);
  const uint64_t wait_ns = ctx->batch_wait_ns ? ctx->batch_wait_ns : sm103::kWaitNs;
  {
    Launch L(ctx, "batch_kernel", s);
    if (jmax >= 3)
      batch_kernel<3><<<grid, 256, smem, s>>>(table, starts, (int)nph, done, bs, total_units, tile_bytes,
                                              wait_ns, ctx->d_status);
    else
      batch_kernel<2><<<grid, 256, smem, s>>>(table, starts, (int)nph, done, bs, total_units, tile_bytes,
                                              wait_ns, ctx->d_status);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "batch kernel launch");
}

lre_status batch_tune(lre_ctx *ctx, const lre_instance *inst, int count, cudaStream_t s, float *best_ms) {
  lre_status st = validate(inst, count);
  if (st != LRE_OK) return st;
  const int cand_j[2] = {2, 3};
  const int cand_occ[2] = {1, 2};       // resident CTAs per SM (the kernel fits at most two)
  const int cand_first[2] = {256, 1024};  // items per unit of the count-reading first passes
  const int cand_unit[3] = {256, 1024, 4096};  // items per unit of the other fold and assembly passes
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return LRE_ERR_CUDA;
  }
  float best = 1e30f;
  int bj = ctx->batch_jmax, bo = ctx->batch_ctas_per_sm, bf = ctx->batch_first_unit, bu = ctx->batch_unit;
  for (int j : cand_j) {
    for (int o : cand_occ) {
      for (int cand = 0; cand < 6; ++cand) {
        const int f = cand_first[cand & 1], u = cand_unit[cand >> 1];
        ctx->batch_jmax = j;
        ctx->batch_ctas_per_sm = o;
        ctx->batch_first_unit = f;
        ctx->batch_unit = u;
        if ((st = batch_run(ctx, inst, count, s)) != LRE_OK) break;  // warm-up
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < 3 && st == LRE_OK; ++rep) st = batch_run(ctx, inst, count, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = LRE_ERR_CUDA;
        if (st != LRE_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.f;
        if (ms < best) {
          best = ms;
          bj = j;
          bo = o;
          bf = f;
          bu = u;
        }
      }
      if (st != LRE_OK) break;
    }
    if (st != LRE_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->batch_jmax = bj;
  ctx->batch_ctas_per_sm = bo;
  ctx->batch_first_unit = bf;
  ctx->batch_unit = bu;
  if (best_ms) *best_ms = best;
  return st;
}

}  // namespace lre

// Test hook (host only, no device work): the pass table lre_batch_run would
// build for these descriptors and this schedule.  Per phase, 8 int64 at
// out + 8 k: instance, code, dep, dep_units, per_unit, unit_begin, units,
// items (at most max_phases phases written).  Returns the number of phases,
// or -1 when the descriptors are rejected.
extern "C" int lre_debug_batch_plan(const lre_instance *descs, int count, int jmax, int first_unit, int unit,
                                    int64_t *out, int max_phases) {
  if (lre::validate(descs, count) != LRE_OK || jmax < 1 || first_unit < 256 || unit < 256) return -1;
  const lre::Plan plan = lre::build_plan(descs, count, jmax, first_unit, unit, nullptr);
  const int nph = (int)plan.phases.size();
  for (int k = 0; out && k < nph && k < max_phases; ++k) {
    const lre::BPhase &b = plan.phases[k];
    const int64_t v[8] = {b.inst, b.code, b.dep, (int64_t)b.dep_units, b.per_unit, b.unit_begin, b.units, b.items};
    for (int f = 0; f < 8; ++f) out[8 * k + f] = v[f];
  }
  return nph;
}

// Test hook (not part of include/lre.h): failure injection for the batched
// kernel's bounded waits.  wait_ms > 0 bounds every dependency wait of later
// lre_batch_run calls by that many milliseconds (0 restores the default 2 s);
// stall_phase >= 0 makes the first dependent phase of the pass table at or
// after that index wait for one unit more than its dependency has, so its
// units never become ready and their waits run out (LRE_ERR_TIMEOUT, every
// CTA leaves); -1 turns that off.  Host-side table data only: no kernel is
// changed.
extern "C" lre_status lre_debug_batch_fault(lre_ctx *ctx, int wait_ms, int stall_phase) {
  if (!ctx || wait_ms < 0 || stall_phase < -1) return LRE_ERR_INVALID_ARG;
  ctx->batch_wait_ns = (uint64_t)wait_ms * 1000000ull;
  ctx->batch_stall_phase = stall_phase;
  return LRE_OK;
}
