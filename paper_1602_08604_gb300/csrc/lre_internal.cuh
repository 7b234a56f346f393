// Internal declarations shared by the translation units of liblre.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lre.h"

struct cusolverDnContext;
struct cublasContext;

struct lre_prof_entry {
  const char *name;
  cudaEvent_t start, stop;
};

// One batched plan kept on the device (lre_batch_run), keyed by the
// instance descriptors and the schedule: the pass table's device copy, the
// workspace it points into, and what a launch over it needs.  Entries are
// immutable, so a CUDA graph that captured a launch over one stays valid.
struct lre_batch_entry {
  std::vector<char> key;      // descriptors + schedule
  void *table = nullptr;      // device: phases, then their first units
  void *ws = nullptr;
  size_t nph = 0, head = 0, ws_bytes = 0;
  int64_t total_units = 0;
  int tile_bytes = 0;
};

struct lre_ctx {
  int device = 0;
  int num_sms = 0;
  size_t ws_limit = 0;        // 0 = unlimited
  void *ws = nullptr;         // device workspace
  size_t ws_bytes = 0;
  int *d_status = nullptr;    // device-side latched error code (0 = none)
  cusolverDnContext *solver = nullptr;
  cublasContext *blas = nullptr;
  std::string last_error;
  bool prof = false;                      // record CUDA events around each launch
  std::vector<lre_prof_entry> prof_pool;  // reused events
  size_t prof_used = 0;
  uint64_t launches = 0;                  // kernels of this library launched so far
  // first fold pass: 0 register kernel, 1 TMA pipeline (default), 2 fused
  // with the second pass through L2 (the ALU pipeline, or the tensor-core
  // pass where that runs)
  int first_variant = 1;
  int fused_consumers = 0;    // tensor-core fused pass: CTAs on the second pass (0: a sixth of the SMs)
  int fused_discard = 0;      // tensor-core fused pass: 1 = drop consumed ring lines from L2
  int first_grid = 0;         // tensor-core first pass: CTAs (0: one per SM)
  int first7 = 0;             // tensor-core raw first pass: 1 = fold seven qubits where it applies
  int fold_path = 1;          // first pass: 0 FWHT on the ALU, 1 tensor cores for int16 counts, 2 also int32
  void *mma_operand = nullptr;  // device copy of the constant tensor-core operand
  int mma_biased = 0;         // tensor-core operand: 0 raw counts as fp16 bits, 1 fp16(1024 + c)
  int project_mode = 1;       // step (iii): 1 eigenvalue-first where it applies, 0 full eigendecomposition
  int generic_tma = 1;        // later fold passes: 1 TMA-staged kernel where it applies, 0 register loads
  int batch_jmax = 3;         // batched schedule: qubits per fold pass
  int batch_ctas_per_sm = 2;  // batched schedule: resident CTAs per SM
  int batch_first_unit = 1024;  // batched schedule: items per unit of the count-reading first passes
  int batch_unit = 256;         // batched schedule: items per unit of the other fold and assembly passes
  int batch_occupancy[2] = {0, 0};  // most resident CTAs per SM of batch_kernel<2>, <3>
  std::vector<lre_batch_entry> batch_cache;  // device pass tables of earlier batched calls
  uint64_t batch_wait_ns = 0;   // batched kernel: bound of a dependency wait (0 = the default 2 s)
  int batch_stall_phase = -1;   // test hook: the first dependent phase at or after it never becomes ready
  size_t host_chunk_bytes = 256ull << 20; // host-input streaming: bytes of input per chunk
  int records_direct = 0;                 // host shot records: 1 = always the records-fed first pass
  cudaStream_t copy_stream = nullptr;     // host-input streaming (lre_estimate_host)
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_free[2] = {nullptr, nullptr};
  cudaEvent_t ev_theta = nullptr;         // theta final: its copy-back may start
  // streamed estimate (lre_stream_*): the instance, and the bases whose first
  // fold pass is done (a prefix of whole tile rows)
  int stream_active = 0;
  int stream_n = 0;
  lre_count_kind stream_kind = LRE_COUNTS_I16;
  int64_t stream_shots = 0, stream_rows_done = 0;
  void *stream_ws = nullptr;  // the workspace the streamed state lives in
  int canaries = 0;           // test hook: a patterned guard after the workspace
};
constexpr size_t kCanaryBytes = 1 << 16;
constexpr unsigned char kCanaryByte = 0xA5;

namespace lre {

// Status codes written by kernels into ctx->d_status (first writer wins).
__device__ __forceinline__ void latch(int *status, int code) { atomicCAS(status, 0, code); }

// Ensure ctx->ws holds at least `bytes` (respecting the cap).
lre_status ensure_workspace(lre_ctx *ctx, size_t bytes);
lre_status cuda_fail(lre_ctx *ctx, cudaError_t e, const char *where);

// Brackets one launch (or one library call when own == false): counts our
// own kernel launches and, when profiling is on, records a pair of events on
// the launch stream.
class Launch {
 public:
  Launch(lre_ctx *ctx, const char *name, cudaStream_t s, int own = 1);
  ~Launch();

 private:
  lre_ctx *ctx_;
  cudaStream_t s_;
  long idx_ = -1;  // index into ctx->prof_pool (the pool may grow)
};

inline int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}

// ---- step (i): counts -> S (int64) or theta (FP64) --------------------------
struct FoldArgs {
  const void *counts;
  lre_count_kind kind;
  int n;
  const int64_t *shots;   // per-basis (device) or nullptr
  int64_t shots_uniform;  // used when shots == nullptr
  double *theta;          // final FP64 output (estimate mode) or nullptr
  int64_t *S;             // final int64 output (parity-sum mode) or nullptr
  int64_t *T = nullptr;   // optional exact integers S_i 3^(n-k_i) (uniform shots)
  // Split execution for streamed input: stage 0 runs every pass; stage 1 only
  // the six-qubit first pass over basis rows [ah_begin, ah_end) * 729; stage 2
  // every pass after it (the first pass's output already in the workspace).
  int stage = 0;
  int64_t ah_begin = 0, ah_end = -1;
  // stage 1 only: counts from shot records grouped by tile (tile_bucket_run
  // over tile rows ah_begin..ah_end) instead of dense counts
  const uint16_t *rec_entries = nullptr;
  const int32_t *rec_offs = nullptr;
  // stage 1 only: `counts` holds rows [row_base, row_base + rows_in) of the
  // count matrix (rows_in = 0: all 3^n rows from row 0)
  int64_t row_base = 0, rows_in = 0;
};
size_t fold_workspace_bytes(int n, lre_count_kind kind, bool weighted, int64_t shots_bound,
                            int variant = 2);
lre_status fold_run(lre_ctx *ctx, const FoldArgs &a, void *ws, size_t ws_bytes, cudaStream_t s);
// Basis rows per unit of the stage-1 split (729), or 0 when these arguments
// cannot be split (no six-qubit first pass, or one without tile ranges).
int64_t fold_split_rows(lre_ctx *ctx, const FoldArgs &a);
// True when the first pass for these arguments is the tensor-core one (the
// one that can take its counts from bucketed shot records).
bool fold_first_is_tensor(lre_ctx *ctx, const FoldArgs &a);

// Tiled TMA descriptor of an int32 tensor (dims and box innermost first,
// strides in bytes of dims 1..rank-1); false if the driver rejects it.
bool encode_tensor_map_i32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                           const uint64_t *strides, const uint32_t *box);
bool encode_tensor_map(CUtensorMap *map, CUtensorMapDataType type, const void *base, int rank,
                       const uint64_t *dims, const uint64_t *strides, const uint32_t *box);

// ---- step (ii): theta -> rho -------------------------------------------------
size_t assemble_workspace_bytes(int n);
lre_status assemble_run(lre_ctx *ctx, const double *theta, int n, lre_c64 *rho, void *ws,
                        cudaStream_t s);
// Load the kernels of assemble_run into the current device (see assemble.cu).
lre_status assemble_preload();
// Text of the last failure of lre_assemble_noalloc on the calling thread.
const char *noalloc_last_error();
// Exact-integer variant for uniform shots: T_i = S_i 3^(n-k_i) (= t_i N 3^n).
lre_status assemble_int_run(lre_ctx *ctx, const int64_t *T, int n, int64_t shots, lre_c64 *rho,
                            void *ws, cudaStream_t s);
struct LastScaleArgs {
  float sh, sl;  // 1/(2^n N 3^n) = sh + sl
};
LastScaleArgs int_assembly_scale(int n, int64_t shots);

// ---- step (iii): rho -> physical rho ----------------------------------------
lre_status project_run(lre_ctx *ctx, const lre_c64 *rho_in, int n, lre_c64 *rho_out,
                       double *eig_mu, double *eig_rho, cudaStream_t s);

// tridiagonal eigenproblem kernels (tridiag.cu)
constexpr int TRI_THREADS = 256;
__global__ void tri_bisect_kernel(const double *a, const double *b2, int64_t n, double lo0, double hi0, double tol,
                                  double pivmin, double *W, int64_t j0, int64_t cnt);
__global__ void tri_multisect_kernel(const double *a, const double *b2, int64_t n, double lo0, double hi0,
                                     double tol, double pivmin, double *W, int64_t j0, int64_t cnt);
// Gershgorin bounds of T (stats[0], stats[1]), the largest squared
// off-diagonal (stats[2]) and the squares b2 (one CTA of 256 threads).
__global__ void tri_prepare(const double *a, const double *b, int64_t n, double *b2, double *stats);

// Smolin threshold: eigenvalues kept and the shift added to each.
struct SmolinResult {
  int64_t kept;
  double shift;
};
// The projected matrix from m unit vectors Z (column-major d x m, the
// eigenvectors of conj(mu)) and their eigenvalues w, in the kept form
// sum (w + s) z z^dag or the dropped form mu + s I + sum -(w + s) z z^dag
// (C holding conj(mu) column-major on entry), written to rho_out as
// row-major complex64.  Z is scaled in place; C is the working matrix.
lre_status rebuild_emit(lre_ctx *ctx, struct cublasContext *blas, double2 *C, double2 *Z, const double *w,
                        int64_t d, int64_t m, bool kept_form, const SmolinResult *res, lre_c64 *rho_out,
                        cudaStream_t s);
// The Krylov projection (krylov.cu): *fallback = true, with nothing written to
// the outputs, when it cannot decide or certify the threshold; eig_rho
// (device, or NULL) is filled only in the kept form (*fallback otherwise).
lre_status project_krylov(lre_ctx *ctx, struct cublasContext *blas, const lre_c64 *rho_in, int64_t d,
                          lre_c64 *rho_out, double *eig_rho, cudaStream_t s, bool *fallback);
constexpr int TRI_ROUNDS = 3;  // inverse-iteration rounds
__global__ void tri_factor(const double *a, const double *b, int64_t n, const double *lam, int m, double tnorm,
                           double *lu);
__global__ void tri_solve(const double *lu, int64_t n, int m, double *X, int first);
__global__ void tri_orthonormalise(double *X, int64_t n, const int *cl);
__global__ void tri_clusters(const double *lam, int m, double gap_tol, int *cl, int *k_out);

// ---- end to end from host memory ---------------------------------------------
lre_status estimate_host_run(lre_ctx *ctx, const void *host_in, int host_kind, int64_t shots,
                             int n, double *theta_host, lre_c64 *rho_host, cudaStream_t s);

// ---- tensor-core first pass (fold_mma.cu) ----------------------------------------
size_t mma_operand_bytes();
// TMA box rows of the count maps: which 0 the main box (216 rows; SPLIT 108),
// 1 the tail (81 rows)
uint32_t mma_box_rows(int which, int variant);
// largest count the operand encoding keeps exact: variant 0 raw int16 (2047),
// 1 biased int16 (1023), 3 int32 in two planes (16383), MMA_SEVEN raw int16
int64_t mma_max_count(int variant);
// variant of mma_first_pass that folds seven qubits (the raw encoding)
constexpr int MMA_SEVEN = 5;
lre_status mma_operand_upload(lre_ctx *ctx, void *a_dev, cudaStream_t s);
// the raw tensor-core pass fused with the second fold pass through an L2 ring
lre_status mma_first_pass_fused9(lre_ctx *ctx, const CUtensorMap &map_big, const CUtensorMap &map_tail,
                                 const void *a_dev, int32_t *out, int32_t *scratch, unsigned *f9, int n,
                                 int64_t shots, int consumers, bool discard, cudaStream_t s);
size_t mma_fused9_scratch_bytes();
size_t mma_fused9_counter_bytes();
// records grouped by count tile (records.cu) and the first pass over them
lre_status tile_bucket_run(lre_ctx *ctx, const uint16_t *records, int64_t tile_rows, int64_t shots, int n,
                           uint16_t *entries, int32_t *offs, cudaStream_t s);
lre_status mma_first_pass_records(lre_ctx *ctx, const void *a_dev, const uint16_t *entries, const int32_t *offs,
                                  int64_t shots, int32_t *out, int8_t *out_hi, int n, int64_t tile_begin,
                                  int64_t tile_end, cudaStream_t s);
lre_status mma_first_pass(lre_ctx *ctx, const CUtensorMap &map_big, const CUtensorMap &map_tail, const void *a_dev,
                          int32_t *out, int8_t *out_hi, int n, int variant, int64_t shots, int64_t tile_begin,
                          int64_t tile_end, int64_t row_base, cudaStream_t s);
// Streamed first pass (lre_stream_*): the layout of the first pass's output
// for these arguments -- split planes or int32, elements in all -- and
// whether the arguments can be streamed at all (a six-qubit first pass that
// takes tile ranges).
bool fold_stage1_layout(lre_ctx *ctx, const FoldArgs &a, bool *planes, int64_t *elems);

// ---- batched instances (one persistent launch) ---------------------------------
lre_status batch_run(lre_ctx *ctx, const lre_instance *inst, int count, cudaStream_t s);
lre_status batch_tune(lre_ctx *ctx, const lre_instance *inst, int count, cudaStream_t s, float *best_ms);

// ---- ingest ------------------------------------------------------------------
lre_status histogram_run(lre_ctx *ctx, const uint16_t *records, int64_t num_bases,
                         int64_t shots_per_basis, int n, void *counts, lre_count_kind kind,
                         cudaStream_t s);

}  // namespace lre
