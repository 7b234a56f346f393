/*
 * lre.h -- C ABI of the GB300 linear-regression-estimation (LRE) hot path for
 * full quantum state tomography under Pauli measurements
 * (arXiv:1602.08604, "Full reconstruction of a 14-qubit state within four
 * hours").
 *
 * The three steps of the paper (Sec. II):
 *   step (i)   measured frequencies of the 6^n Pauli eigenprojectors ->
 *              least-squares coefficient vector theta (Eq. 3, Sec. III);
 *   step (ii)  theta -> Hermitian unit-trace mu = sum_i theta_i Omega_i
 *              (Eq. 4);
 *   step (iii) mu -> the closest physical density matrix (Sec. II, the
 *              Smolin-Gambetta-Smith algorithm).
 *
 * Conventions (every index has qubit 1 as its most significant digit):
 *   basis   b = sum_q a_q 3^(n-q),  a_q in {0:X, 1:Y, 2:Z}      (3^n bases)
 *   outcome o = sum_q o_q 2^(n-q),  o_q = 0: the +1 eigenvector (2^n outcomes)
 *   Pauli   i = sum_q p_q 4^(n-q),  p_q in {0:I, 1:X, 2:Y, 3:Z} (Eq. 5 order)
 *   counts  [3^n][2^n] row-major (int32 or int16), counts[b][o] = number of
 *           shots of basis b that gave outcome o.
 *   theta   FP64 [4^n] in Eq. (5) order, holding the Pauli expectation
 *           estimates t_i = 2^{n/2} theta_i^{LS}; theta[0] = 1 exactly.
 *           (The paper's orthonormal-basis coefficient is 2^{-n/2} t_i.)
 *   rho     complex64 [2^n][2^n] row-major, rho = (1/2^n) sum_i t_i P_i.
 *
 * Memory: every pointer argument named "device" must be CUDA device memory
 * on the context's device; the caller owns it, the library only borrows it
 * for the call.  The context owns its workspace (device memory grown on
 * demand, capped by lre_set_workspace_limit) and its library handles.
 *
 * Asynchrony: compute calls enqueue work on `stream` and return.  Argument
 * errors are returned synchronously and nothing is enqueued.  Errors found
 * by kernels (a count total that disagrees with the stated shots, a shot
 * record outside [0, 2^n)) are latched in the context and returned by
 * lre_sync().  No C++ exception crosses this ABI.
 *
 * Supported sizes: 1 <= n <= 14 for every call (n <= 12 for lre_project on
 * hosts without enough device memory for three d x d complex128 matrices).
 */
#ifndef LRE_H
#define LRE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRE_OK = 0,
  LRE_ERR_INVALID_ARG = 1,    /* bad pointer, size, kind or shot count        */
  LRE_ERR_UNSUPPORTED = 2,    /* n outside the supported range                */
  LRE_ERR_SHOTS_MISMATCH = 3, /* counts do not add up to the stated shots     */
  LRE_ERR_OOM = 4,            /* workspace above the limit or cudaMalloc fail */
  LRE_ERR_CUDA = 5,           /* a CUDA runtime / library call failed         */
  LRE_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up           */
  LRE_ERR_EIG_FAILED = 7      /* the Hermitian eigensolver reported failure   */
} lre_status;

/* Layout of the per-basis measurement results (Sec. III: the results of the
 * 6^n operators are stored per basis group, 3^n groups of 2^n outcomes). */
typedef enum {
  LRE_COUNTS_I32 = 0, /* int32 counts [3^n][2^n]                                  */
  LRE_COUNTS_I16 = 1, /* int16 counts [3^n][2^n] (each count <= 32767)            */
  LRE_SHOTS_U16 = 2   /* uint16 shot records [3^n][N]: outcome index of each shot
                         (lre_estimate with uniform shots N only)                 */
} lre_count_kind;

typedef enum {
  LRE_HOST_COUNTS_I32 = 0,  /* host int32 counts [3^n][2^n]                        */
  LRE_HOST_COUNTS_I16 = 1,  /* host int16 counts [3^n][2^n]                        */
  LRE_HOST_RECORDS_U16 = 2  /* host uint16 shot records [3^n][shots]: outcome index */
} lre_host_kind;

typedef struct {
  float re, im;
} lre_c64;

typedef struct CUstream_st *lre_stream; /* the same handle as cudaStream_t   */

/* One instance of a batched run (lre_batch_run). */
typedef struct {
  const void *counts; /* device [3^n][2^n] counts of `kind`                     */
  int32_t kind;       /* lre_count_kind                                          */
  int32_t n;          /* qubits, 1 <= n <= 9                                     */
  int64_t shots;      /* shots per basis (> 0), the same for every basis         */
  double *theta;      /* device FP64 [4^n] output                                */
  lre_c64 *rho;       /* device complex64 [2^n][2^n] output, or NULL             */
} lre_instance;
typedef struct lre_ctx lre_ctx;

/* Create a context on CUDA device `device` (creates its cuSOLVER/cuBLAS
 * handles lazily).  *out receives the context. */
lre_status lre_create(lre_ctx **out, int device);

/* Free the context, its workspace and handles.  NULL is allowed. */
void lre_destroy(lre_ctx *ctx);

/* Cap the workspace the context may hold (bytes; 0 = no cap).  A call whose
 * plan needs more returns LRE_ERR_OOM without enqueuing anything. */
lre_status lre_set_workspace_limit(lre_ctx *ctx, size_t bytes);

/* Workspace bytes lre_estimate needs for this n and count kind, rho
 * included (per_basis_shots != 0 for the per-basis FP64 weighting; for
 * LRE_SHOTS_U16 the dense int16 counts the records are histogrammed into,
 * i.e. at most 32767 shots per basis). */
lre_status lre_workspace_size(lre_ctx *ctx, int n, lre_count_kind kind, int per_basis_shots,
                              size_t *bytes);

/* Step (i) without the weight: exact integer parity sums
 *   S[i] = sum over bases b compatible with Pauli string i of
 *          sum_o counts[b][o] * (-1)^{popcount(o & support(i))},
 * where b is compatible with i when i's non-identity letters equal b's axes
 * (Sec. III: the 2^n nonzeros of each Gamma^(j) and the shared 2^n x 2^n
 * nonzero matrix of each basis group).  counts: device [3^n][2^n];
 * row_total_bound: an upper bound on every row's sum of counts (the shots
 * per basis), or 0 if unknown (then all partial sums are int64); S: device
 * int64 [4^n], overwritten.  Bit-exact whenever the bound holds. */
lre_status lre_parity_sums(lre_ctx *ctx, const void *counts, lre_count_kind kind, int n,
                           int64_t row_total_bound, int64_t *S, lre_stream stream);

/* Steps (i)+(ii): Eq. (3) with the diagonal X^T X of Sec. III, i.e.
 *   theta[i] = S[i] / (N * 3^k(i))           (uniform shots N)
 *   theta[i] = (sum_b Shat_b[i] / N_b) / 3^k (per-basis shots N_b)
 * with k(i) the number of identity letters of i, then, when rho != NULL,
 * Eq. (4): rho = (1/2^n) sum_i theta[i] P_i.
 * counts: device [3^n][2^n] counts (LRE_COUNTS_*), or device uint16 shot
 * records [3^n][shots_uniform] (LRE_SHOTS_U16, which the call histograms into
 * dense counts in its workspace; a record >= 2^n latches
 * LRE_ERR_INVALID_ARG); shots: device int64 [3^n] per-basis totals (counts
 * only), or NULL to use shots_uniform (> 0) for every basis; theta: device
 * FP64 [4^n]; rho: device complex64 [2^n][2^n] or NULL.  With uniform shots
 * theta is the correctly rounded quotient of two exact integers.  When the
 * counts' grand total differs from shots_uniform * 3^n,
 * LRE_ERR_SHOTS_MISMATCH is latched (returned by lre_sync).  Every count must
 * lie in [0, shots_uniform]: the tensor-core first pass (lre_set_fold_path)
 * reads counts in a form where a larger value would change the result, so it
 * checks every count it reads and latches LRE_ERR_SHOTS_MISMATCH for one
 * outside that range (theta is then not defined); it also relies on every
 * basis row summing to shots_uniform for the width of the partial sums it
 * keeps, checks each partial against it, and latches the same error for a
 * row whose partials exceed it.  The FWHT path computes the exact sums of
 * whatever counts it is given. */
lre_status lre_estimate(lre_ctx *ctx, const void *counts, lre_count_kind kind, const int64_t *shots,
                        int64_t shots_uniform, int n, double *theta, lre_c64 *rho,
                        lre_stream stream);

/* Step (i) for one instance split over several GPUs by the axis of qubit 1
 * (the basis groups of Sec. III partitioned by their first letter).
 * slab: device [3^(n-1)][2^n] counts of the bases whose qubit-1 axis is one
 * fixed a (rows a 3^(n-1) .. (a+1) 3^(n-1) - 1 of the full count matrix);
 * row_total_bound as in lre_parity_sums.  ident: device int64 [4^(n-1)],
 * the slab's share of the parity sums of the strings whose qubit-1 letter is
 * I (the three slabs' shares add up to S[0 .. 4^(n-1))); own: device int64
 * [4^(n-1)], the parity sums of the strings whose qubit-1 letter is a + 1,
 * S[(a+1) 4^(n-1) + j], to which no other slab contributes.  Indices over
 * qubits 2..n in Eq. (5) order.  2 <= n <= 14; exact integers whenever the
 * bound holds.  The shares of ident are summed across GPUs by the caller
 * (one reduce-scatter); lre_weight turns sums into theta. */
lre_status lre_slab_sums(lre_ctx *ctx, const void *slab, lre_count_kind kind, int n, int64_t row_total_bound,
                         int64_t *ident, int64_t *own, lre_stream stream);

/* The weight of Eq. (3) with the diagonal X^T X of Sec. III on a block of
 * exact parity sums: theta[j] = S[j] / (N 3^k), k the number of identity
 * letters of the n-qubit Pauli index first + j, correctly rounded (the
 * quotient lre_estimate computes).  S: device int64 [count]; theta: device
 * FP64 [count]; shots N > 0 with N 3^n < 2^53; first + count <= 4^n. */
lre_status lre_weight(lre_ctx *ctx, const int64_t *S, int n, int64_t first, int64_t count, int64_t shots,
                      double *theta, lre_stream stream);

/* Steps (i)+(ii) with 4^n measurement operators instead of 6^n (Sec. VI,
 * which states the cost drop to O(8^n) but names no operator set; read as
 * the minimal informationally complete subset of the Pauli eigenprojectors,
 * |0>, |1>, |+>, |+i> per qubit).  Their frequencies come from the same Pauli
 * counts -- |0>, |1> from the Z basis, |+> and |+i> from outcome 0 of the X
 * and Y bases -- so counts, kind and shots_uniform are as for lre_estimate
 * (uniform shots N; N 3^n < 2^53).  Eq. (3) with these 4^n rows (X square
 * and invertible, X^T X = G^{(x)n} not diagonal) is exact: per qubit
 * <I> = p_0 + p_1, <X> = 2p_+ - p_0 - p_1, <Y> = 2p_+i - p_0 - p_1,
 * <Z> = p_0 - p_1; theta (same units and order as lre_estimate) is one
 * correctly rounded division of exact integer sums by N.  rho (or NULL) as
 * lre_assemble.  Only the 4^n used counts are read. */
lre_status lre_estimate_ic4(lre_ctx *ctx, const void *counts, lre_count_kind kind, int64_t shots_uniform, int n,
                            double *theta, lre_c64 *rho, lre_stream stream);

/* Step (ii) alone, Eq. (4): rho = (1/2^n) sum_i theta[i] P_i, computed in
 * FP64 and rounded once to complex64.  theta: device FP64 [4^n];
 * rho: device complex64 [2^n][2^n]. */
lre_status lre_assemble(lre_ctx *ctx, const double *theta, int n, lre_c64 *rho, lre_stream stream);

/* Step (ii) for callers that cannot allocate device memory (the paper has
 * no counterpart: this is a deployment variant of lre_assemble).  Same
 * arguments, result and FP64 arithmetic as lre_assemble, but no context and
 * no allocation: the FP64 scratch of the butterfly passes is a fixed 32 MiB
 * array in the library's device image, which every GPU that loads the
 * library holds until the process exits.  Runs on the calling thread's
 * current device, on `stream`.  1 <= n <= 10; a larger n returns
 * LRE_ERR_UNSUPPORTED (the scratch would not fit) and enqueues nothing.
 * CUDA loads device code and variables lazily, so the first call on a device
 * sets it up: it loads the array and the assembly kernels (about 32 MiB of
 * device memory must be free then) and looks up the array's device address.
 * Make that first call at start-up, before your allocator reserves the
 * device and before any stream capture; later calls allocate nothing.  All
 * calls share the array: calls that overlap on the GPU race on it and must
 * be serialised by the caller.  No part of the array needs to start at
 * zero.  On failure, lre_last_error(NULL) gives the reason (per thread). */
lre_status lre_assemble_noalloc(const double *theta, int n, lre_c64 *rho, lre_stream stream);

/* Step (iii): rho_out = argmin over density matrices sigma of
 * ||sigma - rho_in||_F (Sec. II, Smolin et al.): the eigenpairs of rho_in
 * on the needed side of the threshold (Lanczos in double-float arithmetic
 * with FP64 scalars, certified; else an FP64
 * Hermitian eigendecomposition of rho_in promoted to complex128), the
 * eigenvalue correction onto the probability simplex, and the
 * reconstruction in FP64 rounded once to complex64.  rho_in, rho_out: device complex64
 * [2^n][2^n] (may alias); eig_mu, eig_rho: device FP64 [2^n] or NULL,
 * receiving the spectra of rho_in and rho_out in decreasing order.  The call
 * synchronises `stream` once (to size the reconstruction). */
lre_status lre_project(lre_ctx *ctx, const lre_c64 *rho_in, int n, lre_c64 *rho_out,
                       double *eig_mu, double *eig_rho, lre_stream stream);

/* Count ingest from shot records (Sec. III: the measured results are stored
 * per basis group): counts[b][o] = #{s : records[b][s] == o}.
 * records: device uint16 [num_bases][shots_per_basis]; counts: device
 * [num_bases][2^n] of `kind`, overwritten.  A record >= 2^n latches
 * LRE_ERR_INVALID_ARG. */
lre_status lre_histogram(lre_ctx *ctx, const uint16_t *records, int64_t num_bases,
                         int64_t shots_per_basis, int n, void *counts, lre_count_kind kind,
                         lre_stream stream);

/* Steps (i)+(ii) end to end from HOST memory (Sec. II steps (i) and (ii) on
 * the per-basis results of Sec. III, as lre_estimate).  host_in: pinned host buffer
 * of `host_kind` (dense counts, or shot records that the ingest kernel
 * histograms on the device); shots_uniform: shots per basis (> 0);
 * theta_host: host FP64 [4^n]; rho_host: host complex64 [2^n][2^n] or NULL.
 * The input is copied in row chunks on a copy stream owned by the context,
 * each copy overlapped with the device work on the chunk before it: the
 * ingest and, for n >= 7, the six-qubit first fold pass over the chunk's
 * whole tile rows (729 bases).  The other passes run after the last chunk;
 * theta is copied back on the copy stream while rho is assembled on
 * `stream`.  The call returns when theta (and rho) are in host memory, with
 * any latched kernel error.  Device memory used: the counts (3^n 2^n x 2 or
 * 4 bytes), theta, rho and the fold workspace, all held in the context's
 * workspace.  When a workspace limit (lre_set_workspace_limit) leaves no
 * room for the dense counts, shot records with at most 2047 shots per basis
 * (a multiple of 8) take a path without them: each chunk's records are
 * grouped by count tile on the device and the tensor-core first pass builds
 * its count tiles from them in shared memory (slower on states whose shots
 * concentrate on few outcomes; same results). */
lre_status lre_estimate_host(lre_ctx *ctx, const void *host_in, lre_host_kind host_kind,
                             int64_t shots_uniform, int n, double *theta_host, lre_c64 *rho_host,
                             lre_stream stream);

/* Steps (i)+(ii) for many independent instances in ONE persistent kernel
 * launch (the paper treats one state at a time; batching is for many small
 * reconstructions).  Each instance gets exactly the result of lre_estimate
 * with uniform shots (bit-identical theta; rho from the same exact-integer
 * assembly).  descs: host array of `count` instance descriptors (copied
 * during the call; the buffers they point to are device memory).  The pass
 * lists of all instances are cut into 256-item work units that the CTAs of
 * one grid claim in pass-major order; a unit waits (bounded by time, then
 * LRE_ERR_TIMEOUT is latched) for its instance's previous pass.  n > 9 in
 * any instance returns LRE_ERR_UNSUPPORTED (use lre_estimate).
 * CUDA graphs: the call may be captured (cudaStreamBeginCapture or any
 * wrapper of it) once the same batch -- the same descriptors -- has run
 * uncaptured on this context; that run sizes the workspace and stores the
 * batch's pass table in a device buffer the context keeps until
 * lre_destroy, and the captured launch reuses both (a capture without such a
 * run returns LRE_ERR_UNSUPPORTED and enqueues nothing).  A replay reads the
 * buffers the descriptors point to at replay time, and uses the context's
 * workspace: replays and other calls on the same context must not overlap,
 * and a later call that grows the workspace invalidates earlier graphs. */
lre_status lre_batch_run(lre_ctx *ctx, const lre_instance *descs, int count, lre_stream stream);

/* Autotuner for lre_batch_run: times the candidate schedules (qubits per
 * fold pass 2 or 3; 1 or 2 resident CTAs per SM; 256 or 1024 items per work
 * unit of the count-reading first passes; 256, 1024 or 4096 items per work
 * unit of the other fold and assembly passes) on this batch, keeps the
 * fastest in the context for later lre_batch_run calls, and returns its time
 * per launch in *best_ms (may be NULL).  Synchronises `stream`. */
lre_status lre_batch_tune(lre_ctx *ctx, const lre_instance *descs, int count, lre_stream stream,
                          float *best_ms);

/* The batched schedule this context uses (set by lre_batch_tune, or the
 * defaults): qubits per fold pass (jmax), resident CTAs per SM, items per
 * work unit of the count-reading first passes and of the other passes.  Any
 * output pointer may be NULL.  Host only; LRE_ERR_INVALID_ARG for ctx NULL. */
lre_status lre_batch_schedule(const lre_ctx *ctx, int *jmax, int *ctas_per_sm, int *first_unit, int *unit);

/* First fold pass of step (i) (the first six qubits) on later calls of this
 * context:
 * LRE_FOLD_TENSOR (default): the level-A contraction of each 729 x 64 count
 *   tile is a GEMM on the 5th-generation tensor cores (tcgen05.mma kind::f16,
 *   FP32 accumulation in TMEM) against the constant +-1/0 matrix of the
 *   per-qubit map of Sec. III / Eq. 3: the int16 count c is read unchanged as
 *   the fp16 bit pattern of c * 2^-24, exact for c < 2048, and every partial
 *   sum stays below 2^24 units, so the result is bit-identical to the FWHT
 *   path.  It applies to int16 counts whose per-basis shot number (hence
 *   every count) is at most 2047, with uniform shots; every other call runs
 *   the FWHT path.  Every count is checked (see lre_estimate).
 * LRE_FOLD_TENSOR_SPLIT: as LRE_FOLD_TENSOR, and int32 counts with at most
 *   16383 shots per basis on the tensor cores too, each count split into two
 *   fp16 planes (c mod 2048 and (c >> 11) 2^11) contracted in one MMA chain;
 *   bit-identical, but slower than the FWHT path on GB300 (the in-place
 *   conversion holds each shared-memory slot longer), hence not the default.
 * LRE_FOLD_FWHT: the parity transform (Walsh-Hadamard butterflies) and the
 *   ternary fold on the integer ALUs, for every input. */
#define LRE_FOLD_FWHT 0
#define LRE_FOLD_TENSOR 1
#define LRE_FOLD_TENSOR_SPLIT 2
lre_status lre_set_fold_path(lre_ctx *ctx, int path);

/* Steps (i)+(ii) on counts that arrive in chunks (Sec. III's per-group
 * results produced or received over time), so the whole [3^n][2^n] matrix
 * never has to exist on the device: each chunk of whole tile rows (729
 * consecutive bases) goes through the six-qubit first fold pass at once and
 * only its partial sums are kept; lre_stream_end runs the other passes and
 * the assembly.  Results are bit-identical to lre_estimate with uniform shots
 * on the whole matrix.  7 <= n <= 14.
 * lre_stream_begin: start an instance (kind int16/int32, shots per basis N);
 *   sizes the workspace (first-pass partials, later passes, T).
 * lre_stream_chunk: counts device [num_bases][2^n] of `kind`, 16-byte
 *   aligned, holding bases first_basis .. first_basis + num_bases - 1;
 *   chunks come in order (first_basis = the bases done so far), both numbers
 *   multiples of 729.  The chunk may be reused as soon as the stream has
 *   passed this call's work.
 * lre_stream_end: once all 3^n bases are in; theta device FP64 [4^n], rho
 *   device complex64 [2^n][2^n] or NULL, as lre_estimate (including the
 *   latched LRE_ERR_SHOTS_MISMATCH on a wrong grand total).
 * lre_stream_checkpoint: copy the state (a header and the partial sums of the
 *   bases done, 3 or 4 bytes per partial) into host memory: *needed receives
 *   its size; host NULL only queries it; synchronises `stream`.
 * lre_stream_resume: restore a checkpoint into this (for instance a new)
 *   context; the next chunk starts at the checkpoint's bases done.
 * No other call may use the context between begin and end (they share its
 * workspace); a call that reallocates it makes the stream calls return
 * LRE_ERR_INVALID_ARG. */
lre_status lre_stream_begin(lre_ctx *ctx, int n, lre_count_kind kind, int64_t shots_uniform);
lre_status lre_stream_chunk(lre_ctx *ctx, const void *counts, int64_t first_basis, int64_t num_bases,
                            lre_stream stream);
lre_status lre_stream_end(lre_ctx *ctx, double *theta, lre_c64 *rho, lre_stream stream);
lre_status lre_stream_checkpoint(lre_ctx *ctx, void *host, size_t bytes, size_t *needed, lre_stream stream);
lre_status lre_stream_resume(lre_ctx *ctx, const void *host, size_t bytes, lre_stream stream);

/* Synchronise `stream` and return (and clear) the first error latched by a
 * kernel since the last lre_sync. */
lre_status lre_sync(lre_ctx *ctx, lre_stream stream);

/* Static text for a status code. */
const char *lre_status_string(lre_status s);

/* Text of the last CUDA / library error seen by this context ("" if none);
 * with ctx NULL, the reason for the last failure of lre_assemble_noalloc on
 * the calling thread. */
const char *lre_last_error(lre_ctx *ctx);

/* Tracing: when enabled, every kernel launch (and every cuSOLVER / cuBLAS
 * call) made by the context is bracketed by a pair of CUDA events on its
 * stream.  lre_profile(ctx, 1) clears the record and starts recording;
 * lre_profile(ctx, 0) stops.  After the stream is synchronised,
 * lre_profile_get(ctx, i, &name, &ms) returns the i-th record (0 <=
 * i < lre_profile_count(ctx)): a static name and its device time in ms. */
lre_status lre_profile(lre_ctx *ctx, int enable);
int lre_profile_count(lre_ctx *ctx);
lre_status lre_profile_get(lre_ctx *ctx, int i, const char **name, float *ms);

/* Number of this library's own kernels launched by the context so far
 * (library calls such as the eigensolver are not counted). */
uint64_t lre_launch_count(lre_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* LRE_H */
