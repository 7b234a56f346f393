// lre_estimate_host: steps (i)+(ii) end to end from host memory.
//
// The input (dense counts or per-basis shot records) is streamed to the
// device in row chunks on a copy stream owned by the context, each chunk's
// copy overlapping the device work on the previous one, and where the fold
// plan starts with the six-qubit first pass (n >= 7, uniform shots) that pass
// runs on each chunk's whole tile rows (729 basis rows each) as soon as they
// have landed.  Shot records are histogrammed into dense device counts; when
// the context's workspace limit leaves no room for those (or a test forces
// it), records feeding the tensor-core first pass (at most 2047 shots per
// basis) are instead grouped by count tile per chunk and the pass builds its
// count tiles from them in shared memory, so no dense counts exist on the
// device.  The
// remaining passes follow; theta is copied back on the copy stream while the
// assembly of rho runs, and rho last.  Host buffers should be pinned
// (cudaHostAlloc / cudaHostRegister) for the copies to run asynchronously;
// pageable memory works but serialises.
#include <cuda_runtime.h>

#include "lre_internal.cuh"

namespace lre {
namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

lre_status estimate_host_run(lre_ctx *ctx, const void *host_in, int host_kind, int64_t shots,
                             int n, double *theta_host, lre_c64 *rho_host, cudaStream_t s) {
  const int64_t B = ipow(3, n);
  const int64_t d = 1ll << n;
  const bool records = host_kind == LRE_HOST_RECORDS_U16;
  const lre_count_kind ck = records ? (shots <= 32767 ? LRE_COUNTS_I16 : LRE_COUNTS_I32)
                                    : static_cast<lre_count_kind>(host_kind);
  const size_t csz = (ck == LRE_COUNTS_I16) ? 2 : 4;
  const size_t counts_bytes = (size_t)B * d * csz;
  const size_t theta_bytes = (size_t)ipow(4, n) * sizeof(double);
  const size_t rho_bytes = rho_host ? (size_t)d * d * sizeof(lre_c64) : 0;
  // the device buffers come first (the first-pass split depends on the
  // counts' alignment); chunk: a whole number of rows, about 256 MB of host
  // input, and a whole number of tile rows when the first pass runs per chunk
  const size_t row_in = records ? (size_t)shots * sizeof(uint16_t) : (size_t)d * csz;
  FoldArgs probe{nullptr, ck, n, nullptr, shots, nullptr, nullptr};
  probe.counts = reinterpret_cast<const void *>((uintptr_t)256);  // 256-byte aligned, as in the workspace
  const int64_t unit = fold_split_rows(ctx, probe);
  // shot records that can feed the tensor-core first pass directly (grouped
  // by tile per chunk): no dense counts on the device at all
  const bool direct_ok = records && unit > 0 && shots % 8 == 0 && fold_first_is_tensor(ctx, probe);
  int64_t rows = (int64_t)(ctx->host_chunk_bytes / row_in);
  if (unit > 0) rows = (rows / unit > 0 ? rows / unit : 1) * unit;
  if (rows < 1) rows = 1;
  if (rows > B) rows = B;
  const size_t chunk_in = (size_t)rows * row_in;
  const size_t fold_ws = fold_workspace_bytes(n, ck, false, shots, ctx->first_variant);
  const size_t asm_ws = rho_host ? assemble_workspace_bytes(n) : 0;
  const size_t dev_ws = up256(fold_ws > asm_ws ? fold_ws : asm_ws);
  const size_t t_bytes = rho_host ? up256((size_t)ipow(4, n) * sizeof(int64_t)) : 0;
  const size_t fixed = dev_ws + up256(theta_bytes) + up256(rho_bytes) + (records ? 2 * up256(chunk_in) : 0) + t_bytes;
  const size_t offs_bytes = up256((size_t)(rows / 729 + 1) * ((size_t)2 << (n - 6)) * sizeof(int32_t));
  const size_t need_dense = fixed + up256(counts_bytes);
  const size_t need_direct = fixed + 256 + 2 * (up256(chunk_in) + offs_bytes);
  // Dense device counts (ingest, then the TMA-fed first pass) are faster on
  // skewed data: a structured state sends most shots of a tile row into a few
  // count cells, whose shared-memory adds serialise in the records-fed pass.
  // The records-fed pass runs when forced, or when the context's workspace
  // limit holds it but not the dense counts.
  const bool direct = direct_ok && (ctx->records_direct ||
                                    (ctx->ws_limit > 0 && need_dense > ctx->ws_limit && need_direct <= ctx->ws_limit));
  const size_t counts_held = direct ? 256 : up256(counts_bytes);
  const size_t need = direct ? need_direct : need_dense;
  lre_status st = ensure_workspace(ctx, need);
  if (st != LRE_OK) return st;
  char *p = static_cast<char *>(ctx->ws);
  void *ws = p;
  char *counts = p + dev_ws;
  double *theta = reinterpret_cast<double *>(counts + counts_held);
  lre_c64 *rho = reinterpret_cast<lre_c64 *>(reinterpret_cast<char *>(theta) + up256(theta_bytes));
  char *tail = reinterpret_cast<char *>(rho) + up256(rho_bytes);
  int64_t *T = rho_host ? reinterpret_cast<int64_t *>(tail) : nullptr;
  char *stage[2] = {tail + t_bytes, tail + t_bytes + up256(chunk_in)};  // records only
  char *grouped = stage[1] + up256(chunk_in);                              // direct only
  uint16_t *entries[2] = {reinterpret_cast<uint16_t *>(grouped),
                          reinterpret_cast<uint16_t *>(grouped + up256(chunk_in) + offs_bytes)};
  int32_t *offs[2] = {reinterpret_cast<int32_t *>(grouped + up256(chunk_in)),
                      reinterpret_cast<int32_t *>(grouped + 2 * up256(chunk_in) + offs_bytes)};

  cudaError_t e = cudaSuccess;
  if (!ctx->copy_stream) {
    e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&ctx->ev_copied[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_free[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_theta, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream");
  }
  FoldArgs fa{counts, ck, n, nullptr, shots, theta, nullptr};
  fa.T = T;
  const bool split = unit > 0 && fold_split_rows(ctx, fa) == unit;
  if (direct && !split) return LRE_ERR_UNSUPPORTED;  // the records path has no dense counts to fall back on
  cudaStream_t cs = ctx->copy_stream;
  // the copy stream must not run ahead of work the caller queued on s
  e = cudaEventRecord(ctx->ev_free[0], s);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_free[1], s);
  const char *src = static_cast<const char *>(host_in);
  for (int64_t r0 = 0, k = 0; r0 < B && e == cudaSuccess; r0 += rows, ++k) {
    const int64_t nr = (r0 + rows <= B) ? rows : (B - r0);
    const int slot = (int)(k & 1);
    char *dst = records ? stage[slot] : counts + (size_t)r0 * d * csz;
    e = cudaStreamWaitEvent(cs, ctx->ev_free[slot], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst, src + (size_t)r0 * row_in, (size_t)nr * row_in, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_copied[slot], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->ev_copied[slot], 0);
    if (e == cudaSuccess && direct) {
      st = tile_bucket_run(ctx, reinterpret_cast<const uint16_t *>(dst), nr / 729, shots, n, entries[slot],
                           offs[slot], s);
      if (st != LRE_OK) return st;
    } else if (e == cudaSuccess && records) {
      st = histogram_run(ctx, reinterpret_cast<const uint16_t *>(dst), nr, shots, n,
                         counts + (size_t)r0 * d * csz, ck, s);
      if (st != LRE_OK) return st;
    }
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_free[slot], s);
    if (e == cudaSuccess && split) {  // first pass over this chunk's tile rows
      FoldArgs f1 = fa;
      f1.stage = 1;
      f1.ah_begin = r0 / unit;
      f1.ah_end = (r0 + nr) / unit;
      if (direct) {
        f1.rec_entries = entries[slot];
        f1.rec_offs = offs[slot];
      }
      if ((st = fold_run(ctx, f1, ws, dev_ws, s)) != LRE_OK) return st;
    }
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "host input streaming");
  FoldArgs rest = fa;
  rest.stage = split ? 2 : 0;
  if ((st = fold_run(ctx, rest, ws, dev_ws, s)) != LRE_OK) return st;
  // theta is final: copy it back on the copy stream while rho is assembled
  e = cudaEventRecord(ctx->ev_theta, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->ev_theta, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(theta_host, theta, theta_bytes, cudaMemcpyDeviceToHost, cs);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "theta copy-back");
  if (rho_host && (st = assemble_int_run(ctx, T, n, shots, rho, ws, s)) != LRE_OK) return st;
  if (rho_host) e = cudaMemcpyAsync(rho_host, rho, rho_bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "host outputs");
  int code = 0;
  e = cudaMemcpy(&code, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && code != 0) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "status");
  return static_cast<lre_status>(code);
}

}  // namespace lre
