// Streamed steps (i)+(ii): the count matrix arrives in chunks of whole tile
// rows (729 consecutive bases) -- produced on the device just in time by a
// generator, or received over time -- and each chunk goes through the
// six-qubit first fold pass at once, so the 3^n x 2^n matrix never exists
// whole.  The first pass's partials of the tile rows done so far (a prefix
// of its output, tile rows being contiguous there) are the whole state
// between chunks: a checkpoint copies them to host memory with a header, and
// a resume restores them into another context.  lre_stream_end runs the
// remaining passes (the same ones lre_estimate runs) and the assembly.
#include <cuda_runtime.h>

#include <cstring>

#include "lre_internal.cuh"

namespace lre {
namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct StreamHeader {
  char magic[8];  // "LRESTRM1"
  int64_t n, kind, shots, rows_done, planes, elems, done_elems;
};

// fold + assembly workspace and the exact integers T, as lre_estimate.
void stream_sizes(lre_ctx *ctx, int n, lre_count_kind kind, int64_t shots, size_t *shared, size_t *tbytes) {
  const size_t f = fold_workspace_bytes(n, kind, false, shots, ctx->first_variant);
  const size_t a = assemble_workspace_bytes(n);
  *shared = up256(f > a ? f : a);
  *tbytes = up256((size_t)8 << (2 * n));
}

FoldArgs stream_args(lre_ctx *ctx, const void *counts) {
  FoldArgs fa{counts, ctx->stream_kind, ctx->stream_n, nullptr, ctx->stream_shots, nullptr, nullptr};
  return fa;
}

lre_status begin(lre_ctx *ctx, int n, lre_count_kind kind, int64_t shots) {
  if (n < 7) return LRE_ERR_UNSUPPORTED;  // the streamed first pass contracts six qubits of n > 6
  if (n > 14) return LRE_ERR_UNSUPPORTED;
  if ((kind != LRE_COUNTS_I16 && kind != LRE_COUNTS_I32) || shots <= 0) return LRE_ERR_INVALID_ARG;
  ctx->stream_active = 0;
  ctx->stream_n = n;
  ctx->stream_kind = kind;
  ctx->stream_shots = shots;
  ctx->stream_rows_done = 0;
  // a 256-byte aligned probe stands for every chunk (chunks must be 16-byte aligned)
  FoldArgs probe = stream_args(ctx, reinterpret_cast<const void *>((uintptr_t)256));
  if (fold_split_rows(ctx, probe) != 729) return LRE_ERR_UNSUPPORTED;
  size_t shared, tbytes;
  stream_sizes(ctx, n, kind, shots, &shared, &tbytes);
  lre_status st = ensure_workspace(ctx, shared + tbytes);
  if (st != LRE_OK) return st;
  ctx->stream_active = 1;
  ctx->stream_ws = ctx->ws;
  return LRE_OK;
}

}  // namespace
}  // namespace lre

using namespace lre;

extern "C" lre_status lre_stream_begin(lre_ctx *ctx, int n, lre_count_kind kind, int64_t shots_uniform) {
  if (!ctx) return LRE_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  return begin(ctx, n, kind, shots_uniform);
}

extern "C" lre_status lre_stream_chunk(lre_ctx *ctx, const void *counts, int64_t first_basis, int64_t num_bases,
                                       lre_stream stream) {
  if (!ctx || !counts || !ctx->stream_active) return LRE_ERR_INVALID_ARG;
  const int64_t B = ipow(3, ctx->stream_n);
  if (first_basis != ctx->stream_rows_done || num_bases <= 0 || first_basis % 729 != 0 || num_bases % 729 != 0 ||
      first_basis + num_bases > B || (reinterpret_cast<uintptr_t>(counts) & 15) != 0)
    return LRE_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  size_t shared, tbytes;
  stream_sizes(ctx, ctx->stream_n, ctx->stream_kind, ctx->stream_shots, &shared, &tbytes);
  if (ctx->ws != ctx->stream_ws) return LRE_ERR_INVALID_ARG;  // another call reallocated the workspace
  FoldArgs f1 = stream_args(ctx, counts);
  f1.stage = 1;
  f1.ah_begin = first_basis / 729;
  f1.ah_end = (first_basis + num_bases) / 729;
  f1.row_base = first_basis;
  f1.rows_in = num_bases;
  lre_status st = fold_run(ctx, f1, ctx->ws, shared, reinterpret_cast<cudaStream_t>(stream));
  if (st == LRE_OK) ctx->stream_rows_done += num_bases;
  return st;
}

extern "C" lre_status lre_stream_end(lre_ctx *ctx, double *theta, lre_c64 *rho, lre_stream stream) {
  if (!ctx || !theta || !ctx->stream_active || ctx->stream_rows_done != ipow(3, ctx->stream_n) ||
      ctx->ws != ctx->stream_ws)
    return LRE_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  size_t shared, tbytes;
  stream_sizes(ctx, ctx->stream_n, ctx->stream_kind, ctx->stream_shots, &shared, &tbytes);
  int64_t *T = rho ? reinterpret_cast<int64_t *>(static_cast<char *>(ctx->ws) + shared) : nullptr;
  FoldArgs rest = stream_args(ctx, ctx->ws);  // aligned, as every chunk was; not read
  rest.stage = 2;
  rest.theta = theta;
  rest.T = T;
  ctx->stream_active = 0;
  lre_status st = fold_run(ctx, rest, ctx->ws, shared, s);
  if (st != LRE_OK || !rho) return st;
  return assemble_int_run(ctx, T, ctx->stream_n, ctx->stream_shots, rho, ctx->ws, s);
}

extern "C" lre_status lre_stream_checkpoint(lre_ctx *ctx, void *host, size_t bytes, size_t *needed,
                                            lre_stream stream) {
  if (!ctx || !needed || !ctx->stream_active || ctx->ws != ctx->stream_ws) return LRE_ERR_INVALID_ARG;
  bool planes = false;
  int64_t elems = 0;
  FoldArgs probe = stream_args(ctx, reinterpret_cast<const void *>((uintptr_t)256));
  if (!fold_stage1_layout(ctx, probe, &planes, &elems)) return LRE_ERR_UNSUPPORTED;
  const int64_t tiles_per_row = (int64_t)1 << (ctx->stream_n - 6);
  const int64_t done = ctx->stream_rows_done / 729 * tiles_per_row * 4096;  // partials of the rows done
  const size_t body = (size_t)done * (planes ? 3 : 4);
  *needed = sizeof(StreamHeader) + body;
  if (!host) return LRE_OK;  // size query
  if (bytes < *needed) return LRE_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  StreamHeader h;
  std::memcpy(h.magic, "LRESTRM1", 8);
  h.n = ctx->stream_n;
  h.kind = ctx->stream_kind;
  h.shots = ctx->stream_shots;
  h.rows_done = ctx->stream_rows_done;
  h.planes = planes;
  h.elems = elems;
  h.done_elems = done;
  std::memcpy(host, &h, sizeof(h));
  char *dst = static_cast<char *>(host) + sizeof(h);
  const char *ws = static_cast<const char *>(ctx->ws);  // the first pass writes at the workspace's start
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (planes) {  // low halves, then the high bytes (a region of elems x 2 bytes further)
    e = cudaMemcpyAsync(dst, ws, (size_t)done * 2, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst + done * 2, ws + elems * 2, (size_t)done, cudaMemcpyDeviceToHost, s);
  } else {
    e = cudaMemcpyAsync(dst, ws, (size_t)done * 4, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "checkpoint copy");
}

extern "C" lre_status lre_stream_resume(lre_ctx *ctx, const void *host, size_t bytes, lre_stream stream) {
  if (!ctx || !host || bytes < sizeof(StreamHeader)) return LRE_ERR_INVALID_ARG;
  StreamHeader h;
  std::memcpy(&h, host, sizeof(h));
  if (std::memcmp(h.magic, "LRESTRM1", 8) != 0 || h.n < 7 || h.n > 14 || h.rows_done < 0 || h.rows_done % 729 != 0)
    return LRE_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  lre_status st = begin(ctx, (int)h.n, static_cast<lre_count_kind>(h.kind), h.shots);
  if (st != LRE_OK) return st;
  bool planes = false;
  int64_t elems = 0;
  FoldArgs probe = stream_args(ctx, reinterpret_cast<const void *>((uintptr_t)256));
  if (!fold_stage1_layout(ctx, probe, &planes, &elems) || planes != (h.planes != 0) || elems != h.elems ||
      h.done_elems != h.rows_done / 729 * ((int64_t)1 << (h.n - 6)) * 4096 ||
      bytes < sizeof(h) + (size_t)h.done_elems * (planes ? 3 : 4)) {
    ctx->stream_active = 0;
    return LRE_ERR_INVALID_ARG;  // a checkpoint of another instance or configuration
  }
  const char *src = static_cast<const char *>(host) + sizeof(h);
  char *ws = static_cast<char *>(ctx->ws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t done = h.done_elems;
  if (planes) {
    e = cudaMemcpyAsync(ws, src, (size_t)done * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws + elems * 2, src + done * 2, (size_t)done, cudaMemcpyHostToDevice, s);
  } else {
    e = cudaMemcpyAsync(ws, src, (size_t)done * 4, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ctx->stream_active = 0;
    return cuda_fail(ctx, e, "resume copy");
  }
  ctx->stream_rows_done = h.rows_done;
  return LRE_OK;
}
