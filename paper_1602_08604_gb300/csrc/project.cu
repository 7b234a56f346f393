// Step (iii) of the LRE (arXiv:1602.08604 Sec. II): the closest density
// matrix to mu in the Frobenius norm, by the algorithm of Smolin, Gambetta
// and Smith that the paper uses: eigendecompose mu = V diag(l) V^dag, walk the
// eigenvalues from the smallest, dropping l_j while l_j + a/i < 0 (a the sum
// of the dropped values, i the number kept), shift the kept ones by a/i, and
// rebuild.  All of it in FP64 (the promoted complex64 input is exact).
//
// The row-major complex64 input read as a column-major matrix is mu^T =
// conj(mu); the projection commutes with conjugation, so the solver works on
// conj(mu) and the column-major result, read back row-major, is rho_hat.
//
// Two ways to the spectrum and the vectors the rebuild needs:
//   eigenvalue-first (default for d >= 64): cuSOLVER reduces conj(mu) to a
//     real tridiagonal T = Q^dag conj(mu) Q (the O(d^3) part), every
//     eigenvalue of T comes from bisection (tridiag.cu), the Smolin walk runs
//     on them, and eigenvectors are formed only for the smaller of the kept
//     and dropped sets (inverse iteration on T, then Q applied to those few
//     columns).  At n = 14 the estimate keeps a few dozen of 16384 eigenvalues,
//     so the back-transformation of the full eigenbasis is skipped;
//   full: cuSOLVER's divide-and-conquer eigendecomposition (Xsyevd), used
//     for small d and whenever the needed set exceeds PARTIAL_MAX vectors.
//
// Rebuild with the cheaper of two equal forms (K kept, D dropped, s = a/i):
//   rho_hat = sum_{j in K} (l_j + s) v_j v_j^dag                       (|K| <= |D|)
//   rho_hat = mu + s I + sum_{j in D} (-(l_j + s)) v_j v_j^dag          (|D| <  |K|)
// (-(l_j + s) >= 0 for every dropped j), each as one Hermitian rank-k update.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <cfloat>
#include <string>
#include <vector>

#include "lre_internal.cuh"

namespace lre {
namespace {

__global__ void promote_kernel(const float2 *in, double2 *a, double2 *b, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = in[i];
    const double2 w = make_double2((double)v.x, (double)v.y);
    a[i] = w;
    b[i] = w;
  }
}

// Serial Smolin walk over the ascending spectrum W (one thread).
__global__ void smolin_kernel(const double *W, int64_t d, SmolinResult *res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t dropped = 0, kept = d;
  double a = 0.0;
  while (kept > 0 && W[dropped] + a / (double)kept < 0.0) {
    a += W[dropped];
    ++dropped;
    --kept;
  }
  res->kept = kept;
  res->shift = kept > 0 ? a / (double)kept : 0.0;
}

__global__ void spectra_kernel(const double *W, int64_t d, const SmolinResult *res, double *eig_mu,
                               double *eig_rho) {
  const int64_t kept = res->kept;
  const double s = res->shift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double l = W[d - 1 - i];
    if (eig_mu) eig_mu[i] = l;
    if (eig_rho) eig_rho[i] = (i < kept) ? l + s : 0.0;
  }
}

// Scale column t of the column-major d x m block Z by sqrt(sign * (w[t] + s)).
__global__ void scale_block(double2 *Z, const double *w, int64_t d, int64_t m, const SmolinResult *res,
                            double sign) {
  const double s = res->shift;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    double c = sign * (w[e / d] + s);
    c = c > 0.0 ? sqrt(c) : 0.0;
    Z[e].x *= c;
    Z[e].y *= c;
  }
}

// Real column-major block -> complex (imaginary part zero).
__global__ void to_complex(const double *X, double2 *Z, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    Z[e] = make_double2(X[e], 0.0);
}

}  // namespace

// Gershgorin bounds and norm of T, and the squared off-diagonal (one CTA).
__global__ void tri_prepare(const double *a, const double *b, int64_t n, double *b2, double *stats) {
  __shared__ double lo_s[256], hi_s[256], bb_s[256];
  double lo = 1e308, hi = -1e308, bb = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const double l = k > 0 ? fabs(b[k - 1]) : 0.0, r = k + 1 < n ? fabs(b[k]) : 0.0;
    lo = fmin(lo, a[k] - l - r);
    hi = fmax(hi, a[k] + l + r);
    if (k + 1 < n) {
      b2[k] = b[k] * b[k];
      bb = fmax(bb, b2[k]);
    }
  }
  lo_s[threadIdx.x] = lo; hi_s[threadIdx.x] = hi; bb_s[threadIdx.x] = bb;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      lo_s[threadIdx.x] = fmin(lo_s[threadIdx.x], lo_s[threadIdx.x + o]);
      hi_s[threadIdx.x] = fmax(hi_s[threadIdx.x], hi_s[threadIdx.x + o]);
      bb_s[threadIdx.x] = fmax(bb_s[threadIdx.x], bb_s[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[0] = lo_s[0];
    stats[1] = hi_s[0];
    stats[2] = bb_s[0];
  }
}

namespace {

__global__ void add_diag(double2 *C, int64_t d, const SmolinResult *res) {
  const double s = res->shift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
       i += (int64_t)gridDim.x * blockDim.x)
    C[i * d + i].x += s;
}

// out[r][c] (row-major) from the lower triangle of column-major C = conj(rho_hat):
//   r >= c: conj(C(r, c)) = conj(buf[r + c d]);   r < c: buf[c + r d].
// 32 x 32 tiles, both reads staged through shared memory so that every global
// access is coalesced.
__global__ void emit_kernel(const double2 *C, float2 *out, int64_t d) {
  __shared__ double2 up[32][33];  // up[i][j] = buf[(c0 + i) + (r0 + j) d]
  __shared__ double2 lo[32][33];  // lo[i][j] = buf[(r0 + i) + (c0 + j) d]
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const bool need_up = (r0 < c0 + 31);   // some r < c in this tile
  const bool need_lo = (r0 + 31 >= c0);  // some r >= c in this tile
  for (int j = ty; j < 32; j += 8) {
    if (need_up) up[tx][j] = C[(c0 + tx) + (r0 + j) * d];
    if (need_lo) lo[tx][j] = C[(r0 + tx) + (c0 + j) * d];
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int64_t r = r0 + i, c = c0 + tx;
    double2 v;
    if (r < c) {
      v = up[tx][i];
    } else {
      const double2 w = lo[i][tx];
      v = make_double2(w.x, -w.y);
    }
    if (r == c) v.y = 0.0;  // a Hermitian matrix has a real diagonal
    out[r * d + c] = make_float2((float)v.x, (float)v.y);
  }
}

__global__ void emit_small(const double2 *C, float2 *out, int64_t d) {
  for (int64_t e = threadIdx.x; e < d * d; e += blockDim.x) {
    const int64_t r = e / d, c = e % d;
    double2 v;
    if (r < c) {
      v = C[c + r * d];
    } else {
      const double2 w = C[r + c * d];
      v = make_double2(w.x, -w.y);
    }
    if (r == c) v.y = 0.0;
    out[e] = make_float2((float)v.x, (float)v.y);
  }
}

lre_status get_handles(lre_ctx *ctx, cudaStream_t s, cusolverDnHandle_t &solver, cublasHandle_t &blas) {
  solver = reinterpret_cast<cusolverDnHandle_t>(ctx->solver);
  blas = reinterpret_cast<cublasHandle_t>(ctx->blas);
  if (!solver) {
    if (cusolverDnCreate(&solver) != CUSOLVER_STATUS_SUCCESS) {
      ctx->last_error = "cusolverDnCreate failed";
      return LRE_ERR_CUDA;
    }
    ctx->solver = reinterpret_cast<cusolverDnContext *>(solver);
  }
  if (!blas) {
    if (cublasCreate(&blas) != CUBLAS_STATUS_SUCCESS) {
      ctx->last_error = "cublasCreate failed";
      return LRE_ERR_CUDA;
    }
    ctx->blas = reinterpret_cast<cublasContext *>(blas);
  }
  cusolverDnSetStream(solver, s);
  cublasSetStream(blas, s);
  return LRE_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// C <- the projected matrix from the m vectors Z (column-major d x m, unit
// norm, eigenvalues w): kept form C = sum (w + s) z z^dag, or dropped form
// C = mu + s I + sum -(w + s) z z^dag with C holding mu on entry; then the
// complex64 row-major output.  Z is scaled in place.
lre_status rebuild_emit(lre_ctx *ctx, cublasContext *blas_ctx, double2 *C, double2 *Z, const double *w, int64_t d,
                        int64_t m, bool kept_form, const SmolinResult *res, lre_c64 *rho_out, cudaStream_t s) {
  cublasHandle_t blas = reinterpret_cast<cublasHandle_t>(blas_ctx);
  const int grid = ctx->num_sms * 8;
  if (kept_form) {
    {
      Launch L(ctx, "scale_columns", s);
      scale_block<<<grid, 256, 0, s>>>(Z, w, d, m, res, 1.0);
    }
    const double alpha = 1.0, beta = 0.0;
    Launch L(ctx, "herk(cublas)", s, 0);
    cublasStatus_t bs = cublasZherk(blas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, (int)d, (int)m, &alpha,
                                    reinterpret_cast<const cuDoubleComplex *>(Z), (int)d, &beta,
                                    reinterpret_cast<cuDoubleComplex *>(C), (int)d);
    if (bs != CUBLAS_STATUS_SUCCESS) {
      ctx->last_error = "cublasZherk failed";
      return LRE_ERR_CUDA;
    }
  } else if (m > 0) {
    {
      Launch L(ctx, "scale_columns", s, 2);
      scale_block<<<grid, 256, 0, s>>>(Z, w, d, m, res, -1.0);
      add_diag<<<(int)((d + 255) / 256), 256, 0, s>>>(C, d, res);
    }
    const double alpha = 1.0, beta = 1.0;
    Launch L(ctx, "herk(cublas)", s, 0);
    cublasStatus_t bs = cublasZherk(blas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, (int)d, (int)m, &alpha,
                                    reinterpret_cast<const cuDoubleComplex *>(Z), (int)d, &beta,
                                    reinterpret_cast<cuDoubleComplex *>(C), (int)d);
    if (bs != CUBLAS_STATUS_SUCCESS) {
      ctx->last_error = "cublasZherk failed";
      return LRE_ERR_CUDA;
    }
  }
  Launch L(ctx, "emit", s);
  if (d >= 32) {
    dim3 g((unsigned)(d / 32), (unsigned)(d / 32)), b(32, 8);
    emit_kernel<<<g, b, 0, s>>>(C, reinterpret_cast<float2 *>(rho_out), d);
  } else {
    emit_small<<<1, 256, 0, s>>>(C, reinterpret_cast<float2 *>(rho_out), d);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "projection kernels");
  return LRE_OK;
}

namespace {

// Reads back the Smolin result and a cuSOLVER info word.
lre_status read_back(lre_ctx *ctx, const SmolinResult *res, const int *info, const char *what, SmolinResult &hres,
                     cudaStream_t s) {
  int hinfo = 0;
  cudaError_t e = cudaMemcpyAsync(&hres, res, sizeof(hres), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "projection spectrum");
  if (hinfo != 0) {
    ctx->last_error = std::string(what) + " info = " + std::to_string(hinfo);
    return LRE_ERR_EIG_FAILED;
  }
  return LRE_OK;
}

constexpr int64_t PARTIAL_MAX = 1024;  // most eigenvectors the eigenvalue-first path forms
constexpr int64_t KRYLOV_MIN_D = 2048;  // smallest d the Krylov path takes

// Eigenvalue-first projection; *fallback = true (nothing written to rho_out)
// when the smaller of the kept and dropped sets exceeds PARTIAL_MAX.
lre_status project_partial(lre_ctx *ctx, cusolverDnHandle_t solver, cublasHandle_t blas, const lre_c64 *rho_in,
                           int64_t d, lre_c64 *rho_out, double *eig_mu, double *eig_rho, cudaStream_t s,
                           bool *fallback) {
  *fallback = false;
  const int N = (int)d;
  int lw_trd = 0, lw_mtr = 0;
  if (cusolverDnZhetrd_bufferSize(solver, CUBLAS_FILL_MODE_LOWER, N, nullptr, N, nullptr, nullptr, nullptr,
                                  &lw_trd) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnZunmtr_bufferSize(solver, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, N,
                                  (int)(d < PARTIAL_MAX ? d : PARTIAL_MAX), nullptr, N, nullptr, nullptr, N,
                                  &lw_mtr) != CUSOLVER_STATUS_SUCCESS) {
    ctx->last_error = "tridiagonal reduction buffer size query failed";
    return LRE_ERR_CUDA;
  }
  const int64_t mmax = d < PARTIAL_MAX ? d : PARTIAL_MAX;
  const size_t mat = up256((size_t)d * d * sizeof(double2));
  const size_t vec = up256((size_t)d * sizeof(double));
  const size_t lw = up256((size_t)(lw_trd > lw_mtr ? lw_trd : lw_mtr) * sizeof(double2));
  const size_t need = 2 * mat + 5 * vec + up256((size_t)d * sizeof(double2)) + lw +
                      up256((size_t)d * mmax * sizeof(double)) + up256((size_t)d * mmax * sizeof(double2)) +
                      up256((size_t)mmax * 5 * d * sizeof(double)) + up256((mmax + 2) * sizeof(int)) + 1024;
  lre_status st = ensure_workspace(ctx, need);
  if (st != LRE_OK) return st;
  char *p = static_cast<char *>(ctx->ws);
  double2 *A = reinterpret_cast<double2 *>(p);                p += mat;
  double2 *C = reinterpret_cast<double2 *>(p);                p += mat;
  double *ta = reinterpret_cast<double *>(p);                 p += vec;   // T diagonal
  double *tb = reinterpret_cast<double *>(p);                 p += vec;   // T off-diagonal
  double *tb2 = reinterpret_cast<double *>(p);                p += vec;   // its squares
  double *W = reinterpret_cast<double *>(p);                  p += vec;   // ascending eigenvalues
  double *stats = reinterpret_cast<double *>(p);              p += vec;   // lo, hi, max b^2
  double2 *tau = reinterpret_cast<double2 *>(p);              p += up256((size_t)d * sizeof(double2));
  double2 *work = reinterpret_cast<double2 *>(p);             p += lw;
  double *Xr = reinterpret_cast<double *>(p);                 p += up256((size_t)d * mmax * sizeof(double));
  double2 *Z = reinterpret_cast<double2 *>(p);                p += up256((size_t)d * mmax * sizeof(double2));
  double *scratch = reinterpret_cast<double *>(p);            p += up256((size_t)mmax * 5 * d * sizeof(double));
  int *cl = reinterpret_cast<int *>(p);                       p += up256((mmax + 2) * sizeof(int));
  SmolinResult *res = reinterpret_cast<SmolinResult *>(p);    p += 256;
  int *info = reinterpret_cast<int *>(p);                     p += 256;
  int *nclust = reinterpret_cast<int *>(p);

  const int grid = ctx->num_sms * 8;
  {
    Launch L(ctx, "promote", s);
    promote_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float2 *>(rho_in), A, C, d * d);
  }
  {
    Launch L(ctx, "hetrd(cusolver)", s, 0);
    if (cusolverDnZhetrd(solver, CUBLAS_FILL_MODE_LOWER, N, reinterpret_cast<cuDoubleComplex *>(A), N, ta, tb,
                         reinterpret_cast<cuDoubleComplex *>(tau), reinterpret_cast<cuDoubleComplex *>(work),
                         lw_trd, info) != CUSOLVER_STATUS_SUCCESS) {
      ctx->last_error = "cusolverDnZhetrd failed";
      return LRE_ERR_EIG_FAILED;
    }
  }
  {
    Launch L(ctx, "tri_prepare", s);
    tri_prepare<<<1, 256, 0, s>>>(ta, tb, d, tb2, stats);
  }
  double hst[3];
  cudaError_t e = cudaMemcpyAsync(hst, stats, sizeof(hst), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tridiagonal bounds");
  const double tnorm = fmax(fabs(hst[0]), fabs(hst[1]));
  const double pivmin = DBL_MIN * fmax(1.0, hst[2]);
  const double pad = 2.0 * DBL_EPSILON * tnorm + 2.0 * pivmin;
  {
    Launch L(ctx, "tri_bisect", s);
    tri_bisect_kernel<<<(int)((d + 127) / 128), 128, 0, s>>>(ta, tb2, d, hst[0] - pad, hst[1] + pad,
                                                             4.0 * DBL_EPSILON * fmax(tnorm, DBL_MIN), pivmin, W,
                                                             0, d);
  }
  {
    Launch L(ctx, "smolin", s);
    smolin_kernel<<<1, 32, 0, s>>>(W, d, res);
  }
  if (eig_mu || eig_rho) {
    Launch L(ctx, "spectra", s);
    spectra_kernel<<<(int)((d + 255) / 256), 256, 0, s>>>(W, d, res, eig_mu, eig_rho);
  }
  SmolinResult hres;
  if ((st = read_back(ctx, res, info, "cusolverDnZhetrd", hres, s)) != LRE_OK) return st;
  const int64_t kept = hres.kept, dropped = d - kept;
  const bool kept_form = kept <= dropped;
  const int64_t m = kept_form ? kept : dropped;
  const int64_t off = kept_form ? d - kept : 0;  // first selected ascending index
  if (m > PARTIAL_MAX) {
    *fallback = true;
    return LRE_OK;
  }
  if (m > 0) {
    int hk = 0;
    {
      Launch L(ctx, "tri_clusters", s);
      tri_clusters<<<1, 32, 0, s>>>(W + off, (int)m, 1e-3 * tnorm, cl, nclust);
    }
    e = cudaMemcpyAsync(&hk, nclust, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "eigenvalue clusters");
    {
      Launch L(ctx, "tri_inverse_iteration", s, 1 + 2 * TRI_ROUNDS);
      tri_factor<<<(int)((m + 31) / 32), 32, 0, s>>>(ta, tb, d, W + off, (int)m, tnorm, scratch);
      for (int it = 0; it < TRI_ROUNDS; ++it) {
        tri_solve<<<(int)((m + 31) / 32), 32, 0, s>>>(scratch, d, (int)m, Xr, it == 0);
        tri_orthonormalise<<<hk, TRI_THREADS, 0, s>>>(Xr, d, cl);
      }
    }
    {
      Launch L(ctx, "to_complex", s);
      to_complex<<<grid, 256, 0, s>>>(Xr, Z, d * m);
    }
    Launch L(ctx, "unmtr(cusolver)", s, 0);
    if (cusolverDnZunmtr(solver, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, N, (int)m,
                         reinterpret_cast<cuDoubleComplex *>(A), N, reinterpret_cast<cuDoubleComplex *>(tau),
                         reinterpret_cast<cuDoubleComplex *>(Z), N, reinterpret_cast<cuDoubleComplex *>(work),
                         lw_mtr, info) != CUSOLVER_STATUS_SUCCESS) {
      ctx->last_error = "cusolverDnZunmtr failed";
      return LRE_ERR_EIG_FAILED;
    }
  }
  if ((st = rebuild_emit(ctx, reinterpret_cast<cublasContext *>(blas), C, Z, W + off, d, m, kept_form, res, rho_out, s)) != LRE_OK) return st;
  int hinfo = 0;
  e = cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "projection");
  if (hinfo != 0) {
    ctx->last_error = "cusolverDnZunmtr info = " + std::to_string(hinfo);
    return LRE_ERR_EIG_FAILED;
  }
  return LRE_OK;
}

}  // namespace

lre_status project_run(lre_ctx *ctx, const lre_c64 *rho_in, int n, lre_c64 *rho_out,
                       double *eig_mu, double *eig_rho, cudaStream_t s) {
  const int64_t d = 1ll << n;
  const int64_t N2 = d * d;
  cusolverDnHandle_t solver;
  cublasHandle_t blas;
  lre_status st0 = get_handles(ctx, s, solver, blas);
  if (st0 != LRE_OK) return st0;
  // Krylov path: without eig_mu (which asks for the whole spectrum), from
  // d = 2048 on; it falls back to the tridiagonal reduction when it cannot
  // decide or certify the threshold
  if (ctx->project_mode == 1 && d >= KRYLOV_MIN_D && !eig_mu) {
    bool fallback = false;
    st0 = project_krylov(ctx, reinterpret_cast<cublasContext *>(blas), rho_in, d, rho_out, eig_rho, s, &fallback);
    if (st0 != LRE_OK || !fallback) return st0;
  }
  if (ctx->project_mode >= 1 && d >= 64) {
    bool fallback = false;
    st0 = project_partial(ctx, solver, blas, rho_in, d, rho_out, eig_mu, eig_rho, s, &fallback);
    if (st0 != LRE_OK || !fallback) return st0;
  }
  cusolverDnParams_t params;
  if (cusolverDnCreateParams(&params) != CUSOLVER_STATUS_SUCCESS) {
    ctx->last_error = "cusolverDnCreateParams failed";
    return LRE_ERR_CUDA;
  }
  size_t dev_bytes = 0, host_bytes = 0;
  cusolverStatus_t st = cusolverDnXsyevd_bufferSize(
      solver, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, d, CUDA_C_64F, nullptr, d,
      CUDA_R_64F, nullptr, CUDA_C_64F, &dev_bytes, &host_bytes);
  if (st != CUSOLVER_STATUS_SUCCESS) {
    cusolverDnDestroyParams(params);
    ctx->last_error = "cusolverDnXsyevd_bufferSize failed";
    return LRE_ERR_CUDA;
  }
  const size_t mat = up256((size_t)N2 * sizeof(double2));
  const size_t need = 2 * mat + up256(d * sizeof(double)) + up256(dev_bytes) + up256(sizeof(SmolinResult)) + 256;
  lre_status ws = ensure_workspace(ctx, need);
  if (ws != LRE_OK) {
    cusolverDnDestroyParams(params);
    return ws;
  }
  char *p = static_cast<char *>(ctx->ws);
  double2 *A = reinterpret_cast<double2 *>(p);
  double2 *C = reinterpret_cast<double2 *>(p + mat);
  double *W = reinterpret_cast<double *>(p + 2 * mat);
  void *work = p + 2 * mat + up256(d * sizeof(double));
  SmolinResult *res = reinterpret_cast<SmolinResult *>(p + 2 * mat + up256(d * sizeof(double)) + up256(dev_bytes));
  int *info = reinterpret_cast<int *>(reinterpret_cast<char *>(res) + up256(sizeof(SmolinResult)));
  std::vector<char> host_work(host_bytes > 0 ? host_bytes : 1);

  const int grid = ctx->num_sms * 8;
  {
    Launch L(ctx, "promote", s);
    promote_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float2 *>(rho_in), A, C, N2);
  }
  {
    Launch L(ctx, "eigh(cusolver)", s, 0);
    st = cusolverDnXsyevd(solver, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, d,
                          CUDA_C_64F, A, d, CUDA_R_64F, W, CUDA_C_64F, work, dev_bytes,
                          host_work.data(), host_bytes, info);
  }
  cusolverDnDestroyParams(params);
  if (st != CUSOLVER_STATUS_SUCCESS) {
    ctx->last_error = "cusolverDnXsyevd failed";
    return LRE_ERR_EIG_FAILED;
  }
  {
    Launch L(ctx, "smolin", s);
    smolin_kernel<<<1, 32, 0, s>>>(W, d, res);
  }
  if (eig_mu || eig_rho) {
    Launch L(ctx, "spectra", s);
    spectra_kernel<<<(int)((d + 255) / 256), 256, 0, s>>>(W, d, res, eig_mu, eig_rho);
  }
  SmolinResult hres;
  lre_status rs = read_back(ctx, res, info, "cusolverDnXsyevd", hres, s);
  if (rs != LRE_OK) return rs;
  const int64_t kept = hres.kept, dropped = d - kept;
  // the eigenvectors are the columns of A, ascending: kept = the last `kept`
  if (kept <= dropped)
    return rebuild_emit(ctx, reinterpret_cast<cublasContext *>(blas), C, A + (d - kept) * d, W + (d - kept), d, kept, true, res, rho_out, s);
  return rebuild_emit(ctx, reinterpret_cast<cublasContext *>(blas), C, A, W, d, dropped, false, res, rho_out, s);
}

}  // namespace lre
