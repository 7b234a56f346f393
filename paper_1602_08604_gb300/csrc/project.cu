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
// Rebuild with the cheaper of two equal forms (K kept, D dropped, s = a/i):
//   rho_hat = sum_{j in K} (l_j + s) v_j v_j^dag                       (|K| <= |D|)
//   rho_hat = mu + s I + sum_{j in D} (-(l_j + s)) v_j v_j^dag          (|D| <  |K|)
// (-(l_j + s) >= 0 for every dropped j), each as one Hermitian rank-k update.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <vector>

#include "lre_internal.cuh"

namespace lre {
namespace {

struct SmolinResult {
  int64_t kept;
  double shift;
};

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

// Scale columns [j0, j1) of column-major V (d x d) by sqrt(sign * (W_j + s)).
__global__ void scale_columns(double2 *V, const double *W, int64_t d, int64_t j0, int64_t j1,
                              const SmolinResult *res, double sign) {
  const double s = res->shift;
  const int64_t total = (j1 - j0) * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = j0 + e / d;
    double c = sign * (W[j] + s);
    c = c > 0.0 ? sqrt(c) : 0.0;
    double2 &x = V[j * d + (e % d)];
    x.x *= c;
    x.y *= c;
  }
}

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

}  // namespace

lre_status project_run(lre_ctx *ctx, const lre_c64 *rho_in, int n, lre_c64 *rho_out,
                       double *eig_mu, double *eig_rho, cudaStream_t s) {
  const int64_t d = 1ll << n;
  const int64_t N2 = d * d;
  cusolverDnHandle_t solver = reinterpret_cast<cusolverDnHandle_t>(ctx->solver);
  cublasHandle_t blas = reinterpret_cast<cublasHandle_t>(ctx->blas);
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
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t mat = up((size_t)N2 * sizeof(double2));
  const size_t need = 2 * mat + up(d * sizeof(double)) + up(dev_bytes) + up(sizeof(SmolinResult)) + 256;
  lre_status ws = ensure_workspace(ctx, need);
  if (ws != LRE_OK) {
    cusolverDnDestroyParams(params);
    return ws;
  }
  char *p = static_cast<char *>(ctx->ws);
  double2 *A = reinterpret_cast<double2 *>(p);
  double2 *C = reinterpret_cast<double2 *>(p + mat);
  double *W = reinterpret_cast<double *>(p + 2 * mat);
  void *work = p + 2 * mat + up(d * sizeof(double));
  SmolinResult *res = reinterpret_cast<SmolinResult *>(p + 2 * mat + up(d * sizeof(double)) + up(dev_bytes));
  int *info = reinterpret_cast<int *>(reinterpret_cast<char *>(res) + up(sizeof(SmolinResult)));
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
  int hinfo = 0;
  cudaError_t e = cudaMemcpyAsync(&hres, res, sizeof(hres), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "projection spectrum");
  if (hinfo != 0) {
    ctx->last_error = "cusolverDnXsyevd info = " + std::to_string(hinfo);
    return LRE_ERR_EIG_FAILED;
  }
  const int64_t kept = hres.kept, dropped = d - kept;
  if (kept <= dropped) {
    // rho_hat = W W^dag, W = V_K diag(sqrt(l + s)); K = the `kept` largest (last columns)
    {
      Launch L(ctx, "scale_columns", s);
      scale_columns<<<grid, 256, 0, s>>>(A, W, d, d - kept, d, res, 1.0);
    }
    const double alpha = 1.0, beta = 0.0;
    Launch L(ctx, "herk(cublas)", s, 0);
    cublasStatus_t bs = cublasZherk(blas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, (int)d, (int)kept, &alpha,
                                    reinterpret_cast<const cuDoubleComplex *>(A + (d - kept) * d),
                                    (int)d, &beta, reinterpret_cast<cuDoubleComplex *>(C), (int)d);
    if (bs != CUBLAS_STATUS_SUCCESS) {
      ctx->last_error = "cublasZherk failed";
      return LRE_ERR_CUDA;
    }
  } else if (dropped > 0) {
    // rho_hat = mu + s I + U U^dag, U = V_D diag(sqrt(-(l + s)))
    {
      Launch L(ctx, "scale_columns", s, 2);
      scale_columns<<<grid, 256, 0, s>>>(A, W, d, 0, dropped, res, -1.0);
      add_diag<<<(int)((d + 255) / 256), 256, 0, s>>>(C, d, res);
    }
    const double alpha = 1.0, beta = 1.0;
    Launch L(ctx, "herk(cublas)", s, 0);
    cublasStatus_t bs = cublasZherk(blas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, (int)d, (int)dropped,
                                    &alpha, reinterpret_cast<const cuDoubleComplex *>(A), (int)d, &beta,
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
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "projection kernels");
  return LRE_OK;
}

}  // namespace lre
