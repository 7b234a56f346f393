// Step (iii) without the O(d^3) reduction: the Smolin et al. projection of
// Sec. II needs only the eigenpairs on one side of its threshold, so they are
// computed by the Lanczos method (FP64 scalars and work vector; the basis as
// FP32 pairs, the product with mu and the reorthogonalisation in double-float
// arithmetic) with full reorthogonalisation, on
// hand-written kernels (matrix-vector product, Gram-Schmidt projections,
// norms, Ritz vectors), and the small tridiagonal problem is solved by the
// bisection and inverse-iteration kernels of tridiag.cu.
//
// Threshold.  With the eigenvalues l_1 >= ... >= l_d of mu (trace 1), the
// projection keeps l_1..l_r, shifted by s = (1 - sum_{i<=r} l_i) / r, where r
// is the largest k with l_k - (sum_{i<=k} l_i - 1)/k > 0 -- the condition
// holds exactly for k <= r, so the top eigenvalues decide r as soon as the
// first failing one is known.  From the other end, Smolin's own walk over the
// smallest eigenvalues (drop l_j while l_j + a/i < 0) decides r once the
// eigenvalue that stops it is known.  Lanczos converges at both ends of the
// spectrum at once; the first end that decides r gives the vectors to form
// (the kept set, or the dropped set for the rebuild mu + sI - sum (l_j + s)
// v v^dag), and the other end is not needed.
//
// Certification.  Ritz values are accepted when their residual
// beta_J |s_J| is below 1e-11 ||mu||.  Krylov spaces see each multiple
// eigenvalue once, so a value whose copy was missed could move r; a second,
// short Lanczos run from a new start vector, with the accepted vectors in its
// basis (so it works on the deflated operator), must find nothing beyond the
// threshold, else the call falls back to the tridiagonal reduction.  The
// fallback also runs when r is not decided within KRYLOV_MAX steps.
//
// Layout: mu (row-major complex64) is promoted once to complex128 M (the
// same row-major order; the rebuild's working matrix, its norm and trace),
// while the Lanczos product reads the complex64 input itself; the Krylov
// basis Q holds one d-vector per row (vector t at Q + t d) as FP32 pairs.  y = mu x is the
// row-major product, so the vectors are eigenvectors of mu; the rebuild of
// project.cu works on conj(mu), whose eigenvectors are their conjugates.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "lre_internal.cuh"

namespace lre {
namespace {

constexpr int MV_RPW = 1;          // rows of M per warp of the product (eight warps per CTA)
constexpr int MV_CHUNK = 1024;     // x entries staged in shared memory at a time
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- the Lanczos product y = mu x in double-float arithmetic on the FP32 pipes --
// mu arrives as complex64, so its entries are exact FP32 numbers; with x held
// as two FP32 parts (x = xh + xl, |x - xh - xl| about 2^-48 |x|), each real
// product m x is p = RN(m xh) plus its exact error e = fma(m, xh, -p) plus
// m xl, and the row sums are kept as unevaluated FP32 pairs (sh, sl) with
// Knuth's TwoSum on the leading part: about 2^-44 relative per term, against
// 2^-53 in FP64 -- far inside the Lanczos tolerances -- at the FP32 rate,
// where GB300's FP64 rate had made the product FP64-bound, and reading 8
// bytes per entry of mu instead of 16.  The _rn intrinsics keep the compiler
// from contracting the steps into FMAs, which would break the exact errors.
__device__ __forceinline__ void df_mac(float &sh, float &sl, float m, float xh, float xl) {
  const float p = __fmul_rn(m, xh);
  const float e = __fmaf_rn(m, xh, -p);
  const float t = __fadd_rn(sh, p);  // TwoSum(sh, p) = t + err exactly
  const float bp = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, __fmaf_rn(m, xl, e)));
}

// The same for a product of two such pairs, (ah + al)(bh + bl): the leading
// product exactly (p and its error), the cross terms into the error part.
__device__ __forceinline__ void df_mac2(float &sh, float &sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float t = __fadd_rn(sh, p);
  const float bp = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// complex128 <-> {re hi, re lo, im hi, im lo} as FP32 (the Krylov basis, the
// split copies of the work vector): about 2^-48 relative per component
__device__ __forceinline__ float4 df_split(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}
__device__ __forceinline__ double2 df_join(float4 q) {
  return make_double2((double)q.x + (double)q.y, (double)q.z + (double)q.w);
}

__global__ void kry_split(const double2 *__restrict__ x, float4 *__restrict__ xs, int64_t d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
    xs[i] = df_split(x[i]);
}

// y = M x with M the row-major d x d complex64 matrix and x a basis row in
// split form; y also in split form for the reorthogonalisation.  MV_RPW rows
// per warp, x staged in shared memory (d a multiple of MV_CHUNK or d <
// MV_CHUNK); with one row per warp and whole chunks each lane loads its 32
// entries of the chunk before their products (more loads in flight: 4.9
// against 3.5 TB/s at d = 16384); the warp's partial sums are added in FP64.
template <int RPW>
__global__ void __launch_bounds__(256, 3) kry_matvec_df(const float2 *__restrict__ M, const float4 *__restrict__ xsplit,
                                                     double2 *__restrict__ y, float4 *__restrict__ ysplit,
                                                     int64_t d) {
  __shared__ float4 xs[MV_CHUNK];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = ((int64_t)blockIdx.x * 8 + warp) * RPW;
  float rh[RPW], rl[RPW], ih[RPW], il[RPW];
#pragma unroll
  for (int r = 0; r < RPW; ++r) rh[r] = rl[r] = ih[r] = il[r] = 0.f;
  const int64_t chunk = d < MV_CHUNK ? d : MV_CHUNK;
  for (int64_t c0 = 0; c0 < d; c0 += chunk) {
    __syncthreads();
    for (int k = threadIdx.x; k < chunk; k += blockDim.x) xs[k] = xsplit[c0 + k];
    __syncthreads();
    if (r0 < d) {
      const float2 *row = M + r0 * d + c0;
      if (RPW == 1 && chunk % 1024 == 0) {
        // thirty-two entries of the row loaded ahead of their products
        for (int k0 = lane; k0 < chunk; k0 += 1024) {
          float2 u[32];
#pragma unroll
          for (int q = 0; q < 32; ++q) u[q] = row[k0 + 32 * q];
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const float4 xv = xs[k0 + 32 * q];
            df_mac(rh[0], rl[0], u[q].x, xv.x, xv.y);
            df_mac(rh[0], rl[0], -u[q].y, xv.z, xv.w);
            df_mac(ih[0], il[0], u[q].x, xv.z, xv.w);
            df_mac(ih[0], il[0], u[q].y, xv.x, xv.y);
          }
        }
      } else {
        for (int k = lane; k < chunk; k += 32) {
          const float4 xv = xs[k];  // x re = xv.x + xv.y, x im = xv.z + xv.w
#pragma unroll
          for (int r = 0; r < RPW; ++r) {
            if (r0 + r < d) {
              const float2 u = row[(int64_t)r * d + k];
              df_mac(rh[r], rl[r], u.x, xv.x, xv.y);   // re += ur xr - ui xi
              df_mac(rh[r], rl[r], -u.y, xv.z, xv.w);
              df_mac(ih[r], il[r], u.x, xv.z, xv.w);   // im += ur xi + ui xr
              df_mac(ih[r], il[r], u.y, xv.x, xv.y);
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const double re = warp_sum((double)rh[r] + (double)rl[r]), im = warp_sum((double)ih[r] + (double)il[r]);
    if (lane == 0 && r0 + r < d) {
      y[r0 + r] = make_double2(re, im);
      ysplit[r0 + r] = df_split(make_double2(re, im));
    }
  }
}

// h[t] = q_t^dag w for t < m (one CTA per vector), the basis rows and w in
// split form, products and sums in double-float, the partial sums added in
// FP64.
__global__ void __launch_bounds__(RED_THREADS) kry_dots(const float4 *__restrict__ Q, int m,
                                                        const float4 *__restrict__ w, double2 *__restrict__ h,
                                                        int64_t d) {
  __shared__ double sr[RED_THREADS / 32], si[RED_THREADS / 32];
  for (int t = blockIdx.x; t < m; t += gridDim.x) {
    const float4 *q = Q + (int64_t)t * d;
    float rh = 0, rl = 0, ih = 0, il = 0;
    for (int64_t i = threadIdx.x; i < d; i += blockDim.x) {
      const float4 a = q[i], b = w[i];  // conj(a) b
      df_mac2(rh, rl, a.x, a.y, b.x, b.y);
      df_mac2(rh, rl, a.z, a.w, b.z, b.w);
      df_mac2(ih, il, a.x, a.y, b.z, b.w);
      df_mac2(ih, il, -a.z, -a.w, b.x, b.y);
    }
    const double re = warp_sum((double)rh + (double)rl), im = warp_sum((double)ih + (double)il);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
      sr[warp] = re;
      si[warp] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0, b = 0;
      for (int k = 0; k < RED_THREADS / 32; ++k) {
        a += sr[k];
        b += si[k];
      }
      h[t] = make_double2(a, b);
    }
    __syncthreads();
  }
}

// w -= sum_{t < m} h[t] q_t (basis rows in split form, h split into shared
// memory; dynamic shared memory m float4), and ws = the split w.  A CTA
// takes 64 entries of w; its four warp pairs sum over t = slice, slice + 4,
// ... in double-float, and the four partial sums meet in FP64.
constexpr int UPD_SLICES = 4;
__global__ void __launch_bounds__(256) kry_update(double2 *__restrict__ w, float4 *__restrict__ ws,
                                                  const float4 *__restrict__ Q, int m,
                                                  const double2 *__restrict__ h, int64_t d) {
  extern __shared__ float4 hs[];
  __shared__ double2 part[UPD_SLICES][64];
  for (int t = threadIdx.x; t < m; t += blockDim.x) hs[t] = df_split(h[t]);
  __syncthreads();
  const int e = threadIdx.x & 63, slice = threadIdx.x >> 6;
  for (int64_t i0 = (int64_t)blockIdx.x * 64; i0 < d; i0 += (int64_t)gridDim.x * 64) {
    const int64_t i = i0 + e;
    float rh = 0, rl = 0, ih = 0, il = 0;
    if (i < d) {
      for (int t = slice; t < m; t += UPD_SLICES) {
        const float4 q = Q[(int64_t)t * d + i];
        const float4 c = hs[t];  // q c
        df_mac2(rh, rl, q.x, q.y, c.x, c.y);
        df_mac2(rh, rl, -q.z, -q.w, c.z, c.w);
        df_mac2(ih, il, q.x, q.y, c.z, c.w);
        df_mac2(ih, il, q.z, q.w, c.x, c.y);
      }
    }
    part[slice][e] = make_double2((double)rh + (double)rl, (double)ih + (double)il);
    __syncthreads();
    if (slice == 0 && i < d) {
      double re = 0, im = 0;
#pragma unroll
      for (int k = 0; k < UPD_SLICES; ++k) {
        re += part[k][e].x;
        im += part[k][e].y;
      }
      double2 v = w[i];
      v.x -= re;
      v.y -= im;
      w[i] = v;
      ws[i] = df_split(v);
    }
    __syncthreads();
  }
}

// Sum of |w_i|^2 in one CTA per slice, added atomically into *acc (zeroed by
// the caller).
__global__ void __launch_bounds__(RED_THREADS) kry_norm2(const double2 *__restrict__ w, int64_t d, double *acc) {
  __shared__ double s[RED_THREADS / 32];
  double v = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = w[i];
    v = fma(a.x, a.x, v);
    v = fma(a.y, a.y, v);
  }
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < RED_THREADS / 32; ++k) t += s[k];
    atomicAdd(acc, t);
  }
}

// Close Lanczos step j: alpha[j] = Re(h1[c] + h2[c]) (c the column of q_j),
// beta[j] = ||w||, q_{j+1} = w / beta[j] (every thread recomputes the two
// scalars from device memory).  A vanishing beta (an invariant subspace) sets
// *breakdown and leaves q_{j+1} = 0.
__global__ void kry_close(const double2 *h1, const double2 *h2, int c, const double *nrm2, double tiny, double *alpha,
                          double *beta, int j, const double2 *w, float4 *qn, int64_t d, int *breakdown) {
  const double b = sqrt(*nrm2);
  const bool dead = !(b > tiny);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    alpha[j] = h1[c].x + h2[c].x;
    beta[j] = dead ? 0.0 : b;
    if (dead && *breakdown == 0) *breakdown = j + 1;  // the first vanishing step
  }
  if (!qn) return;
  const double inv = dead ? 0.0 : 1.0 / b;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = w[i];
    qn[i] = df_split(make_double2(v.x * inv, v.y * inv));  // the basis in split form
  }
}

// A deterministic start vector (splitmix64 of the index and a seed), not yet
// normalised.
__global__ void kry_start(double2 *q, int64_t d, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double a = (double)(z >> 11) * 0x1.0p-53 - 0.5;
    const double b = (double)((z << 11) >> 11) * 0x1.0p-53 - 0.5;
    q[i] = make_double2(a, b);
  }
}

// q (a basis row, split form) = v / ||v||
__global__ void kry_scale(const double2 *v, float4 *q, int64_t d, const double *nrm2) {
  const double inv = 1.0 / sqrt(*nrm2);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = v[i];
    q[i] = df_split(make_double2(a.x * inv, a.y * inv));
  }
}

// Ritz vectors: Z[:, k] = conj(sum_t S[t + k J] q_t) for k < m (Z column-major
// d x m, S column-major J x m real); eight columns per thread.
__global__ void __launch_bounds__(256) kry_ritz(const float4 *__restrict__ Q, int J, const double *__restrict__ S,
                                                int m, double2 *__restrict__ Z, int64_t d) {
  const int k0 = blockIdx.y * 8;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    double re[8], im[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) re[k] = im[k] = 0.0;
    for (int t = 0; t < J; ++t) {
      const double2 q = df_join(Q[(int64_t)t * d + i]);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k0 + k < m) {
          const double c = S[t + (int64_t)(k0 + k) * J];
          re[k] = fma(q.x, c, re[k]);
          im[k] = fma(q.y, c, im[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k0 + k < m) Z[i + (int64_t)(k0 + k) * d] = make_double2(re[k], -im[k]);
  }
}

// Row-major copy of the conjugate Ritz vectors back into basis rows (for the
// certification run): Q[t][i] = conj(Z[i + t d]).
__global__ void kry_seed(const double2 *Z, int m, float4 *Q, int64_t d) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = Z[e];
    Q[e] = df_split(make_double2(v.x, -v.y));
  }
}

// *acc += sum of the real diagonal of M (zeroed by the caller).
__global__ void __launch_bounds__(RED_THREADS) kry_trace(const double2 *__restrict__ M, int64_t d, double *acc) {
  __shared__ double s[RED_THREADS / 32];
  double v = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
    v += M[i * d + i].x;
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < RED_THREADS / 32; ++k) t += s[k];
    atomicAdd(acc, t);
  }
}

// Last components S[J-1 + k J] of the m inverse-iteration vectors.
__global__ void kry_last(const double *S, int J, int m, double *out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
    out[k] = S[(J - 1) + (int64_t)k * J];
}

// Promote the row-major complex64 input to complex128 (same order) into M and
// into C (the rebuild's working matrix, read there as column-major conj(mu)).
__global__ void kry_promote(const float2 *in, double2 *M, double2 *C, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = in[i];
    const double2 w = make_double2((double)v.x, (double)v.y);
    M[i] = w;
    C[i] = w;
  }
}

}  // namespace

namespace {

constexpr int KRY_CHECK = 64;           // Lanczos steps between convergence checks
constexpr int KRY_VERIFY = 64;          // steps of the certification run
constexpr int64_t KRY_MAX_VECS = 1024;  // most eigenvectors formed
constexpr int64_t KRY_MAX_STEPS = 2048;
constexpr double KRY_RTOL = 1e-11;      // accepted residual, relative to ||mu||_2

__global__ void kry_eig_rho(const double *w_asc, int64_t r, double shift, double *out, int64_t d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = i < r ? w_asc[r - 1 - i] + shift : 0.0;
}

struct KryBuffers {
  double2 *M, *W, *h1, *h2, *Z;
  float4 *Q;          // the Krylov basis, one row per vector, in split form (about 48 bits)
  const float2 *M32;  // the complex64 input, read by the double-float product
  float4 *Ws;         // the work vector W in split form
  double *alpha, *beta, *b2, *stats, *Wr, *Xr, *lu, *last, *nrm;
  int *cl, *nclust, *breakdown;
  SmolinResult *res;
  int64_t rows, ct_max;
};

// Ritz values and last eigenvector components of the J x J Lanczos matrix
// (alpha, beta) for its CB smallest and CT largest eigenvalues (ascending in
// Wr[0..CB+CT), vectors in Xr), copied to the host with beta[J-1].
struct RitzEnds {
  std::vector<double> w, last;
  double beta_next = 0, tnorm = 0;
};

lre_status ritz_ends(lre_ctx *ctx, const KryBuffers &B, const double *alpha, const double *beta, int J, int CB,
                     int CT, cudaStream_t s, RitzEnds &out) {
  {
    Launch L(ctx, "kry_tri_prepare", s);
    tri_prepare<<<1, 256, 0, s>>>(alpha, beta, J, B.b2, B.stats);
  }
  double hst[3];
  double bnext = 0;
  cudaError_t e = cudaMemcpyAsync(hst, B.stats, sizeof(hst), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bnext, beta + (J - 1), sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "Lanczos matrix bounds");
  const double tnorm = fmax(fabs(hst[0]), fabs(hst[1]));
  const double pivmin = DBL_MIN * fmax(1.0, hst[2]);
  const double pad = 2.0 * DBL_EPSILON * tnorm + 2.0 * pivmin;
  const double tol = 4.0 * DBL_EPSILON * fmax(tnorm, DBL_MIN);
  const int m = CB + CT;
  {
    Launch L(ctx, "kry_bisect", s, 2);  // one warp per Ritz value, two per CTA
    if (CB > 0)
      tri_multisect_kernel<<<(CB + 1) / 2, 64, 0, s>>>(alpha, B.b2, J, hst[0] - pad, hst[1] + pad, tol, pivmin,
                                                       B.Wr, 0, CB);
    tri_multisect_kernel<<<(CT + 1) / 2, 64, 0, s>>>(alpha, B.b2, J, hst[0] - pad, hst[1] + pad, tol, pivmin,
                                                     B.Wr + CB, J - CT, CT);
  }
  int hk = 0;
  {
    Launch L(ctx, "kry_clusters", s);
    tri_clusters<<<1, 32, 0, s>>>(B.Wr, m, 1e-8 * tnorm, B.cl, B.nclust);
  }
  e = cudaMemcpyAsync(&hk, B.nclust, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "Ritz clusters");
  {
    Launch L(ctx, "kry_inverse_iteration", s, 2 + 2 * TRI_ROUNDS);
    tri_factor<<<(m + 31) / 32, 32, 0, s>>>(alpha, beta, J, B.Wr, m, tnorm, B.lu);
    for (int it = 0; it < TRI_ROUNDS; ++it) {
      tri_solve<<<(m + 31) / 32, 32, 0, s>>>(B.lu, J, m, B.Xr, it == 0);
      tri_orthonormalise<<<hk, TRI_THREADS, 0, s>>>(B.Xr, J, B.cl);
    }
    kry_last<<<(m + 255) / 256, 256, 0, s>>>(B.Xr, J, m, B.last);
  }
  out.w.resize(m);
  out.last.resize(m);
  e = cudaMemcpyAsync(out.w.data(), B.Wr, m * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out.last.data(), B.last, m * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "Ritz values");
  out.beta_next = bnext;
  out.tnorm = tnorm;
  return LRE_OK;
}

// Lanczos steps [j0, j1) on basis rows base + j (rows 0..base + j - 1 fixed):
// every step reorthogonalises against all earlier rows (classical
// Gram-Schmidt, twice) and writes alpha[j], beta[j] and row base + j + 1.
lre_status lanczos_steps(lre_ctx *ctx, const KryBuffers &B, int64_t d, int64_t base, int j0, int j1, double *alpha,
                         double *beta, double tiny, cudaStream_t s) {
  const int red_grid = (int)std::min<int64_t>((d + RED_THREADS - 1) / RED_THREADS, (int64_t)ctx->num_sms * 4);
  const int upd_grid = (int)((d + 63) / 64);
  for (int j = j0; j < j1; ++j) {
    const int64_t c = base + j;  // the row of q_j
    const int cols = (int)(c + 1);
    {
      Launch L(ctx, "kry_matvec", s);  // W = mu q_j and its split copy
      kry_matvec_df<MV_RPW><<<(unsigned)((d + 8 * MV_RPW - 1) / (8 * MV_RPW)), 256, 0, s>>>(B.M32, B.Q + c * d, B.W,
                                                                                          B.Ws, d);
    }
    {
      Launch L(ctx, "kry_reorth", s, 4);
      const int dg = (int)std::min<int64_t>(cols, 2048);
      const size_t hs = (size_t)cols * sizeof(float4);
      kry_dots<<<dg, RED_THREADS, 0, s>>>(B.Q, cols, B.Ws, B.h1, d);
      kry_update<<<upd_grid, 256, hs, s>>>(B.W, B.Ws, B.Q, cols, B.h1, d);
      kry_dots<<<dg, RED_THREADS, 0, s>>>(B.Q, cols, B.Ws, B.h2, d);
      kry_update<<<upd_grid, 256, hs, s>>>(B.W, B.Ws, B.Q, cols, B.h2, d);
    }
    {
      Launch L(ctx, "kry_close", s, 2);
      cudaMemsetAsync(B.nrm, 0, sizeof(double), s);
      kry_norm2<<<red_grid, RED_THREADS, 0, s>>>(B.W, d, B.nrm);
      float4 *next = c + 1 < B.rows ? B.Q + (c + 1) * d : nullptr;
      kry_close<<<red_grid, RED_THREADS, 0, s>>>(B.h1, B.h2, (int)c, B.nrm, tiny, alpha, beta, j, B.W, next, d,
                                                 B.breakdown);
    }
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "Lanczos step");
}

// A fresh unit start vector in row `row`, orthogonal to rows [0, row).
lre_status start_vector(lre_ctx *ctx, const KryBuffers &B, int64_t d, int64_t row, uint64_t seed, cudaStream_t s) {
  const int red_grid = (int)std::min<int64_t>((d + RED_THREADS - 1) / RED_THREADS, (int64_t)ctx->num_sms * 4);
  // built in the FP64 work vector, stored into the basis row in split form
  Launch L(ctx, "kry_start", s, row > 0 ? 8 : 3);
  kry_start<<<red_grid, RED_THREADS, 0, s>>>(B.W, d, seed);
  if (row > 0) {
    const int cols = (int)row;
    const size_t hs = (size_t)cols * sizeof(float4);
    kry_split<<<red_grid, RED_THREADS, 0, s>>>(B.W, B.Ws, d);
    for (int pass = 0; pass < 2; ++pass) {
      kry_dots<<<(int)std::min<int64_t>(cols, 2048), RED_THREADS, 0, s>>>(B.Q, cols, B.Ws, B.h1, d);
      kry_update<<<(unsigned)((d + 63) / 64), 256, hs, s>>>(B.W, B.Ws, B.Q, cols, B.h1, d);
    }
  }
  cudaMemsetAsync(B.nrm, 0, sizeof(double), s);
  kry_norm2<<<red_grid, RED_THREADS, 0, s>>>(B.W, d, B.nrm);
  kry_scale<<<red_grid, RED_THREADS, 0, s>>>(B.W, B.Q + row * d, d, B.nrm);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "Lanczos start vector");
}

}  // namespace

lre_status project_krylov(lre_ctx *ctx, cublasContext *blas, const lre_c64 *rho_in, int64_t d, lre_c64 *rho_out,
                          double *eig_rho, cudaStream_t s, bool *fallback) {
  *fallback = true;
  const int64_t kmax = std::min<int64_t>(d / 2, KRY_MAX_STEPS);
  KryBuffers B{};
  B.rows = std::max<int64_t>(kmax + 1, KRY_MAX_VECS + KRY_VERIFY + 1);
  B.ct_max = KRY_MAX_VECS + 64;
  auto u = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t need = u(2 * sizeof(double)) + u((size_t)d * d * sizeof(double2)) + u((size_t)B.rows * d * sizeof(double2)) +
                      u((size_t)d * sizeof(double2)) + 2 * u((size_t)B.rows * sizeof(double2)) +
                      u((size_t)d * KRY_MAX_VECS * sizeof(double2)) + 3 * u((size_t)B.rows * sizeof(double)) +
                      u(4 * sizeof(double)) + u((size_t)B.ct_max * sizeof(double)) +
                      u((size_t)B.rows * B.ct_max * sizeof(double)) + u((size_t)5 * B.rows * B.ct_max * sizeof(double)) +
                      u((size_t)B.ct_max * sizeof(double)) + u(sizeof(double)) + u((size_t)(B.ct_max + 2) * sizeof(int)) +
                      3 * 256 + 2 * u((size_t)KRY_VERIFY * sizeof(double)) + u((size_t)d * sizeof(float4)) + 1024;
  lre_status st = ensure_workspace(ctx, need);
  if (st != LRE_OK) return st;
  char *p = static_cast<char *>(ctx->ws);
  auto take = [&](size_t bytes) {
    char *q = p;
    p += u(bytes);
    return q;
  };
  B.M = reinterpret_cast<double2 *>(take((size_t)d * d * sizeof(double2)));
  B.Q = reinterpret_cast<float4 *>(take((size_t)B.rows * d * sizeof(float4)));
  B.W = reinterpret_cast<double2 *>(take((size_t)d * sizeof(double2)));
  B.h1 = reinterpret_cast<double2 *>(take((size_t)B.rows * sizeof(double2)));
  B.h2 = reinterpret_cast<double2 *>(take((size_t)B.rows * sizeof(double2)));
  B.Z = reinterpret_cast<double2 *>(take((size_t)d * KRY_MAX_VECS * sizeof(double2)));
  B.alpha = reinterpret_cast<double *>(take((size_t)B.rows * sizeof(double)));
  B.beta = reinterpret_cast<double *>(take((size_t)B.rows * sizeof(double)));
  B.b2 = reinterpret_cast<double *>(take((size_t)B.rows * sizeof(double)));
  B.stats = reinterpret_cast<double *>(take(4 * sizeof(double)));
  B.Wr = reinterpret_cast<double *>(take((size_t)B.ct_max * sizeof(double)));
  B.Xr = reinterpret_cast<double *>(take((size_t)B.rows * B.ct_max * sizeof(double)));
  B.lu = reinterpret_cast<double *>(take((size_t)5 * B.rows * B.ct_max * sizeof(double)));
  B.last = reinterpret_cast<double *>(take((size_t)B.ct_max * sizeof(double)));
  B.nrm = reinterpret_cast<double *>(take(2 * sizeof(double)));
  B.cl = reinterpret_cast<int *>(take((size_t)(B.ct_max + 2) * sizeof(int)));
  B.nclust = reinterpret_cast<int *>(take(sizeof(int)));
  B.breakdown = reinterpret_cast<int *>(take(sizeof(int)));
  B.res = reinterpret_cast<SmolinResult *>(take(sizeof(SmolinResult)));
  double *alpha2 = reinterpret_cast<double *>(take((size_t)KRY_VERIFY * sizeof(double)));
  double *beta2 = reinterpret_cast<double *>(take((size_t)KRY_VERIFY * sizeof(double)));
  B.Ws = reinterpret_cast<float4 *>(take((size_t)d * sizeof(float4)));
  B.M32 = reinterpret_cast<const float2 *>(rho_in);  // unchanged until the rebuild writes rho_out

  const int grid = ctx->num_sms * 8;
  {
    Launch L(ctx, "kry_promote", s, 3);
    kry_promote<<<grid, 256, 0, s>>>(reinterpret_cast<const float2 *>(rho_in), B.M, B.M, d * d);
    cudaMemsetAsync(B.nrm, 0, 2 * sizeof(double), s);
    kry_norm2<<<grid, RED_THREADS, 0, s>>>(B.M, d * d, B.nrm);
    kry_trace<<<(int)((d + RED_THREADS - 1) / RED_THREADS), RED_THREADS, 0, s>>>(B.M, d, B.nrm + 1);
  }
  double fro_tr[2] = {0, 0};
  cudaError_t e = cudaMemsetAsync(B.breakdown, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(fro_tr, B.nrm, sizeof(fro_tr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "Krylov set-up");
  const double tiny = 1e-14 * sqrt(fro_tr[0]);
  const double trace = fro_tr[1];  // Tr mu (1 up to the complex64 rounding of the diagonal)
  if ((st = start_vector(ctx, B, d, 0, 0x5EED0001ull, s)) != LRE_OK) return st;

  int ct_want = 64, cb_want = 32;
  int J = 0;
  bool kept_form = true;
  int64_t r = -1, m = 0;
  double shift = 0.0;
  int sel0 = 0;  // first column (in Wr / Xr) of the selected vectors
  RitzEnds E;
  while (J < kmax) {
    const int J1 = (int)std::min<int64_t>(kmax, J + KRY_CHECK);
    if ((st = lanczos_steps(ctx, B, d, 0, J, J1, B.alpha, B.beta, tiny, s)) != LRE_OK) return st;
    J = J1;
    int brk = 0;
    e = cudaMemcpyAsync(&brk, B.breakdown, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "Lanczos breakdown flag");
    const bool broke = brk > 0;
    if (broke) J = brk;  // an invariant subspace: T_J holds exact eigenvalues
    // windows of Ritz values at each end, together at most ct_max (the
    // buffers' width) and J
    const int CT = (int)std::min<int64_t>(std::min(ct_want, J), B.ct_max - 1);
    const int CB = (int)std::min<int64_t>(std::min(cb_want, J - CT), B.ct_max - CT);
    if ((st = ritz_ends(ctx, B, B.alpha, B.beta, J, CB, CT, s, E)) != LRE_OK) return st;
    const int mm = CB + CT;
    const double anorm = fmax(fabs(E.w[0]), fabs(E.w[mm - 1]));
    auto conv = [&](int k) { return fabs(E.beta_next * E.last[k]) <= KRY_RTOL * anorm; };
    // top end: l_k - (S_k - Tr)/k > 0 exactly for k <= r
    int64_t r_top = -1;
    bool top_open = true;
    double S = 0.0, S_r = 0.0;
    for (int k = 1; k <= CT; ++k) {
      const int col = mm - k;
      if (!conv(col)) {
        top_open = false;
        break;
      }
      S += E.w[col];
      if (E.w[col] - (S - trace) / k <= 0.0) {
        r_top = k - 1;
        break;
      }
      S_r = S;
    }
    // bottom end: Smolin's walk over the smallest eigenvalues
    int64_t r_bot = -1;
    bool bot_open = CB > 0;
    double a = 0.0;
    int64_t kept = d;
    for (int t = 0; t < CB && bot_open; ++t) {
      if (!conv(t)) {
        bot_open = false;
        break;
      }
      if (E.w[t] + a / (double)kept < 0.0) {
        a += E.w[t];
        --kept;
      } else {
        r_bot = kept;
        break;
      }
    }
    if (r_top >= 0 && r_bot >= 0 && r_top != r_bot) return LRE_OK;  // the two ends disagree: reduction path
    if (r_top >= 0 && r_top <= KRY_MAX_VECS) {
      kept_form = true;
      r = r_top;
      m = r;
      shift = (trace - S_r) / (double)r;
      sel0 = mm - (int)r;
    } else if (r_bot >= 0 && d - r_bot <= KRY_MAX_VECS && !eig_rho) {
      kept_form = false;
      r = r_bot;
      m = d - r;
      shift = r > 0 ? a / (double)r : 0.0;
      sel0 = 0;
    }
    if (r >= 0) break;
    if (r_top >= 0 || r_bot >= 0) return LRE_OK;  // decided, but too many vectors: reduction path
    if (broke) return LRE_OK;  // exact but undecided: reduction path
    // widen an end whose values all converged without deciding; when both
    // ends are at their widest and still undecided, both sets are too large
    const bool top_full = top_open && r_top < 0 && CT == ct_want;
    const bool bot_full = bot_open && r_bot < 0 && CB == cb_want;
    const int ct_cap = (int)(B.ct_max - 256), cb_cap = 256;
    if (top_full && bot_full && ct_want >= ct_cap && cb_want >= cb_cap) return LRE_OK;  // reduction path
    if (top_full) ct_want = std::min(2 * ct_want, ct_cap);
    if (bot_full) cb_want = std::min(2 * cb_want, cb_cap);
  }
  if (r < 0) return LRE_OK;  // undecided within the step limit: reduction path

  // the selected Ritz vectors (conjugated: eigenvectors of conj(mu)) and their values
  if (m > 0) {
    Launch L(ctx, "kry_ritz", s);
    dim3 g((unsigned)std::min<int64_t>((d + 255) / 256, (int64_t)ctx->num_sms * 4), (unsigned)((m + 7) / 8));
    kry_ritz<<<g, 256, 0, s>>>(B.Q, J, B.Xr + (int64_t)sel0 * J, (int)m, B.Z, d);
  }
  // certification: Lanczos on the operator deflated by the selected vectors
  // (seeded as the first basis rows) from a new start vector; the kept form
  // needs its largest Ritz value <= tau = -shift, the dropped form its
  // smallest >= tau
  const double tau = -shift;
  const double anorm = fmax(fabs(E.w.front()), fabs(E.w.back()));
  {
    if (m > 0) {
      Launch L(ctx, "kry_seed", s);
      kry_seed<<<grid, 256, 0, s>>>(B.Z, (int)m, B.Q, d);
    }
    if ((st = start_vector(ctx, B, d, m, 0x5EED0002ull, s)) != LRE_OK) return st;
    e = cudaMemsetAsync(B.breakdown, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "certification set-up");
    const int L2 = (int)std::min<int64_t>(KRY_VERIFY, d - m - 1);
    if (L2 >= 2) {
      if ((st = lanczos_steps(ctx, B, d, m, 0, L2, alpha2, beta2, tiny, s)) != LRE_OK) return st;
      int brk = 0;
      e = cudaMemcpyAsync(&brk, B.breakdown, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "certification breakdown flag");
      const int J2 = brk > 0 ? brk : L2;
      RitzEnds V;
      if ((st = ritz_ends(ctx, B, alpha2, beta2, J2, 1, 1, s, V)) != LRE_OK) return st;  // smallest, largest
      const double slack = 1e-10 * anorm;
      if (kept_form && V.w.back() > tau + slack) return LRE_OK;
      if (!kept_form && V.w.front() < tau - slack) return LRE_OK;
    }
  }
  // rebuild from the selected vectors
  SmolinResult hres{r, shift};
  e = cudaMemcpyAsync(B.res, &hres, sizeof(hres), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "projection threshold");
  // the selected Ritz values: Wr was overwritten by the certification, so
  // upload them (ascending, as the vectors)
  std::vector<double> wsel(E.w.begin() + sel0, E.w.begin() + sel0 + m);
  if (m > 0) {
    e = cudaMemcpyAsync(B.Wr, wsel.data(), m * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "selected eigenvalues");
  }
  *fallback = false;
  if ((st = rebuild_emit(ctx, blas, B.M, B.Z, B.Wr, d, m, kept_form, B.res, rho_out, s)) != LRE_OK) return st;
  if (eig_rho) {  // kept form only (the dropped form falls back when eig_rho is asked for)
    Launch L(ctx, "kry_eig_rho", s);
    kry_eig_rho<<<(int)((d + 255) / 256), 256, 0, s>>>(B.Wr, r, shift, eig_rho, d);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? LRE_OK : cuda_fail(ctx, e, "Krylov projection");
}

}  // namespace lre
