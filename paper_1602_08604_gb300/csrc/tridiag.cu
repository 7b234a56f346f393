// Symmetric tridiagonal eigenproblem kernels for the eigenvalue-first
// projection (step (iii), Sec. II): after the Hermitian matrix has been
// reduced to a real tridiagonal T (diagonal a, off-diagonal b), every
// eigenvalue comes from bisection on Sturm counts, and eigenvectors are
// computed only for the eigenvalues the projection needs, by inverse
// iteration with re-orthogonalisation inside clusters of close eigenvalues
// (the classical scheme of Wilkinson and Peters; see also Demmel, Applied
// Numerical Linear Algebra, Sec. 5.3).  Everything is FP64.
#include <cuda_runtime.h>

#include <cfloat>

#include "lre_internal.cuh"

namespace lre {

namespace {

// Number of eigenvalues of T strictly below x (Sylvester's law of inertia on
// the LDL^T factorisation of T - xI).  A pivot smaller than pivmin in
// magnitude is replaced by -pivmin, which keeps the count consistent.
__device__ __forceinline__ int64_t sturm_count(const double *a, const double *b2, int64_t n, double x,
                                               double pivmin) {
  double q = a[0] - x;
  int64_t neg = 0;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++neg;
  for (int64_t k = 1; k < n; ++k) {
    q = (a[k] - x) - b2[k - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++neg;
  }
  return neg;
}

}  // namespace

// W[j - j0] = the j-th smallest eigenvalue for j in [j0, j0 + cnt), one
// thread per eigenvalue; [lo, hi) brackets every eigenvalue (Gershgorin),
// tol is the absolute accuracy asked for.
__global__ void tri_bisect_kernel(const double *a, const double *b2, int64_t n, double lo0, double hi0, double tol,
                                  double pivmin, double *W, int64_t j0, int64_t cnt) {
  for (int64_t jj = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; jj < cnt; jj += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = j0 + jj;
    double lo = lo0, hi = hi0;  // invariant: count(lo) <= j < count(hi)
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (hi - lo <= tol || mid <= lo || mid >= hi) break;
      if (sturm_count(a, b2, n, mid, pivmin) <= j)
        lo = mid;
      else
        hi = mid;
    }
    W[jj] = 0.5 * (lo + hi);
  }
}

// The same eigenvalues by multisection, one warp per eigenvalue: each round
// the 32 lanes split the bracket into 32 parts and evaluate the Sturm count at
// the 31 inner points, so the bracket shrinks 32-fold per round (about 12
// rounds to 4 eps ||T||) instead of 2-fold; for the few extreme eigenvalues a
// Krylov check needs, which bisection would run on a handful of threads.
// Warps beyond j0 + cnt idle; blockDim a multiple of 32.
__global__ void tri_multisect_kernel(const double *a, const double *b2, int64_t n, double lo0, double hi0, double tol,
                                     double pivmin, double *W, int64_t j0, int64_t cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t jj = wid; jj < cnt; jj += nw) {
    const int64_t j = j0 + jj;
    double lo = lo0, hi = hi0;  // invariant: count(lo) <= j < count(hi)
    for (int it = 0; it < 40; ++it) {
      if (hi - lo <= tol) break;
      const double step = (hi - lo) / 32.0;
      const double x = lo + step * (double)(lane + 1);  // lane 31: x = hi (not evaluated)
      const bool below = lane < 31 && x > lo && x < hi && sturm_count(a, b2, n, x, pivmin) <= j;
      // the points where count <= j form a prefix: the new lo is the last of them
      const unsigned m = __ballot_sync(0xffffffffu, below);
      const int k = m ? 31 - __clz(m) : -1;  // last lane with count(x) <= j
      const double nlo = k >= 0 ? lo + step * (double)(k + 1) : lo;
      const double nhi = k + 1 <= 30 ? lo + step * (double)(k + 2) : hi;
      if (!(nhi < hi || nlo > lo)) break;  // no progress (rounding): the bracket is as tight as it gets
      lo = nlo;
      hi = nhi;
    }
    if (lane == 0) W[jj] = 0.5 * (lo + hi);
  }
}

namespace {

__device__ __forceinline__ double start_entry(int64_t i, int64_t j) {
  // splitmix64 of (i, j) -> uniform in [-1, 1): a fixed, well-spread start vector
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + (uint64_t)j * 0xD1B54A32D192ED03ull + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

template <int THREADS>
__device__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < THREADS / 32; ++k) s += red[k];
  return s;
}

}  // namespace

// Inverse iteration for the selected eigenvalues lam[0..m) (ascending), all
// members at once: tri_factor factors T - lam_j I = P L U for every j
// (Gaussian elimination with partial pivoting, one thread per member; U has
// two super-diagonals, its pivots stored as reciprocals so that the solves
// need no division), then TRI_ROUNDS rounds of tri_solve (every column of X
// through its own factors, in parallel) and tri_orthonormalise (one CTA per
// cluster of close eigenvalues: modified Gram-Schmidt in eigenvalue order,
// then unit norm).  X: column-major [n][m]; lu: 5 n doubles per member.
static_assert(TRI_ROUNDS >= 2, "at least two inverse-iteration rounds");

__global__ void tri_factor(const double *a, const double *b, int64_t n, const double *lam, int m, double tnorm,
                           double *lu) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const double x = lam[j];
  double *ui = lu + (size_t)j * 5 * n;  // 1 / U diagonal
  double *u1 = ui + n;                  // U first super-diagonal
  double *u2 = u1 + n;                  // U second super-diagonal
  double *mul = u2 + n;                 // multipliers (row k+1 -= mul[k] * pivot row k)
  double *swp = mul + n;                // 1.0 where rows k, k+1 were exchanged
  const double small = DBL_EPSILON * tnorm > DBL_MIN ? DBL_EPSILON * tnorm : DBL_MIN;
  // the pending row holds (p, q) at columns k, k+1 (its column k+2 entry is zero)
  double p = a[0] - x, q = n > 1 ? b[0] : 0.0;
  for (int64_t k = 0; k + 1 < n; ++k) {
    const double lo = b[k];                          // row k+1, column k
    const double dk = a[k + 1] - x;                  // row k+1, column k+1
    const double up = (k + 2 < n) ? b[k + 1] : 0.0;  // row k+1, column k+2
    if (fabs(lo) > fabs(p)) {
      const double r = 1.0 / lo;
      ui[k] = r; u1[k] = dk; u2[k] = up; swp[k] = 1.0;
      const double f = p * r;
      mul[k] = f;
      p = q - f * dk;
      q = -f * up;
    } else {
      if (fabs(p) < small) p = small;
      const double r = 1.0 / p;
      ui[k] = r; u1[k] = q; u2[k] = 0.0; swp[k] = 0.0;
      const double f = lo * r;
      mul[k] = f;
      p = dk - f * q;
      q = up;
    }
  }
  if (fabs(p) < small) p = small;
  ui[n - 1] = 1.0 / p; u1[n - 1] = 0.0; u2[n - 1] = 0.0;
}

__global__ void tri_solve(const double *lu, int64_t n, int m, double *X, int first) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const double *ui = lu + (size_t)j * 5 * n, *u1 = ui + n, *u2 = u1 + n, *mul = u2 + n, *swp = mul + n;
  double *v = X + (size_t)j * n;
  // forward: row exchanges and multipliers; the pending right-hand side stays
  // in a register (the start vector is generated on the fly in round one)
  double pend = first ? start_entry(0, j) : v[0];
  for (int64_t k = 0; k + 1 < n; ++k) {
    const double nxt = first ? start_entry(k + 1, j) : v[k + 1];
    if (swp[k] != 0.0) {
      v[k] = nxt;
      pend = pend - mul[k] * nxt;
    } else {
      v[k] = pend;
      pend = nxt - mul[k] * pend;
    }
  }
  v[n - 1] = pend;
  // back substitution with U
  double x1 = 0.0, x2 = 0.0;
  for (int64_t k = n - 1; k >= 0; --k) {
    const double xk = (v[k] - u1[k] * x1 - u2[k] * x2) * ui[k];
    v[k] = xk;
    x2 = x1;
    x1 = xk;
  }
}

__global__ void __launch_bounds__(TRI_THREADS) tri_orthonormalise(double *X, int64_t n, const int *cl) {
  __shared__ double red[TRI_THREADS / 32];
  const int j0 = cl[blockIdx.x], j1 = cl[blockIdx.x + 1];
  for (int j = j0; j < j1; ++j) {
    double *v = X + (size_t)j * n;
    for (int pass = 0; pass < 2; ++pass) {
      // pass 0: unit norm first (a solve grows the vector by up to 1/eps);
      // pass 1: Gram-Schmidt against the cluster's earlier vectors, unit norm
      if (pass == 1) {
        for (int k = j0; k < j; ++k) {
          const double *w = X + (size_t)k * n;
          double dot = 0.0;
          for (int64_t i = threadIdx.x; i < n; i += blockDim.x) dot += w[i] * v[i];
          dot = block_sum<TRI_THREADS>(dot, red);
          for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v[i] -= dot * w[i];
          __syncthreads();
        }
      }
      double nrm = 0.0;
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) nrm += v[i] * v[i];
      nrm = block_sum<TRI_THREADS>(nrm, red);
      const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v[i] *= inv;
      __syncthreads();
    }
  }
}

// Cluster boundaries of the ascending selection lam[0..m): a new cluster
// starts where the gap to the previous eigenvalue exceeds gap_tol.  cl[0..k]
// (k clusters, cl[k] = m), *k_out = k.  One thread.
__global__ void tri_clusters(const double *lam, int m, double gap_tol, int *cl, int *k_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int k = 0;
  cl[0] = 0;
  for (int j = 1; j < m; ++j)
    if (lam[j] - lam[j - 1] > gap_tol) cl[++k] = j;
  cl[++k] = m;
  *k_out = k;
}

}  // namespace lre
