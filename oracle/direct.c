/*
 * Direct zero-dropped LRE sums -- TEST INFRASTRUCTURE ONLY (CPU oracle).
 *
 * Restates the algorithm of arXiv:1602.08604 Sec. III-IV in plain C:
 *
 * Step (i), Sec. III (Eqs. 2, 3) and Sec. IV: the 6^n Pauli eigenprojectors
 *   fall into 3^n groups (bases).  In the tensor-product Pauli representation
 *   (Eq. 5) every Gamma^(j) of a group has its 2^n nonzeros at the same 2^n
 *   locations -- the Pauli strings whose non-identity letters follow the
 *   group's axes -- and the nonzero values of the whole group form one
 *   2^n x 2^n "nonzero matrix", identical for every group.  For each group
 *   and each of its nonzero locations we take the dot product of that
 *   location's row of the nonzero matrix with the group's outcome counts and
 *   add it into the coefficient at that location.  X^T X is diagonal
 *   (Sec. III); its diagonal is accumulated from the same locations.
 *
 *   Scaling: with Gamma values 2^{-n/2}(+-1) and p_j = c_j / N_b,
 *     (sum_j p_j Gamma^(j))_i = 2^{-n/2} S_i / N     (uniform N)
 *     (X^T X)_ii             = sum_j Gamma_ij^2 = #groups containing i
 *   so theta_i = 2^{-n/2} S_i / (N diag_i) and the Pauli expectation
 *   estimate t_i = 2^{n/2} theta_i = S_i / (N diag_i).
 *
 * Step (ii), Eq. (4) and Sec. IV: mu = sum_i theta_i Omega_i, evaluated per
 *   output element from the 2^n Omega_i that are nonzero there (the group of
 *   strings with the same X/Y pattern x = row ^ col), each entry a product
 *   of single-qubit Pauli matrix entries.
 *
 * Index conventions: qubit 1 is the most significant digit of every index;
 * basis digits a in {0:X,1:Y,2:Z}; outcome bit 0 = +1 eigenvector; Pauli
 * digits p in {0:I,1:X,2:Y,3:Z}; counts are [3^n][2^n] row-major.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
  return omp_get_max_threads();
#else
  (void)t;
  return 1;
#endif
}

/* Pauli index of the location of group b with support mask m. */
static int64_t location_index(int n, int64_t b, uint32_t m) {
  int64_t i = 0, w = 1, bb = b;
  for (int j = 0; j < n; ++j) { /* j-th least significant qubit */
    int a = (int)(bb % 3);
    bb /= 3;
    int p = ((m >> j) & 1u) ? a + 1 : 0;
    i += (int64_t)p * w;
    w *= 4;
  }
  return i;
}

/* The shared 2^n x 2^n nonzero matrix: entry [m][o] is the product over
 * qubits of the single-qubit Gamma values (times 2^{n/2}): +1 on identity
 * sites, (-1)^{o_q} on measured sites. */
static int8_t *nonzero_matrix_build(int n) {
  size_t d = (size_t)1 << n;
  int8_t *H = (int8_t *)malloc(d * d);
  if (!H) return NULL;
  for (size_t m = 0; m < d; ++m)
    for (size_t o = 0; o < d; ++o) {
      int v = 1;
      for (int j = 0; j < n; ++j)
        if (((m >> j) & 1u) && ((o >> j) & 1u)) v = -v;
      H[m * d + o] = (int8_t)v;
    }
  return H;
}

/* The nonzero matrix is the same for every group (Sec. III): build it once
 * per n and keep it. */
static int8_t *H_cache = NULL;
static int H_cache_n = -1;
static int8_t *nonzero_matrix(int n) {
  int8_t *H = NULL;
#pragma omp critical(oracle_nonzero_matrix)
  {
    if (H_cache_n != n) {
      free(H_cache);
      H_cache = nonzero_matrix_build(n);
      H_cache_n = H_cache ? n : -1;
    }
    H = H_cache;
  }
  return H;
}

static inline int64_t count_at(const void *counts, int kind, size_t idx) {
  return kind == 1 ? (int64_t)((const int16_t *)counts)[idx]
                   : (int64_t)((const int32_t *)counts)[idx];
}

/* Integer sums S_i += sum_{groups b in [b0,b1)} (nonzero row . counts_b) and
 * diag_i += 1 per group containing location i.  kind: 0 int32, 1 int16.
 * counts points at row b0.  Returns 0, or -1 on allocation failure. */
int oracle_direct_sums(int n, const void *counts, int kind, int64_t b0, int64_t b1,
                       int64_t *S, int64_t *diag) {
  const size_t d = (size_t)1 << n;
  int8_t *H = nonzero_matrix(n);
  if (!H) return -1;
  const int64_t BLK = 16;
  for (int64_t bs = b0; bs < b1; bs += BLK) {
    int64_t be = bs + BLK < b1 ? bs + BLK : b1;
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < (int64_t)d; ++m) {
      const int8_t *h = H + (size_t)m * d;
      for (int64_t b = bs; b < be; ++b) {
        const size_t row = (size_t)(b - b0) * d;
        int64_t dot = 0;
        for (size_t o = 0; o < d; ++o) dot += (int64_t)h[o] * count_at(counts, kind, row + o);
        int64_t i = location_index(n, b, (uint32_t)m);
        S[i] += dot;
        if (diag) diag[i] += 1;
      }
    }
  }
  return 0;
}

/* Per-basis shot totals: acc_i += (nonzero row . counts_b) / N_b in FP64. */
int oracle_direct_weighted(int n, const void *counts, int kind, const int64_t *shots,
                           int64_t b0, int64_t b1, double *acc, int64_t *diag) {
  const size_t d = (size_t)1 << n;
  int8_t *H = nonzero_matrix(n);
  if (!H) return -1;
  const int64_t BLK = 16;
  for (int64_t bs = b0; bs < b1; bs += BLK) {
    int64_t be = bs + BLK < b1 ? bs + BLK : b1;
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < (int64_t)d; ++m) {
      const int8_t *h = H + (size_t)m * d;
      for (int64_t b = bs; b < be; ++b) {
        const size_t row = (size_t)(b - b0) * d;
        int64_t dot = 0;
        for (size_t o = 0; o < d; ++o) dot += (int64_t)h[o] * count_at(counts, kind, row + o);
        int64_t i = location_index(n, b, (uint32_t)m);
        acc[i] += (double)dot / (double)shots[b];
        if (diag) diag[i] += 1;
      }
    }
  }
  return 0;
}

/* t_i = S_i / (N diag_i): one FP64 division of exact integers. */
void oracle_theta_uniform(int n, const int64_t *S, const int64_t *diag, int64_t shots, double *t) {
  const int64_t P = (int64_t)1 << (2 * n);
  for (int64_t i = 0; i < P; ++i) t[i] = (double)S[i] / ((double)shots * (double)diag[i]);
}

void oracle_theta_weighted(int n, const double *acc, const int64_t *diag, double *t) {
  const int64_t P = (int64_t)1 << (2 * n);
  for (int64_t i = 0; i < P; ++i) t[i] = acc[i] / (double)diag[i];
}

/* Single-qubit Pauli matrix entries sigma_p[r][c] as (re, im). */
static const double SIG_RE[4][2][2] = {{{1, 0}, {0, 1}}, {{0, 1}, {1, 0}}, {{0, 0}, {0, 0}}, {{1, 0}, {0, -1}}};
static const double SIG_IM[4][2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}, {{0, -1}, {1, 0}}, {{0, 0}, {0, 0}}};

/* mu[r][c] = 2^{-n} sum_{P in group(r^c)} t_P P[r][c] for the listed
 * elements (step ii per element, Sec. IV). */
void oracle_direct_mu_elements(int n, const double *t, const int64_t *rows, const int64_t *cols,
                               int64_t count, double *out_re, double *out_im) {
  const int64_t d = (int64_t)1 << n;
  const double scale = 1.0 / (double)d;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t e = 0; e < count; ++e) {
    const int64_t r = rows[e], c = cols[e], x = r ^ c;
    double sr = 0.0, si = 0.0;
    for (int64_t z = 0; z < d; ++z) {
      /* member of the group: p_j in {X,Y} where x_j = 1, in {I,Z} where 0 */
      int64_t i = 0, w = 1;
      double er = 1.0, ei = 0.0;
      for (int j = 0; j < n; ++j) {
        int xj = (int)((x >> j) & 1), zj = (int)((z >> j) & 1);
        int p = xj ? (zj ? 2 : 1) : (zj ? 3 : 0);
        int rj = (int)((r >> j) & 1), cj = (int)((c >> j) & 1);
        double ar = SIG_RE[p][rj][cj], ai = SIG_IM[p][rj][cj];
        double nr = er * ar - ei * ai, ni = er * ai + ei * ar;
        er = nr;
        ei = ni;
        i += (int64_t)p * w;
        w *= 4;
      }
      sr += t[i] * er;
      si += t[i] * ei;
    }
    out_re[e] = sr * scale;
    out_im[e] = si * scale;
  }
}

/* Full mu (d x d, row-major re/im planes) by the per-group direct sum. */
void oracle_direct_mu(int n, const double *t, double *mu_re, double *mu_im) {
  const int64_t d = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < d; ++r) {
    const double scale = 1.0 / (double)d;
    for (int64_t c = 0; c < d; ++c) {
      const int64_t x = r ^ c;
      double sr = 0.0, si = 0.0;
      for (int64_t z = 0; z < d; ++z) {
        int64_t i = 0, w = 1;
        double er = 1.0, ei = 0.0;
        for (int j = 0; j < n; ++j) {
          int xj = (int)((x >> j) & 1), zj = (int)((z >> j) & 1);
          int p = xj ? (zj ? 2 : 1) : (zj ? 3 : 0);
          int rj = (int)((r >> j) & 1), cj = (int)((c >> j) & 1);
          double ar = SIG_RE[p][rj][cj], ai = SIG_IM[p][rj][cj];
          double nr = er * ar - ei * ai, ni = er * ai + ei * ar;
          er = nr;
          ei = ni;
          i += (int64_t)p * w;
          w *= 4;
        }
        sr += t[i] * er;
        si += t[i] * ei;
      }
      mu_re[r * d + c] = sr * scale;
      mu_im[r * d + c] = si * scale;
    }
  }
}

/* Spot values of step (i) for chosen Pauli indices (large-n parity checks):
 * S_i = sum over the 3^k groups whose locations include i of the nonzero-
 * matrix row of i times the group's counts.  `row_of(b)` rows are supplied by
 * the caller as `counts` with a row table: rows[k] is the row (in counts) of
 * the k-th compatible group of entry e, enumerated in increasing basis index.
 * Here the caller passes, per entry, its compatible groups' counts
 * contiguously: counts_e = counts + offsets[e] * 2^n, 3^k rows.  kind: 0 int32,
 * 1 int16. */
void oracle_direct_entries(int n, const void *counts, int kind, const int64_t *indices,
                           const int64_t *offsets, int64_t count, int64_t *S) {
  const int64_t d = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t e = 0; e < count; ++e) {
    const int64_t i = indices[e];
    uint32_t m = 0;
    int k = 0;
    for (int j = 0; j < n; ++j) {
      if (((i >> (2 * j)) & 3) != 0) m |= 1u << j;
      else ++k;
    }
    int64_t groups = 1;
    for (int j = 0; j < k; ++j) groups *= 3;
    int64_t acc = 0;
    for (int64_t g = 0; g < groups; ++g) {
      const size_t row = (size_t)(offsets[e] + g) * (size_t)d;
      for (int64_t o = 0; o < d; ++o) {
        int v = 1;
        for (int j = 0; j < n; ++j)
          if (((m >> j) & 1u) && ((o >> j) & 1)) v = -v;
        acc += (int64_t)v * count_at(counts, kind, row + (size_t)o);
      }
    }
    S[e] = acc;
  }
}
