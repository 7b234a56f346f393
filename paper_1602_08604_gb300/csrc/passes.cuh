// Per-item bodies of the register-level passes of steps (i) and (ii), shared
// by the standalone pass kernels (fold.cu, assemble.cu) and the batched
// persistent kernel (batch.cu).
//
// Step (i) (Sec. III, Eq. 3): a pass contracts J qubits of the view
//   X[ah][al][oh][ol][c] -> Y[ah][oh][pl][c]   (al in 3^J, ol in 2^J, pl in 4^J)
// with the per-qubit map T (2-point WHT over the outcome bit, then I = sum
// of the three axes, X/Y/Z = the matching axis); the last pass divides by
// N 3^k (k identity letters) and can also emit T_i = S_i 3^(n-k).
// Step (ii) (Eq. 4): a pass applies the per-qubit map (I,X,Y,Z) ->
// (I+Z, X-iY, X+iY, I-Z) (times 1/2 in FP64; unscaled on exact integers) to
// J qubits of [P_hi][R_lo][C_lo].
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "lre_internal.cuh"

namespace lre {
namespace passes {

// T_I24P: int32 values stored as split planes, the low 16 bits (uint16) then
// the bits above (int8), for partials below 2^23 in magnitude
enum { T_I16 = 0, T_I32 = 1, T_I64 = 2, T_F64 = 3, T_I24P = 4 };
enum { M_STORE = 0, M_FINAL_U = 1, M_FINAL_W = 2, M_PARITY = 3 };

// Pauli-digit index of a pass block: digit q is m_q ? a_q + 1 : 0 (a_q the
// q-th ternary digit of al, m_q the q-th bit of the parity mask).
__host__ __device__ constexpr int block_pauli(int al, int m, int J) {
  int pl = 0, w = 1;
  for (int q = 0; q < J; ++q) {
    pl += (((m >> q) & 1) ? (al % 3) + 1 : 0) * w;
    al /= 3;
    w *= 4;
  }
  return pl;
}

template <int J, typename V>
__device__ __forceinline__ void wht(V (&v)[1 << J]) {
#pragma unroll
  for (int h = 1; h < (1 << J); h <<= 1) {
#pragma unroll
    for (int i = 0; i < (1 << J); ++i) {
      if ((i & h) == 0) {
        V a = v[i], b = v[i + h];
        v[i] = a + b;
        v[i + h] = a - b;
      }
    }
  }
}

__device__ __forceinline__ int identity_letters(uint64_t i, int n) {
  uint64_t nz = (i | (i >> 1)) & 0x5555555555555555ull;
  uint64_t mask = (n >= 32) ? ~0ull : ((1ull << (2 * n)) - 1);
  return n - __popcll(nz & mask);
}

// a / b correctly rounded, from y = RN(1/b): q = RN(a y) is within one ulp of
// a/b, the residual a - b q is exact under FMA, and one more FMA gives the
// correctly rounded quotient (Markstein; Muller et al., Handbook of
// Floating-Point Arithmetic, the FMA-based division correction theorem).
__device__ __forceinline__ double div_by_recip(double a, double b, double y) {
  const double q = a * y;
  const double r = fma(-q, b, a);
  return fma(r, y, q);
}

// RN(S / d) for integers |S| < 2^53 and 0 < d < 2^53, with y = RN(1/d), using
// one FP64 multiply and integer arithmetic (GB300's FP64 pipe is narrow; the
// Markstein form above costs a conversion and three FP64 operations).
//   1. The exponent e of the quotient (a/d in [2^e, 2^(e+1)), a = |S|) comes
//      from the leading bits of a and d; with s = 53 - e the integer
//      quotient Q = floor(a 2^s / d) lies in [2^53, 2^54).
//   2. q0 = RN(a y) has relative error below 2^-52, so q0 2^s (an integer)
//      is within 5 of Q; the exact remainder R = a 2^s - Q d (|R| < 2^56,
//      so its low 64 bits suffice) corrects it to floor, 0 <= R < d.
//   3. The mantissa is Q >> 1 rounded to nearest even from the guard bit
//      Q & 1 and the sticky R != 0; the result is that mantissa times 2^e.
// A quotient of |S| >= 2^53 (not exact as a double anyway) takes the FP64 form.
// ld = the leading-bit position of d, dn = d << (63 - ld) (precomputed per divisor).
__device__ __forceinline__ double div_int_rn(int64_t S, int64_t D, double y, int ld, uint64_t dn) {
  if (S == 0) return 0.0;
  const uint64_t a = S < 0 ? (uint64_t)(-S) : (uint64_t)S;
  if (a >= (1ull << 53)) return div_by_recip((double)S, (double)D, y);
  const uint64_t d = (uint64_t)D;
  const int la = 63 - __clzll((long long)a);
  const int e = la - ld - (((a << (63 - la)) < dn) ? 1 : 0);
  const int s = 53 - e;  // in [1, 106]: a/d >= 2^-53 and <= 2^53
  // a as a double, exactly (a < 2^53), built from its bits
  const double ad = __longlong_as_double((long long)(((uint64_t)(1023 + la) << 52) |
                                                     ((a << (52 - la)) & 0xFFFFFFFFFFFFFull)));
  const uint64_t qb = (uint64_t)__double_as_longlong(ad * y);
  const int sh = (int)((qb >> 52) & 0x7FF) - 1023 - e + 1;  // q0 2^s = mantissa << sh, sh in {0, 1, 2}
  uint64_t Q = ((qb & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << (sh > 0 ? sh : 0);
  if (sh < 0) Q >>= -sh;
  // |R| < 6 d < 2^56, so R is the low 64 bits of a 2^s - Q d read as signed
  int64_t R = (int64_t)((s < 64 ? a << s : 0ull) - Q * d);
#pragma unroll 1
  for (int it = 0; it < 16 && R < 0; ++it) {
    --Q;
    R += (int64_t)d;
  }
#pragma unroll 1
  for (int it = 0; it < 16 && R >= (int64_t)d; ++it) {
    ++Q;
    R -= (int64_t)d;
  }
  uint64_t m = Q >> 1;
  int ee = e;
  if ((Q & 1) && (R != 0 || (m & 1))) {
    if (++m == (1ull << 53)) {
      m = 1ull << 52;
      ++ee;
    }
  }
  const uint64_t bits = ((uint64_t)(S < 0) << 63) | ((uint64_t)(ee + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double div_int_rn(int64_t S, int64_t D, double y) {
  const int ld = 63 - __clzll(D);
  return div_int_rn(S, D, y, ld, (uint64_t)D << (63 - ld));
}

struct GenParams {
  const void *in;
  void *out;
  int64_t C;       // columns already produced (4^(n-r))
  int64_t n_oh;    // 2^(r-J)
  int64_t items;   // 3^(r-J) * 2^(r-J) * C
  int r;           // qubits left before this pass
  int n;
  const double *wgt;     // 1/N_b per basis (weighted first pass)
  double shots;          // N (final uniform)
  int64_t total;         // N * 3^n (final uniform check)
  int *status;
  int64_t *T;            // optional: exact integers S_i 3^(n-k) for the integer assembly
  double denom[16];      // N 3^k (uniform) or 3^k (weighted), exact
  int64_t dint[16];      // N 3^k as an integer (uniform shots)
  double recip[16];      // correctly rounded 1 / denom[k]
  int64_t up3[16];       // 3^(n-k)
  int hi_from = 0;       // split-plane input: see planes_hi_needed
  int hi_letters = 6;    // split-plane input: qubits the first pass folded (6 or 7)
  int top7 = 0;          // last pass: letter 6 of the columns is qubit n's (seven-qubit first pass)
};

// Split-plane partials of the tensor-core first pass: the partial of a letter
// with k identities among its six (or seven) qubits is at most shots 3^k in
// magnitude (each basis row sums to the shots), so its high plane (bits
// 16..23) is needed only from k = hi_from on, the least k with shots 3^k >
// 32767; below that the low 16 bits, read as int16, are the value.  Letters
// are numbered (p7 * 64 +) plB * 64 + plA (2 bits a qubit, 0 = I; p7 only
// for the seven-qubit pass) and a run of 32 from c0 (a multiple of 32) fixes
// every letter above plA and the top bit of plA's third letter: its most
// identities are those of the fixed letters plus 3 (lower half, that letter
// I or X) or 2 (upper half, Y or Z).  The high plane of such a run is
// written only when one of its letters can need it, and read as values only
// then (the reader loads every run's bytes: whole L2 lines stream faster).
__host__ __device__ inline int planes_hi_from(int64_t shots) {
  int k = 0;
  for (int64_t b = shots; k < 8 && b <= 32767; ++k) b *= 3;
  return k;
}
__host__ __device__ inline bool planes_hi_needed(int64_t c0, int hi_from, int letters = 6) {
  int idc = 0;
  for (int q = 3; q < letters; ++q) idc += ((c0 >> (2 * q)) & 3) == 0;
  const int half = (int)((c0 >> 5) & 1);
  return idc + (half ? 2 : 3) >= hi_from;
}

// Loads of pass inputs: the read-only path, or (COHERENT) straight from L2 for
// inputs written earlier by the same kernel launch (the batched kernel).
template <bool COHERENT, typename T>
__device__ __forceinline__ T ld_in(const T *p) {
  if constexpr (COHERENT) return __ldcg(p);
  else return __ldg(p);
}

// The 2^J contiguous counts of one basis row (first pass, C == 1) as vector
// loads on the read-only path (counts are never written by the kernels).
template <int NO, typename InT, typename V>
__device__ __forceinline__ void ld_row_vec(const InT *p, V (&v)[NO]) {
  constexpr int BYTES = NO * (int)sizeof(InT);
  if constexpr (BYTES == 32) {
    const int4 a = __ldg(reinterpret_cast<const int4 *>(p));
    const int4 b = __ldg(reinterpret_cast<const int4 *>(p) + 1);
    const int w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < NO; ++k) v[k] = (V)w[k];
  } else {
    uint32_t w[4];
    if constexpr (BYTES == 16) {
      const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
      w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    } else if constexpr (BYTES == 8) {
      const uint2 a = __ldg(reinterpret_cast<const uint2 *>(p));
      w[0] = a.x; w[1] = a.y;
    } else {
      w[0] = __ldg(reinterpret_cast<const uint32_t *>(p));
    }
#pragma unroll
    for (int k = 0; k < NO; ++k) {
      if constexpr (sizeof(InT) == 2)
        v[k] = (V)(int16_t)(uint16_t)(w[k >> 1] >> (16 * (k & 1)));
      else
        v[k] = (V)(int32_t)w[k];
    }
  }
}

// Per-k divisor tables of a final pass in shared memory: the lanes of a warp
// index them with different k, which the kernel-parameter space would serve
// one distinct address at a time.
struct DivTables {
  double denom[16];
  double recip[16];
  int64_t dint[16];
  int64_t up3[16];
  uint64_t dn[16];  // dint normalised to bit 63
  int ld[16];       // leading-bit position of dint
};

__device__ __forceinline__ void load_div_tables(const GenParams &P, DivTables &t) {
  if (threadIdx.x < 16) {
    const int k = threadIdx.x;
    t.denom[k] = P.denom[k];
    t.recip[k] = P.recip[k];
    t.dint[k] = P.dint[k];
    t.up3[k] = P.up3[k];
    const int64_t d = P.dint[k] > 0 ? P.dint[k] : 1;
    t.ld[k] = 63 - __clzll(d);
    t.dn[k] = (uint64_t)d << (63 - t.ld[k]);
  }
}

// Writes the NP outputs of one column (ahoh, c) of a fold pass: partial sums
// (M_STORE), exact parity sums (M_PARITY), or theta = S / (N 3^k) (uniform
// shots, with the exact T_i = S_i 3^(n-k) when requested) / the weighted sum
// / 3^k (M_FINAL_W).  tab: the divisor tables in shared memory, or nullptr to
// read them from P.
// Index in theta of column i of the last pass (pl * C + c): unchanged, or
// with the seven-qubit first pass (top7) qubit n's letter moved from letter 6
// of c to the top and the letters above it (qubits 7..n-1) one down.  Runs of
// 4096 consecutive columns stay consecutive.
__device__ __forceinline__ int64_t theta_index(const GenParams &P, int64_t i) {
  if (!P.top7) return i;
  return (((i >> 12) & 3) << (2 * (P.n - 1))) | ((i >> 14) << 12) | (i & 4095);
}

template <int J, typename AccT, int MODE>
__device__ __forceinline__ void fold_emit(const GenParams &P, const AccT (&acc)[1 << (2 * J)], int64_t ahoh,
                                          int64_t c, const DivTables *tab = nullptr) {
  constexpr int NP = 1 << (2 * J);
  const int64_t obase = ahoh * NP * P.C + c;
  if constexpr (MODE == M_STORE) {
    AccT *out = static_cast<AccT *>(P.out);
#pragma unroll
    for (int p = 0; p < NP; ++p) out[obase + p * P.C] = acc[p];
  } else if constexpr (MODE == M_PARITY) {
    int64_t *out = static_cast<int64_t *>(P.out);
#pragma unroll
    for (int p = 0; p < NP; ++p) out[theta_index(P, obase + p * P.C)] = (int64_t)acc[p];
  } else {
    double *out = static_cast<double *>(P.out);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int64_t i = theta_index(P, obase + p * P.C);  // ahoh == 0 in the last pass
      const int k = identity_letters((uint64_t)i, P.n);
      if constexpr (MODE == M_FINAL_U) {
        if (i == 0 && (int64_t)acc[p] != P.total) latch(P.status, LRE_ERR_SHOTS_MISMATCH);
        if (tab) {
          // every third output takes the FP64 form, the rest the integer form:
          // both are correctly rounded (identical results), and the split keeps
          // the FP64 pipe and the integer ALUs busy at the same time
          if (p % 3 == 0)
            out[i] = div_by_recip((double)acc[p], tab->denom[k], tab->recip[k]);
          else
            out[i] = div_int_rn((int64_t)acc[p], tab->dint[k], tab->recip[k], tab->ld[k], tab->dn[k]);
          if (P.T) P.T[i] = (int64_t)acc[p] * tab->up3[k];
        } else {
          out[i] = div_int_rn((int64_t)acc[p], P.dint[k], P.recip[k]);
          if (P.T) P.T[i] = (int64_t)acc[p] * P.up3[k];
        }
      } else {
        out[i] = div_by_recip((double)acc[p], P.denom[k], P.recip[k]);
      }
    }
  }
}

// One output column (ah, oh, c) of a fold pass.  VEC: first pass (C == 1),
// the row's 2^J outcomes loaded as one vector.
template <int J, typename InT, typename AccT, int MODE, bool WEIGHT, bool COHERENT = false, bool VEC = false>
__device__ __forceinline__ void fold_item(const GenParams &P, int64_t item, const DivTables *tab = nullptr) {
  constexpr int NA = (J == 1) ? 3 : (J == 2) ? 9 : 27;
  constexpr int NO = 1 << J;
  constexpr int NP = 1 << (2 * J);
  const InT *__restrict__ in = static_cast<const InT *>(P.in);
  const int64_t row_stride = (1ll << P.r) * P.C;  // al stride
  const int64_t c = item % P.C;
  const int64_t ahoh = item / P.C;
  const int64_t oh = ahoh % P.n_oh;
  const int64_t ah = ahoh / P.n_oh;
  const int64_t base = ((ah * NA) << P.r) * P.C + (oh * NO) * P.C + c;
  AccT acc[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) acc[p] = 0;
#pragma unroll
  for (int al = 0; al < NA; ++al) {
    if constexpr (WEIGHT) {
      int32_t v[NO];
#pragma unroll
      for (int ol = 0; ol < NO; ++ol) v[ol] = (int32_t)ld_in<COHERENT>(in + base + al * row_stride + ol * P.C);
      wht<J>(v);
      const double w = __ldg(P.wgt + ah * NA + al);
#pragma unroll
      for (int m = 0; m < NO; ++m) acc[block_pauli(al, m, J)] += (double)v[m] * w;
    } else {
      AccT v[NO];
      if constexpr (VEC) {
        ld_row_vec<NO>(in + base + al * row_stride, v);
      } else {
#pragma unroll
        for (int ol = 0; ol < NO; ++ol) v[ol] = (AccT)ld_in<COHERENT>(in + base + al * row_stride + ol * P.C);
      }
      wht<J>(v);
#pragma unroll
      for (int m = 0; m < NO; ++m) acc[block_pauli(al, m, J)] += v[m];
    }
  }
  fold_emit<J, AccT, MODE>(P, acc, ahoh, c, tab);
}

// TMA-staged generic fold pass (fold_tma.cu) for int32 inputs with C a
// multiple of 32; LRE_ERR_UNSUPPORTED (nothing launched) for other passes.
lre_status tma_pass(lre_ctx *ctx, const GenParams &P, int J, int in_t, int acc_t, int mode, bool weight,
                    cudaStream_t s);

// ---- step (ii) ----------------------------------------------------------------
struct NumF64 {
  using V = double2;
  using In = double;
};
struct NumI64 {
  using V = longlong2;
  using In = long long;
};

struct LastScale {
  float sh, sl;  // 1/(2^n N 3^n) = sh + sl (integer path only)
};

__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ longlong2 mk(long long a, long long b) { return make_longlong2(a, b); }

// One qubit of the butterfly on (I, X, Y, Z) -> (00, 01, 10, 11).
//   -i*Y = (Y.y, -Y.x);  +i*Y = (-Y.y, Y.x)
__device__ __forceinline__ void m_qubit(double2 vI, double2 vX, double2 vY, double2 vZ, double2 &o00,
                                        double2 &o01, double2 &o10, double2 &o11) {
  o00 = mk(0.5 * (vI.x + vZ.x), 0.5 * (vI.y + vZ.y));
  o11 = mk(0.5 * (vI.x - vZ.x), 0.5 * (vI.y - vZ.y));
  o01 = mk(0.5 * (vX.x + vY.y), 0.5 * (vX.y - vY.x));
  o10 = mk(0.5 * (vX.x - vY.y), 0.5 * (vX.y + vY.x));
}
__device__ __forceinline__ void m_qubit(longlong2 vI, longlong2 vX, longlong2 vY, longlong2 vZ,
                                        longlong2 &o00, longlong2 &o01, longlong2 &o10, longlong2 &o11) {
  o00 = mk(vI.x + vZ.x, vI.y + vZ.y);
  o11 = mk(vI.x - vZ.x, vI.y - vZ.y);
  o01 = mk(vX.x + vY.y, vX.y - vY.x);
  o10 = mk(vX.x - vY.y, vX.y + vY.x);
}

__device__ __forceinline__ double2 load_first(const double *in, int64_t i) { return mk(__ldcg(in + i), 0.0); }
__device__ __forceinline__ longlong2 load_first(const long long *in, int64_t i) {
  return mk(__ldcg(in + i), 0ll);
}

// int64 -> float of v * (sh + sl), error about half an ulp of the float.
// 64-bit integer conversions run at the FP64 rate, so v is split as
// a 2^46 + b 2^23 + c with 0 <= b, c < 2^23 and |a| < 2^17; each part becomes
// a float exactly by placing it in the mantissa of 2^23 (or 1.5 * 2^23 for
// the signed a) and subtracting that constant.  X = a 2^46 + b 2^23 is exact
// while |v| < 2^46 (a is 0 or -1) and rounded once above; Knuth's TwoSum then
// gives vh = RN(X + c) and the exact remainder vl, and the product with the
// two-float scale is formed with one final rounding.
__device__ __forceinline__ float scaled(long long v, const LastScale &s) {
  const int a = (int)(v >> 46);
  const unsigned b = (unsigned)(v >> 23) & 0x7FFFFFu, c = (unsigned)v & 0x7FFFFFu;
  const float fa = __int_as_float(0x4B400000 + a) - 12582912.f;
  const float fb = __int_as_float(0x4B000000 | b) - 8388608.f;
  const float fc = __int_as_float(0x4B000000 | c) - 8388608.f;
  const float X = __fmaf_rn(fa, 70368744177664.f, fb * 8388608.f);  // 2^46, 2^23
  const float vh = __fadd_rn(X, fc);
  const float bv = __fsub_rn(vh, X);
  const float vl = __fadd_rn(__fsub_rn(X, __fsub_rn(vh, bv)), __fsub_rn(fc, bv));
  return __fmaf_rn(vh, s.sh, __fmaf_rn(vh, s.sl, vl * s.sh));
}
__device__ __forceinline__ float2 to_c64(double2 v, const LastScale &) {
  return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ float2 to_c64(longlong2 v, const LastScale &s) {
  return make_float2(scaled(v.x, s), scaled(v.y, s));
}

struct AsmParams {
  const void *in;
  void *out;
  int t;          // qubits already transformed
  int n;
  int64_t items;  // 4^(n-t-J) * 4^t
  LastScale scale;
};

// Hermitian half (HERM, passes after the first six qubits): every block of
// the assembly's intermediates, fixed higher letters over the transformed
// qubits, is Hermitian (real coefficients times tensor products of Hermitian
// Paulis), so only the stored entries are written and read: those whose low
// six column bits are at least the low six row bits rounded down to a
// multiple of 8 (whole 128-byte lines of the 16-byte intermediates, whole
// sectors of rho).  A pass's outputs keep the low bits of its inputs, so the
// set carries through, and the mirror (C, R) of every entry left out is
// stored.  The last pass writes the stored entries of rho and assemble_mirror
// the rest, as conjugates (the mirror of an exact butterfly is exactly the
// conjugate).
__device__ __forceinline__ bool herm_stored(int64_t R, int64_t C) { return (C & 63) >= ((R & 63) & ~7); }

// One (P', R_lo, C_lo) item of an assembly pass over J <= 2 qubits.
template <class Num, int J, bool FIRST, bool LAST, bool HERM = false>
__device__ __forceinline__ void asm_item(const AsmParams &P, int64_t item) {
  using V = typename Num::V;
  constexpr int NP = 1 << (2 * J);
  const int t = P.t;
  const int tp = t + J;
  const int64_t L4 = 1ll << (2 * t);  // 4^t
  const int64_t L = item & (L4 - 1);
  const int64_t Pp = item >> (2 * t);
  const int64_t R_lo = L >> t, C_lo = L & ((1ll << t) - 1);
  if (HERM && !herm_stored(R_lo, C_lo)) return;  // not stored: its mirror carries it
  V v[NP];
  const int64_t ibase = Pp * NP * L4 + L;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    if constexpr (FIRST)
      v[p] = load_first(static_cast<const typename Num::In *>(P.in), ibase + p * L4);
    else
      v[p] = __ldcg(static_cast<const V *>(P.in) + ibase + p * L4);
  }
  // digit 0 (qubit t): index p = p1*4 + p0 -> u0 = 2 r0 + c0
#pragma unroll
  for (int h = 0; h < NP / 4; ++h) {
    V a, b, c, d;
    m_qubit(v[4 * h + 0], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3], a, b, c, d);
    v[4 * h + 0] = a; v[4 * h + 1] = b; v[4 * h + 2] = c; v[4 * h + 3] = d;
  }
  if constexpr (J == 2) {
#pragma unroll
    for (int u0 = 0; u0 < 4; ++u0) {
      V a, b, c, d;
      m_qubit(v[u0], v[4 + u0], v[8 + u0], v[12 + u0], a, b, c, d);
      v[u0] = a; v[4 + u0] = b; v[8 + u0] = c; v[12 + u0] = d;
    }
  }
  // v[u1*4 + u0] with u_q = 2 r_q + c_q  ->  rj, cj
  const int64_t W = 1ll << tp;
  const int64_t obase = Pp * W * W;
#pragma unroll
  for (int u = 0; u < NP; ++u) {
    int rj, cj;
    if constexpr (J == 1) {
      rj = u >> 1;
      cj = u & 1;
    } else {
      const int u0 = u & 3, u1 = u >> 2;
      rj = ((u1 >> 1) << 1) | (u0 >> 1);
      cj = ((u1 & 1) << 1) | (u0 & 1);
    }
    const int64_t R = ((int64_t)rj << t) | R_lo;
    const int64_t Cc = ((int64_t)cj << t) | C_lo;
    const int64_t o = obase + R * W + Cc;
    if constexpr (LAST)
      static_cast<float2 *>(P.out)[o] = to_c64(v[u], P.scale);
    else
      static_cast<V *>(P.out)[o] = v[u];
  }
}

// ---- shared-memory tile of the assembly's first six qubits ---------------------
constexpr int ASM_TILE_SMEM = (4096 + 256) * 16;

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// The per-qubit map on two qubits of 16 values (index u = d0 + 4 d1).
template <typename V>
__device__ __forceinline__ void m2(V (&v)[16]) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    V a, b, c, d;
    m_qubit(v[4 * h + 0], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3], a, b, c, d);
    v[4 * h + 0] = a; v[4 * h + 1] = b; v[4 * h + 2] = c; v[4 * h + 3] = d;
  }
#pragma unroll
  for (int u0 = 0; u0 < 4; ++u0) {
    V a, b, c, d;
    m_qubit(v[u0], v[4 + u0], v[8 + u0], v[12 + u0], a, b, c, d);
    v[u0] = a; v[4 + u0] = b; v[8 + u0] = c; v[12 + u0] = d;
  }
}

// Qubits 0..5 of block `blk` (4096 consecutive coefficients of the first
// pass's input) -> [R_lo 64][C_lo 64] at out + blk * 4096, through the padded
// shared tile S (4096 + 256 entries).  All 256 threads of the CTA call it
// together.  LAST: the block is the whole matrix (n = 6) and is written as
// complex64 with the final scale.
// asm_low6_finish: the same after S holds the block's coefficients (and the
// CTA has synchronised): the butterflies and the writes.
template <class Num, bool LAST, bool HERM = false>
__device__ __forceinline__ void asm_low6_finish(void *__restrict__ out, int64_t blk, typename Num::V *S,
                                                const LastScale &scale) {
  using V = typename Num::V;
  const int tid = threadIdx.x;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int sh = 4 * r;
    const int lo = tid & ((1 << sh) - 1), hi = tid >> sh;
    V v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = S[pad16(lo | (u << sh) | (hi << (sh + 4)))];
    m2(v);
#pragma unroll
    for (int u = 0; u < 16; ++u) S[pad16(lo | (u << sh) | (hi << (sh + 4)))] = v[u];
    __syncthreads();
  }
  // S[pos], pos digit q = 2 r_q + c_q  ->  out[R_lo * 64 + C_lo]
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int o = tid + 256 * k;
    const int R = o >> 6, C = o & 63;
    int pos = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) pos |= ((((R >> q) & 1) << 1) | ((C >> q) & 1)) << (2 * q);
    if constexpr (LAST)
      static_cast<float2 *>(out)[blk * 4096 + o] = to_c64(S[pad16(pos)], scale);
    else if (!HERM || herm_stored(R, C))  // HERM: the stored part of the 64 x 64 block
      static_cast<V *>(out)[blk * 4096 + o] = S[pad16(pos)];
  }
  __syncthreads();
}

template <class Num, bool LAST, bool HERM = false>
__device__ __forceinline__ void asm_low6_block(const typename Num::In *__restrict__ in, void *__restrict__ out,
                                               int64_t blk, typename Num::V *S, const LastScale &scale) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int i = tid + 256 * k;
    S[pad16(i)] = load_first(in, blk * 4096 + i);
  }
  __syncthreads();
  asm_low6_finish<Num, LAST, HERM>(out, blk, S, scale);
}

}  // namespace passes
}  // namespace lre
