// Rows of the operators: (H_k x)[r] for CSR, matrix-free XXZ and transverse-field terms, in FP64
// and in fixed point (on an int64 copy of x), and the compile-time operator families of the
// persistent kernels.  Shared by the single-problem kernel (leja_persistent.cu), the batched kernel
// (batched.cu), the adjoint's augmented kernel (adjoint.cu) and the matvec entry point (apply.cu).
#pragma once

#include "magnus_internal.cuh"
#include "persist_common.cuh"

namespace mg {
namespace rows {

// ------------------------------------------------------------- rows of H_k x
// CSR row: sum_e val[e] x[col[e]].  Entries go in rounds of eight (real values) or four (complex)
// so that the column/value loads and the gathers of a whole round are in flight together.
template <int RS>
static __device__ __forceinline__ double2 csr_row_real(const Term &t, const double2 *x, int64_t e, int64_t e1) {
  double2 acc = make_double2(0.0, 0.0);
  const double *rv = t.rv;
  for (; e + 8 <= e1; e += 8) {
    int c[8];
    double a[8];
    double2 xv[8];
#pragma unroll
    for (int q = 0; q < 8; q++) c[q] = __ldg(t.col + e + q);
#pragma unroll
    for (int q = 0; q < 8; q++) a[q] = __ldg(rv + (e + q) * RS);
#pragma unroll
    for (int q = 0; q < 8; q++) xv[q] = ldv(x + c[q]);
#pragma unroll
    for (int q = 0; q < 8; q++) acc = rfma(a[q], xv[q], acc);
  }
  if (e + 4 <= e1) {
    int c[4];
    double a[4];
    double2 xv[4];
#pragma unroll
    for (int q = 0; q < 4; q++) c[q] = __ldg(t.col + e + q);
#pragma unroll
    for (int q = 0; q < 4; q++) a[q] = __ldg(rv + (e + q) * RS);
#pragma unroll
    for (int q = 0; q < 4; q++) xv[q] = ldv(x + c[q]);
#pragma unroll
    for (int q = 0; q < 4; q++) acc = rfma(a[q], xv[q], acc);
    e += 4;
  }
  for (; e < e1; e++) acc = rfma(__ldg(rv + e * RS), ldv(x + __ldg(t.col + e)), acc);
  return acc;
}

// The same sum with a warp-uniform trip count: every lane runs to the longest row among the warp's
// active lanes, loads nothing past its own row and adds zeros there.  Rounds of different lengths
// on different lanes would each take their FP64 slots (1.5x the entries of an XXZ row, whose
// lengths vary by up to 5 within a warp); this way a warp spends exactly its longest row.  Same
// entries in the same order as csr_row_real, so the same result.  Call with the warp converged.
#ifndef MG_CSR_ROUND
#define MG_CSR_ROUND 8
#endif
constexpr int kRound = MG_CSR_ROUND;  // entries per load round of the warp-uniform rows (8 or 4)

template <int RS>
static __device__ __forceinline__ double2 csr_row_real_w(const Term &t, const double2 *x, int64_t r) {
  const int64_t e0 = __ldg(t.rowptr + r);
  const int len = (int)(__ldg(t.rowptr + r + 1) - e0);
  const int lmax = __reduce_max_sync(__activemask(), len);
  const int32_t *col = t.col + e0;
  const double *rv = t.rv + e0 * RS;
  double2 acc = make_double2(0.0, 0.0);
  int k = 0;
  for (; k + kRound <= lmax; k += kRound) {
    int c[kRound];
    double a[kRound];
    double2 xv[kRound];
#pragma unroll
    for (int q = 0; q < kRound; q++) c[q] = (k + q < len) ? __ldg(col + k + q) : -1;
#pragma unroll
    for (int q = 0; q < kRound; q++) a[q] = (k + q < len) ? __ldg(rv + (k + q) * RS) : 0.0;
#pragma unroll
    for (int q = 0; q < kRound; q++) xv[q] = (c[q] >= 0) ? ldv(x + c[q]) : make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 0; q < kRound; q++) acc = rfma(a[q], xv[q], acc);
  }
  if (kRound == 8 && k + 4 <= lmax) {
    int c[4];
    double a[4];
    double2 xv[4];
#pragma unroll
    for (int q = 0; q < 4; q++) c[q] = (k + q < len) ? __ldg(col + k + q) : -1;
#pragma unroll
    for (int q = 0; q < 4; q++) a[q] = (k + q < len) ? __ldg(rv + (k + q) * RS) : 0.0;
#pragma unroll
    for (int q = 0; q < 4; q++) xv[q] = (c[q] >= 0) ? ldv(x + c[q]) : make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 0; q < 4; q++) acc = rfma(a[q], xv[q], acc);
    k += 4;
  }
  for (; k < lmax; k++) {
    const bool in = k < len;
    const double a = in ? __ldg(rv + k * RS) : 0.0;
    const double2 v = in ? ldv(x + __ldg(col + k)) : make_double2(0.0, 0.0);
    acc = rfma(a, v, acc);
  }
  return acc;
}

static __device__ __forceinline__ double2 csr_row(const Term &t, const double2 *x, int64_t r) {
  int64_t e = __ldg(t.rowptr + r);
  const int64_t e1 = __ldg(t.rowptr + r + 1);
  if (t.real_valued) return t.rs == 1 ? csr_row_real<1>(t, x, e, e1) : csr_row_real<2>(t, x, e, e1);
  double2 acc = make_double2(0.0, 0.0);
  for (; e + 4 <= e1; e += 4) {
    int c[4];
    double2 a[4], xv[4];
#pragma unroll
    for (int q = 0; q < 4; q++) c[q] = __ldg(t.col + e + q);
#pragma unroll
    for (int q = 0; q < 4; q++) a[q] = __ldg(t.val + e + q);
#pragma unroll
    for (int q = 0; q < 4; q++) xv[q] = ldv(x + c[q]);
#pragma unroll
    for (int q = 0; q < 4; q++) acc = cfma(a[q], xv[q], acc);
  }
  for (; e < e1; e++) acc = cfma(__ldg(t.val + e), ldv(x + __ldg(t.col + e)), acc);
  return acc;
}

// Open XXZ chain (Sec. 4 embedding, spin s at bit n-s): diagonal sum delta J_s z_s z_{s+1} + h_s z_s,
// and 2 J_s to the state with spins s, s+1 swapped when they are anti-parallel.
static __device__ __forceinline__ double2 xxz_row(const Term &t, const double2 *x, int64_t r) {
  const int n = t.nspins;
  double diag = 0.0;
  double2 acc = make_double2(0.0, 0.0);
  for (int s = 1; s <= n; s++) {
    const double zs = ((r >> (n - s)) & 1) ? -1.0 : 1.0;
    diag = fma(t.hz[s - 1], zs, diag);
    if (s < n) {
      const bool anti = ((r >> (n - s)) ^ (r >> (n - s - 1))) & 1;
      diag = fma(t.delta * t.J[s - 1], anti ? -1.0 : 1.0, diag);
      if (anti) acc = rfma(2.0 * t.J[s - 1], ldv(x + (r ^ ((int64_t)3 << (n - s - 1)))), acc);
    }
  }
  return rfma(diag, ldv(x + r), acc);
}

// sum_i sigma^x_i: the sum over all single-spin flips (all loads issued before the adds).
static __device__ __forceinline__ double2 fieldx_row(int n, const double2 *x, int64_t r) {
  double2 acc = make_double2(0.0, 0.0);
  int b = 0;
  for (; b + 4 <= n; b += 4) {
    const double2 v0 = ldv(x + (r ^ ((int64_t)1 << b))), v1 = ldv(x + (r ^ ((int64_t)2 << b))),
                  v2 = ldv(x + (r ^ ((int64_t)4 << b))), v3 = ldv(x + (r ^ ((int64_t)8 << b)));
    acc.x += (v0.x + v1.x) + (v2.x + v3.x);
    acc.y += (v0.y + v1.y) + (v2.y + v3.y);
  }
  for (; b < n; b++) {
    const double2 v = ldv(x + (r ^ ((int64_t)1 << b)));
    acc.x += v.x;
    acc.y += v.y;
  }
  return acc;
}

// coef * sum_i x[r ^ bit_i] accumulated with FMAs: on GB300 a DFMA with register operands issues
// faster than a DADD (measured 0.60 vs 0.51 T/s), and the weight costs no extra multiply.
static __device__ __forceinline__ double2 fieldx_row_scaled(int n, double coef, const double2 *x, int64_t r,
                                                           double2 acc) {
  int b = 0;
  for (; b + 4 <= n; b += 4) {
    const double2 v0 = ldv(x + (r ^ ((int64_t)1 << b))), v1 = ldv(x + (r ^ ((int64_t)2 << b))),
                  v2 = ldv(x + (r ^ ((int64_t)4 << b))), v3 = ldv(x + (r ^ ((int64_t)8 << b)));
    acc = rfma(coef, v0, acc);
    acc = rfma(coef, v1, acc);
    acc = rfma(coef, v2, acc);
    acc = rfma(coef, v3, acc);
  }
  for (; b < n; b++) acc = rfma(coef, ldv(x + (r ^ ((int64_t)1 << b))), acc);
  return acc;
}

// ------------------------------------------------ exact fixed-point sums of pattern terms
// A pattern term stores one value v on every entry (the transverse field sum_i sx_i, an adjacency
// pattern), so its row is v sum_e x[col_e]: additions only.  On GB300 one FP64 instruction takes
// the issue time of about 32 integer ones, so these sums run in 64-bit integers, exactly, on a
// fixed-point copy Z = trunc(x 2^s) of the vector.  Each vector has one scale s, chosen from a
// bound B >= max_r max(|Re x_r|, |Im x_r|) so that |Z| < 2^(62-hb) and a row sum of up to 2^(hb-1)
// entries stays below 2^61 (fix_scale); the truncation is below 2^-s < 2^(hb-61) B per component.
// The row sum goes back to FP64 once, rounded to nearest (unfix).

// scale s for components bounded by B: the smallest e with B < 2^e gives s = 62 - hb - e, in
// [-963 - hb, 1084 - hb] for every B up to Inf (B = 0 takes the largest), so the copy keeps its
// 62 - hb bits at any magnitude of the vector
static __device__ __forceinline__ int fix_scale(double B, int hb) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(B);
  const int ex = (int)(b >> 52) & 0x7FF;  // B in [2^(ex-1023), 2^(ex-1022)); B < 2^-1022 if ex = 0
  int s = 62 - hb - (ex - 1022);
  if (!(B > 0.0)) s = 1084;
  return min(max(s, -1000), 1100);
}

// trunc(x 2^s) from the bits of x (integer operations only)
static __device__ __forceinline__ long long fix64(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)(b >> 52) & 0x7FF;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (ex ? 0x10000000000000ull : 0ull);
  const int sh = max(ex, 1) - 1075 + s;  // x = m 2^(max(ex,1) - 1075)
  // for |x| <= B the shift is at most 9 to the left; the clamps only keep Inf/NaN shifts defined
  const unsigned long long v = sh >= 0 ? (m << min(sh, 11)) : (sh > -64 ? (m >> -sh) : 0ull);
  return (b >> 63) ? -(long long)v : (long long)v;
}
static __device__ __forceinline__ longlong2 fix2(double2 v, int s) { return make_longlong2(fix64(v.x, s), fix64(v.y, s)); }

// n 2^-s rounded to the nearest double (ties to even), built from the bits of n; a result below
// 2^-1022 flushes to a signed zero and one above the largest double gives a signed infinity (the
// scales of products, s - fe - 2, reach past both ends)
static __device__ __forceinline__ double unfix(long long n, int s) {
  const unsigned long long sg = (unsigned long long)n & 0x8000000000000000ull;
  const unsigned long long a0 = sg ? 0ull - (unsigned long long)n : (unsigned long long)n;
  const int lz = __clzll((long long)a0);
  const unsigned long long a = a0 << (lz & 63);  // leading one at bit 63 (a0 != 0)
  unsigned long long m = a >> 11;                // 53 significant bits
  const unsigned rb = (unsigned)a & 0x7FFu;      // the 11 bits below them
  m += (rb > 0x400u || (rb == 0x400u && (m & 1ull))) ? 1ull : 0ull;
  // value = (m / 2^52) 2^(63 - lz - s); m's leading one (or its carry to 2^53) lands in the exponent,
  // whose field is ef + 1 (ef + 2 after a carry): normal for ef in [0, 2045], 2046 + a carry is Inf
  const int ef = 1085 - lz - s;
  const unsigned long long bits = sg | (((unsigned long long)ef << 52) + m);
  if (!a0 || ef < 0) return __longlong_as_double((long long)sg);
  return __longlong_as_double((long long)(ef > 2045 ? (sg | 0x7FF0000000000000ull) : bits));
}
static __device__ __forceinline__ double2 unfix2(longlong2 n, int s) { return make_double2(unfix(n.x, s), unfix(n.y, s)); }

// High word of max(|Re v|, |Im v|): non-negative doubles order like their bit patterns, so the
// double with high word h + 1 and low word 0 bounds every value whose high word is at most h.
static __device__ __forceinline__ unsigned abshi(double2 v) {
  return max((unsigned)__double2hiint(v.x) & 0x7FFFFFFFu, (unsigned)__double2hiint(v.y) & 0x7FFFFFFFu);
}
static __device__ __forceinline__ double abshi_bound(unsigned h) { return __hiloint2double((int)(h + 1u), 0); }

static __device__ __forceinline__ longlong2 ldz(const longlong2 *p) { return __ldca(p); }
static __device__ __forceinline__ void zadd(longlong2 &acc, longlong2 v) {
  acc.x += v.x;
  acc.y += v.y;
}

// ------------------------------------------------ sliced rows (Term::hbase, slices.cu)
// Head of row r: its slice's first w entries, column-major (entry k at hbase[s] + 32 k + (r & 31)):
// one coalesced load of entry k for the warp's 32 rows, no row pointer.  Tail: the rest, row-major
// behind tptr.  Both sums exact in int64, so the order of the entries does not matter.
static __device__ __forceinline__ void sl_head(const Term &t, int64_t r, int64_t &hb, int &w) {
  const int64_t s = r >> 5;
  hb = __ldg(t.hbase + s);
  w = (int)((__ldg(t.hbase + s + 1) - hb) >> 5);
  hb += r & 31;
}

// sum_e Z[col_e] over the sliced row r of a pattern term
static __device__ __forceinline__ longlong2 sl_row_zsum(const Term &t, const longlong2 *z, int64_t r) {
  int64_t hb;
  int w;
  sl_head(t, r, hb, w);
  const int32_t *hc = t.hcol + hb;
  longlong2 acc = make_longlong2(0, 0);
  int k = 0;
  for (; k + kRound <= w; k += kRound) {
    int c[kRound];
    longlong2 v[kRound];
#pragma unroll
    for (int q = 0; q < kRound; q++) c[q] = __ldg(hc + 32 * (k + q));
#pragma unroll
    for (int q = 0; q < kRound; q++) v[q] = ldz(z + c[q]);
#pragma unroll
    for (int q = 0; q < kRound; q++) zadd(acc, v[q]);
  }
  if (kRound == 8 && k + 4 <= w) {
    int c[4];
    longlong2 v[4];
#pragma unroll
    for (int q = 0; q < 4; q++) c[q] = __ldg(hc + 32 * (k + q));
#pragma unroll
    for (int q = 0; q < 4; q++) v[q] = ldz(z + c[q]);
#pragma unroll
    for (int q = 0; q < 4; q++) zadd(acc, v[q]);
    k += 4;
  }
  for (; k < w; k++) zadd(acc, ldz(z + __ldg(hc + 32 * k)));
  if (t.tptr)
    for (int64_t e = __ldg(t.tptr + r), e1 = __ldg(t.tptr + r + 1); e < e1; e++) zadd(acc, ldz(z + __ldg(t.tcol + e)));
  return acc;
}

// sum_e hi64(fval_e Z[col_e]) over the sliced row r of a product term (the tail with the warp's
// longest tail as the trip count: call with the warp converged)
static __device__ __forceinline__ longlong2 sl_row_zprod(const Term &t, const longlong2 *z, int64_t r) {
  int64_t hb;
  int w;
  sl_head(t, r, hb, w);
  const int32_t *hc = t.hcol + hb;
  const long long *hv = t.hval + hb;
  longlong2 acc = make_longlong2(0, 0);
  int k = 0;
  for (; k + kRound <= w; k += kRound) {
    int c[kRound];
    long long a[kRound];
    longlong2 v[kRound];
#pragma unroll
    for (int q = 0; q < kRound; q++) c[q] = __ldg(hc + 32 * (k + q));
#pragma unroll
    for (int q = 0; q < kRound; q++) a[q] = __ldg(hv + 32 * (k + q));
#pragma unroll
    for (int q = 0; q < kRound; q++) v[q] = ldz(z + c[q]);
#pragma unroll
    for (int q = 0; q < kRound; q++) {
      acc.x += __mul64hi(a[q], v[q].x);
      acc.y += __mul64hi(a[q], v[q].y);
    }
  }
  for (; k < w; k++) {
    const long long a = __ldg(hv + 32 * k);
    const longlong2 v = ldz(z + __ldg(hc + 32 * k));
    acc.x += __mul64hi(a, v.x);
    acc.y += __mul64hi(a, v.y);
  }
  if (t.tptr) {
    const int64_t e0 = __ldg(t.tptr + r);
    const int len = (int)(__ldg(t.tptr + r + 1) - e0);
    const int lmax = __reduce_max_sync(__activemask(), len);
    for (int j = 0; j < lmax; j += 4) {
      long long a[4];
      longlong2 v[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const bool in = j + q < len;
        a[q] = in ? __ldg(t.tval + e0 + j + q) : 0ll;
        v[q] = in ? ldz(z + __ldg(t.tcol + e0 + j + q)) : make_longlong2(0, 0);
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        acc.x += __mul64hi(a[q], v[q].x);
        acc.y += __mul64hi(a[q], v[q].y);
      }
    }
  }
  return acc;
}

// sum_e Z[col_e] over a CSR row, rounds of kRound entries (rows of one length plen start at r plen:
// no row-pointer load before the column loads)
static __device__ __forceinline__ longlong2 csr_row_zsum(const Term &t, const longlong2 *z, int64_t r) {
  if (t.hbase) return sl_row_zsum(t, z, r);
  int64_t e = t.plen ? r * t.plen : __ldg(t.rowptr + r);
  const int64_t e1 = t.plen ? e + t.plen : __ldg(t.rowptr + r + 1);
  longlong2 acc = make_longlong2(0, 0);
  for (; e + kRound <= e1; e += kRound) {
    int c[kRound];
    longlong2 v[kRound];
#pragma unroll
    for (int q = 0; q < kRound; q++) c[q] = __ldg(t.col + e + q);
#pragma unroll
    for (int q = 0; q < kRound; q++) v[q] = ldz(z + c[q]);
#pragma unroll
    for (int q = 0; q < kRound; q++) zadd(acc, v[q]);
  }
  if (kRound == 8 && e + 4 <= e1) {
    int c[4];
    longlong2 v[4];
#pragma unroll
    for (int q = 0; q < 4; q++) c[q] = __ldg(t.col + e + q);
#pragma unroll
    for (int q = 0; q < 4; q++) v[q] = ldz(z + c[q]);
#pragma unroll
    for (int q = 0; q < 4; q++) zadd(acc, v[q]);
    e += 4;
  }
  for (; e < e1; e++) zadd(acc, ldz(z + __ldg(t.col + e)));
  return acc;
}

// sum_e fval[e] Z[col_e] / 2^64 over a CSR row in fixed point (each product's high 64 bits:
// |fval| < 2^62 and |Z| < 2^(62-hb) keep every product below 2^(60-hb) and the sum exact), with a
// warp-uniform trip count; returns the sum and, in fe, the row's exponent.  The row's value is
// sum 2^(fe + 2 - zs) with zs the scale of Z.  Call with the warp converged.
static __device__ __forceinline__ longlong2 csr_row_zprod_w(const Term &t, const longlong2 *z, int64_t r, int &fe) {
  if (t.hbase) {
    fe = __ldg(t.fexp + r);
    return sl_row_zprod(t, z, r);
  }
  const int64_t e0 = __ldg(t.rowptr + r);
  const int len = (int)(__ldg(t.rowptr + r + 1) - e0);
  const int lmax = __reduce_max_sync(__activemask(), len);
  fe = __ldg(t.fexp + r);
  const int32_t *col = t.col + e0;
  const long long *fv = t.fval + e0;
  longlong2 acc = make_longlong2(0, 0);
  int k = 0;
  for (; k + kRound <= lmax; k += kRound) {
    int c[kRound];
    long long a[kRound];
    longlong2 v[kRound];
#pragma unroll
    for (int q = 0; q < kRound; q++) c[q] = (k + q < len) ? __ldg(col + k + q) : -1;
#pragma unroll
    for (int q = 0; q < kRound; q++) a[q] = (k + q < len) ? __ldg(fv + k + q) : 0ll;
#pragma unroll
    for (int q = 0; q < kRound; q++) v[q] = (c[q] >= 0) ? ldz(z + c[q]) : make_longlong2(0, 0);
#pragma unroll
    for (int q = 0; q < kRound; q++) {
      acc.x += __mul64hi(a[q], v[q].x);
      acc.y += __mul64hi(a[q], v[q].y);
    }
  }
  for (; k < lmax; k++) {
    const bool in = k < len;
    const long long a = in ? __ldg(fv + k) : 0ll;
    const longlong2 v = in ? ldz(z + __ldg(col + k)) : make_longlong2(0, 0);
    acc.x += __mul64hi(a, v.x);
    acc.y += __mul64hi(a, v.y);
  }
  return acc;
}

// sum_i Z[r ^ bit_i] (the transverse field)
static __device__ __forceinline__ longlong2 fieldx_row_zsum(int n, const longlong2 *z, int64_t r) {
  longlong2 acc = make_longlong2(0, 0);
  int b = 0;
  for (; b + 4 <= n; b += 4) {
    const longlong2 v0 = ldz(z + (r ^ ((int64_t)1 << b))), v1 = ldz(z + (r ^ ((int64_t)2 << b))),
                    v2 = ldz(z + (r ^ ((int64_t)4 << b))), v3 = ldz(z + (r ^ ((int64_t)8 << b)));
    zadd(acc, v0);
    zadd(acc, v1);
    zadd(acc, v2);
    zadd(acc, v3);
  }
  for (; b < n; b++) zadd(acc, ldz(z + (r ^ ((int64_t)1 << b))));
  return acc;
}

static __device__ __forceinline__ double2 term_row_generic(const Term &t, const double2 *x, int64_t r) {
  switch (t.kind) {
    case MAGNUS_TERM_CSR: return csr_row(t, x, r);
    case MAGNUS_TERM_XXZ: return xxz_row(t, x, r);
    case MAGNUS_TERM_FIELD_X: return fieldx_row(t.nspins, x, r);
    default: return make_double2(0.0, 0.0);
  }
}

// Per-block operator context: terms in shared memory plus, for FAM_MF, the diagonal tables and
// the bond couplings pre-scaled by the current exponential's weight.
struct Ctx {
  const Term *T;
  int nt;
  int n, lbits;
  int64_t lomask;
  const double *dlo, *dhi;
  const double *jb;   // shared: 2 J_bond * bg[0] per bond, bond at bits (p, p-1) stored at p-1
  const double *j2;   // shared: 2 J_bond (unscaled), same indexing
  const long long *cb;  // shared (fixed-point kernel): jb as 62-bit mantissas, cb = round(jb 2^(62 - cbe))
  int cbe;              // with max |jb| < 2^cbe
  const long long *c2;  // shared (fixed-point M4): j2 as mantissas, c2 = round(j2 2^(62 - c2e))
  int c2e;
};

// H_xxz row with the diagonal from the two tables (FAM_MF).  coefj: per-bond coefficients.
// The bonds are visited over the union of the active (anti-parallel) bonds of the warp's rows: a
// warp's rows share their high bits, so high bonds are active for all lanes or none and an inactive
// one costs no FP64 slot; only the low bonds (bits below 5) are taken per lane.  Ascending bond order
// in every case, so the sum is the same as over all active bonds in order.
[[maybe_unused]] constexpr int kMaxBonds = kMaxSpins - 1;
static __device__ __forceinline__ double2 mf_xxz_row(const Ctx &c, const double *coefj, double dscale, double dshift,
                                              const double2 *x, int64_t r, double2 &xr) {
  xr = ldv(x + r);
  const double dg = __ldg(c.dhi + (r >> c.lbits)) + __ldg(c.dlo + (r & c.lomask));
  const double cr = fma(dscale, dg, -dshift);
  double2 acc;
  acc.x = cr * xr.x;
  acc.y = cr * xr.y;
  const int nb = c.n - 1;
  // bit b of `mine`: bond at bits (b + 1, b) is anti-parallel in row r
  const unsigned mine = (unsigned)((r ^ (r >> 1)) & (((int64_t)1 << nb) - 1));
  unsigned mw = __reduce_or_sync(__activemask(), mine);
  while (__popc(mw) >= 4) {
    int bq[4];
    double2 v[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      bq[q] = __ffs(mw) - 1;
      mw &= mw - 1;
    }
#pragma unroll
    for (int q = 0; q < 4; q++) v[q] = ldv(x + (r ^ ((int64_t)3 << bq[q])));
#pragma unroll
    for (int q = 0; q < 4; q++)
      if ((mine >> bq[q]) & 1u) acc = rfma(coefj[bq[q]], v[q], acc);
  }
  while (mw) {
    const int b = __ffs(mw) - 1;
    mw &= mw - 1;
    const double2 v = ldv(x + (r ^ ((int64_t)3 << b)));
    if ((mine >> b) & 1u) acc = rfma(coefj[b], v, acc);
  }
  return acc;
}

// The same row with the bond flips taken in fixed point: each active bond adds the high 64 bits of
// cb[b] Z[r ^ (3 << b)] (|cb| < 2^62, |Z| < 2^(62-hb)), exactly summed in int64, and the sum goes back
// to FP64 once; the diagonal stays FP64.  Same visiting order as mf_xxz_row.
static __device__ __forceinline__ double2 mf_xxz_row_z(const Ctx &c, const long long *cb, int cbe, double dscale,
                                                double dshift, const double2 *x, const longlong2 *z, int zs, int64_t r,
                                                double2 &xr) {
  xr = ldv(x + r);
  const double dg = __ldg(c.dhi + (r >> c.lbits)) + __ldg(c.dlo + (r & c.lomask));
  const double cr = fma(dscale, dg, -dshift);
  const int nb = c.n - 1;
  const unsigned mine = (unsigned)((r ^ (r >> 1)) & (((int64_t)1 << nb) - 1));
  unsigned mw = __reduce_or_sync(__activemask(), mine);
  longlong2 acc = make_longlong2(0, 0);
  while (__popc(mw) >= 4) {
    int bq[4];
    longlong2 v[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      bq[q] = __ffs(mw) - 1;
      mw &= mw - 1;
    }
#pragma unroll
    for (int q = 0; q < 4; q++) v[q] = ldz(z + (r ^ ((int64_t)3 << bq[q])));
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const long long w = ((mine >> bq[q]) & 1u) ? cb[bq[q]] : 0ll;
      acc.x += __mul64hi(w, v[q].x);
      acc.y += __mul64hi(w, v[q].y);
    }
  }
  while (mw) {
    const int b = __ffs(mw) - 1;
    mw &= mw - 1;
    const longlong2 v = ldz(z + (r ^ ((int64_t)3 << b)));
    const long long w = ((mine >> b) & 1u) ? cb[b] : 0ll;
    acc.x += __mul64hi(w, v.x);
    acc.y += __mul64hi(w, v.y);
  }
  const double2 bonds = unfix2(acc, zs - cbe - 2);
  return make_double2(fma(cr, xr.x, bonds.x), fma(cr, xr.y, bonds.y));
}

template <int FAM>
struct Op {
  // (H_k x)[r]
  __device__ static __forceinline__ double2 term(const Ctx &c, int k, const double2 *x, int64_t r) {
    if (FAM == FAM_CSR) return csr_row(c.T[k], x, r);
    if (FAM == FAM_MF) {
      if (k == 0) {
        double2 xr;
        return mf_xxz_row(c, c.j2, 1.0, 0.0, x, r, xr);
      }
      return fieldx_row(c.n, x, r);
    }
    return term_row_generic(c.T[k], x, r);
  }
  // sum_k bg_k (H_k x)[r] - shift x[r]; also returns x[r]
  __device__ static __forceinline__ double2 combo(const Ctx &c, const ExpRec &R, double shift, const double2 *x,
                                                  int64_t r, double2 &xr) {
    if (FAM == FAM_MF) {
      double2 y = mf_xxz_row(c, c.jb, R.bg[0], shift, x, r, xr);
      return fieldx_row_scaled(c.n, R.bg[1], x, r, y);
    }
    double2 y = make_double2(0.0, 0.0);
    for (int k = 0; k < c.nt; k++) y = rfma(R.bg[k], term(c, k, x, r), y);
    xr = ldv(x + r);
    return rfma(-shift, xr, y);
  }
  // (H_k x)[r] from the fixed-point copy Z = trunc(x 2^zs) where the term allows it (pattern sums,
  // mantissa products, matrix-free flips), else in FP64 from x (M4 phases of the fixed-point kernel)
  __device__ static __forceinline__ double2 term_z(const Ctx &c, int k, const double2 *x, const longlong2 *z, int zs,
                                                   int64_t r) {
    if constexpr (FAM == FAM_MF) {
      if (k == 0) {
        double2 xr;
        return mf_xxz_row_z(c, c.c2, c.c2e, 1.0, 0.0, x, z, zs, r, xr);
      }
      const double2 f = unfix2(fieldx_row_zsum(c.n, z, r), zs);
      return f;
    } else {
      const Term &t = c.T[k];
      if (t.pattern) {
        const double2 f = unfix2(csr_row_zsum(t, z, r), zs);
        return make_double2(t.pval * f.x, t.pval * f.y);
      }
      if (t.fval) {
        int fe;
        const longlong2 hs = csr_row_zprod_w(t, z, r, fe);
        return unfix2(hs, zs - fe - 2);
      }
      return csr_row(t, x, r);
    }
  }
  // combo with the pattern terms summed exactly on Z = trunc(x 2^zs) and weighted by wz[k] =
  // bg_k v_k (FAM_CSR: terms flagged `pattern`; FAM_MF: the transverse field)
  __device__ static __forceinline__ double2 combo_z(const Ctx &c, const ExpRec &R, const double *wz, double shift,
                                                    const double2 *x, const longlong2 *z, int zs, int64_t r,
                                                    double2 &xr) {
    if constexpr (FAM == FAM_MF) {
      double2 y = c.cb ? mf_xxz_row_z(c, c.cb, c.cbe, R.bg[0], shift, x, z, zs, r, xr)
                       : mf_xxz_row(c, c.jb, R.bg[0], shift, x, r, xr);
      return rfma(wz[1], unfix2(fieldx_row_zsum(c.n, z, r), zs), y);
    } else {
      double2 y = make_double2(0.0, 0.0);
      for (int k = 0; k < c.nt; k++) {
        const Term &t = c.T[k];
        if (t.pattern) {
          y = rfma(wz[k], unfix2(csr_row_zsum(t, z, r), zs), y);
        } else if (t.fval) {
          int fe;
          const longlong2 hs = csr_row_zprod_w(t, z, r, fe);
          y = rfma(R.bg[k], unfix2(hs, zs - fe - 2), y);
        } else if (t.real_valued)
          y = rfma(R.bg[k], t.rs == 1 ? csr_row_real_w<1>(t, x, r) : csr_row_real_w<2>(t, x, r), y);
        else
          y = rfma(R.bg[k], csr_row(t, x, r), y);
      }
      xr = ldv(x + r);
      return rfma(-shift, xr, y);
    }
  }
};

}  // namespace rows
}  // namespace mg
