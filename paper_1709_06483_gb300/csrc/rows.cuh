// Rows of the operators: (H_k x)[r] for CSR, matrix-free XXZ and transverse-field terms, and the
// compile-time operator families of the persistent kernels.  Shared by the single-problem kernel
// (leja_persistent.cu) and the batched kernel (batched.cu).
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
};

}  // namespace rows
}  // namespace mg
