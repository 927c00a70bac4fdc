// Internal declarations of the GB300 Magnus + Leja library (arXiv:1709.06483).
// Device-side records, small complex helpers and the launch wrappers the host
// API (magnus_api.cu) calls.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "magnus.h"

namespace mg {

// NVTX range for the extent of a scope (a profiler shows the API calls and the launches inside
// them; header-only, inert when no tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kMaxTerms = 4;
constexpr int kMaxPairs = kMaxTerms * (kMaxTerms - 1) / 2;
constexpr int kMaxModes = 64;
constexpr int kMaxSpins = 30;
constexpr int kMmaxLimit = 255;

// One stored term H_k as the kernels see it.
struct Term {
  int kind;          // magnus_term_kind
  int nspins;        // matrix-free terms
  int real_valued;   // CSR / DENSE: every imaginary part is zero (then only the real parts are multiplied)
  int rs;            // CSR / DENSE with real_valued: real part of entry e at rv[e * rs] (2: complex storage, 1: real storage)
  int64_t nnz;
  const int64_t *rowptr;
  const int32_t *col;
  const double2 *val;  // complex storage (nullptr for real storage)
  const double *rv;    // real parts (complex storage viewed as doubles, or the real storage itself)
  double J[kMaxSpins];   // XXZ bond couplings J_1..J_{n-1}
  double hz[kMaxSpins];  // XXZ longitudinal fields h_1..h_n
  double delta;          // XXZ zz anisotropy
  int pattern;           // CSR, real-valued, every stored value equal to pval (sums taken in fixed point)
  int pbits;             // ceil(log2(longest row)) of a pattern term
  int plen;              // pattern term whose rows all hold plen entries (rowptr[r] = r plen), else 0
  int _pad2;
  double pval;
  double gnorm;          // upper bound of ||H_k||_inf (max absolute row sum, from the Gershgorin pass)
  // fixed-point products (real CSR terms in the fixed-point kernel; null: FP64 products): entry e
  // of row r as fval[e] = round(a_e 2^(62 - fexp[r])), with max_e |a_e| < 2^fexp[r]
  const long long *fval;
  const int16_t *fexp;
  // sliced rows (pattern and product terms of fixed-point CSR plans; null: CSR rows): per 32-row
  // slice s the first w_s entries of every row (w_s = the slice's shortest row) column-major,
  // entry k of row 32 s + l at hbase[s] + 32 k + l of hcol (and hval, the mantissas), w_s =
  // (hbase[s+1] - hbase[s]) / 32; the rest of each row (its tail) row-major at [tptr[r], tptr[r+1])
  // of tcol / tval (tptr null: no row has a tail).  Within a row the entries are ordered by how
  // many rows of the slice share their column offset col - r, so that entry k of the 32 rows
  // gathers from one run of the vector where the matrix allows.
  const int64_t *hbase;
  const int32_t *hcol;
  const long long *hval;
  const int64_t *tptr;
  const int32_t *tcol;
  const long long *tval;
};

// Public term (magnus_term) -> storage fields of the internal Term: real-storage kinds become CSR /
// DENSE with real_valued values read at stride 1, complex storage keeps val and exposes its real
// parts at stride 2.
inline void set_term_storage(Term &T, const magnus_term &t) {
  const bool real_store = t.kind == MAGNUS_TERM_CSR_REAL || t.kind == MAGNUS_TERM_DENSE_REAL;
  T.kind = t.kind == MAGNUS_TERM_CSR_REAL ? MAGNUS_TERM_CSR : (t.kind == MAGNUS_TERM_DENSE_REAL ? MAGNUS_TERM_DENSE : t.kind);
  T.val = real_store ? nullptr : (const double2 *)t.val;
  T.rv = (const double *)t.val;
  T.rs = real_store ? 1 : 2;
  if (real_store) T.real_valued = 1;
}

// Drive coefficient f_k(t) = a0 + sum_m (ac_m cos(om_m t) + as_m sin(om_m t)).
struct Coeff {
  double a0;
  int nmodes;
  int _pad;
  double ac[kMaxModes], as[kMaxModes], om[kMaxModes];
};

// Everything one exponential exp(-iK) needs inside the persistent kernel.  K is shifted and
// scaled to X = (K - cI)/gamma with spectrum in [-2,2]; the stored weights already carry 1/gamma.
enum { MODE_LINEAR = 0, MODE_M4 = 1, MODE_M6 = 2 };
struct ExpRec {
  double bg[kMaxTerms];  // beta_k / gamma      (linear part: K = sum_k beta_k H_k + ...)
  double kg[kMaxPairs];  // M4: kappa * coef_kl / gamma, pairs (k<l) in row-major order
  double cg;             // c / gamma
  double gamma;          // quarter width of the spectral enclosure (0: K is a scalar)
  double c;              // centre of the enclosure
  double a, b;           // the enclosure itself (diagnostics)
  int s;                 // substeps
  int mode;              // MODE_LINEAR, MODE_M4 or MODE_M6
  // M6: B_1 = -iP, B_2 = -iQ, B_3 = -iR with P, Q, R = sum_k {p6,q6,r6}_k H_k (not divided by gamma)
  double p6[kMaxTerms], q6[kMaxTerms], r6[kMaxTerms];
};

constexpr int kM6Slots = 23;  // vectors the M6 generator keeps between its stages

// Grid barrier state (one per plan, zero-initialised): count's top bit flips at every completed
// barrier (grid_barrier); gen is unused.
struct GridBar {
  unsigned int count;
  unsigned int gen;
  int error;      // set by the first block whose wait timed out
  int _pad;
};

struct Counters {
  long long n_exp, n_substeps, n_matvec, n_termapply;
  int max_m;
  int status;
  unsigned long long max_drift;  // bits of the largest | ||p|| - ||v|| | / ||v|| (non-negative doubles order like their bits)
};

// After a substep: record | ||p|| - ||v|| | / ||v|| (block 0) and say whether it breaks the norm check
// (every block takes the same decision: pn and vn are the shared totals).
__device__ __forceinline__ bool drift_fails(double pn, double vn, double tol_abs, double tol_rel, double check,
                                            Counters *c, bool record) {
  const double d = fabs(pn - vn);
  if (record && vn > 0.0) atomicMax(&c->max_drift, (unsigned long long)__double_as_longlong(d / vn));
  return check > 0.0 && d > check * (tol_abs + tol_rel * vn) + 1e-13 * vn;
}

// ---------------------------------------------------------------- complex helpers
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + a*b
__host__ __device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc + s*b, s real
__host__ __device__ __forceinline__ double2 rfma(double s, double2 b, double2 acc) {
  acc.x = fma(s, b.x, acc.x);
  acc.y = fma(s, b.y, acc.y);
  return acc;
}
__host__ __device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }

// ---------------------------------------------------------------- launch wrappers
// Leja points xi[0..m] on [-2,2] (Sec. 3); scratch: 2*(m+1) doubles + 1 unsigned.
cudaError_t launch_leja_points(double *xi, int m, double *cand, unsigned *counter, cudaStream_t st);
// Divided differences of exp(-i rho x) at xi[0..m] (Sec. 3) into d[0..m] (device).
cudaError_t launch_divided_differences(const double *xi, int m, double rho, double2 *d, cudaStream_t st);
// Gershgorin enclosure of one term; out[0] = a, out[1] = b (device); scratch: 2*nblk doubles.
cudaError_t launch_gershgorin(const Term *t_dev, const Term &t_host, int64_t dim, double *scratch, int nblk,
                              double *out, cudaStream_t st);
// Real-valuedness check of a CSR / dense term: flag (device int) set to 1 if any imaginary part != 0.
cudaError_t launch_imag_check(const double2 *val, int64_t n, int *flag, cudaStream_t st);
// y = sum_k beta_k H_k x for nv states (the plan's operator family).  With zc and zmax (CSR and
// matrix-free plans in fixed point): the Z copy of x goes to zc [nv][D] at the scale of max |x| per
// state (reduced into zmax[nv]), and the pattern sums and value products run on it; else FP64.
cudaError_t launch_apply(int fam, const Term *terms, int nt, const double *beta, int lbits, const double *dlo,
                         const double *dhi, const double2 *x, double2 *y, int64_t D, int nv, longlong2 *zc,
                         unsigned *zmax, int zhb, int num_sms, cudaStream_t st);
// ab_dev (in: the term's Gershgorin enclosure) <- its intersection with the Lanczos enclosure after
// m steps; synchronises the stream
cudaError_t lanczos_interval(const Term *t_dev, const Term &t_host, int64_t D, int m, double *ab_dev, cudaStream_t st);
constexpr int kLanczosSteps = 48;
// Fixed-point copy of a real CSR term's values (rv[e * rs]): per row r the exponent fexp[r] with
// max_e |a_e| < 2^fexp[r] (0 for an empty or all-zero row) and fval[e] = round(a_e 2^(62 - fexp[r])).
// *wide |= 1 (device int, zeroed by the caller) if a row's exponent is outside [-400, 400] or a value
// is not finite: the copy is then unusable.
cudaError_t launch_fixed_values(const int64_t *rowptr, const double *rv, int rs, int64_t dim, long long *fval,
                                int16_t *fexp, int *wide, cudaStream_t st);
// Real-valued CSR term (values rv[e * rs], nnz > 0): flag |= 1 unless every stored value equals the
// first, |= 2 unless every row holds rowmax entries and rowptr[0] = 0; rowmax (device, zeroed by the
// caller) = longest row.
cudaError_t launch_pattern_check(const int64_t *rowptr, const double *rv, int rs, int64_t dim, int *flag,
                                 unsigned long long *rowmax, cudaStream_t st);
cudaError_t launch_real_parts(const double2 *z, int64_t n, double *out, int *flag, cudaStream_t st);
// Per-exponential records + divided-difference tables for a whole propagation.
cudaError_t launch_exp_setup(int variant, double t0, double h, int64_t nsteps, int nterms, const Coeff *coeffs,
                             const double *term_ab, const double *xi, int m_max, double rho_max, ExpRec *recs,
                             double2 *dd, int64_t nexp, cudaStream_t st);
// Records for a single exponential exp(-i sum_k beta_k H_k) (beta on the host).
cudaError_t launch_exp_setup_batch(int variant, double t0, double h, int64_t nsteps, int count, const int *nterms_dev,
                                   const Coeff *coeffs, const double *term_ab, const double *xi, int m_max,
                                   double rho_max, ExpRec *recs, double2 *dd, int64_t rec_stride, cudaStream_t st);
cudaError_t launch_exp_setup_beta(const double *beta_host, int nterms, const double *term_ab, const double *xi,
                                  int m_max, double rho_max, ExpRec *recs, double2 *dd, cudaStream_t st);

int exps_per_step(int variant);

// The persistent propagation kernel (Sec. 3 Leja loop inside Sec. 2 stepping).
struct PersistArgs {
  int64_t dim;
  int nvec, nterms, gv;    // gv: blocks per vector
  int m_max;
  int64_t nexp;
  double tol_rel, tol_abs;
  double norm_check;       // > 0: a substep whose norm drift exceeds norm_check (tol_abs + tol_rel ||v||) + 1e-13 ||v|| fails with MAGNUS_EDRIFT
  const Term *terms;       // device [nterms]
  const ExpRec *recs;      // device [nexp]
  const double2 *dd;       // device [nexp][m_max+1]
  const double *xi;        // device [m_max+1]
  double2 *psi;            // user buffer (in/out), [nvec][dim]
  double2 *alt;            // second state buffer
  double2 *w0, *w1;        // Leja ping-pong vectors
  double2 *u;              // M4: [nterms][nvec][dim]
  double *partials;        // [2][grid][4]: two sums and two maxima per block
  GridBar *bar;
  Counters *counters;
  int *mlog;               // [capacity] degrees of the substeps (may be null)
  long long mlog_cap;
  long long spin_limit_ns; // bounded waits
  int skip_arrival;        // testing: CTA 0 leaves before its first grid barrier
  int fam;                 // operator family: FAM_GENERIC, FAM_CSR (every term CSR), FAM_MF (XXZ + field)
  int lbits;               // FAM_MF: split of the basis index for the diagonal tables
  const double *dlo;       // FAM_MF: diagonal of H_xxz from the low lbits+1 bits   [2^(lbits+1)]
  const double *dhi;       // FAM_MF: diagonal of H_xxz from bits lbits..n-1         [2^(n-lbits)]
  // FAM_DENSE with MAGNUS_FP32_SPLIT: dense terms as FP32 (hi, lo) pairs of their real parts, and
  // (re_hi, re_lo, im_hi, im_lo) shadows of every vector set a dense matvec reads
  int split;
  const float2 *hsplit[kMaxTerms];
  float4 *sh_cur, *sh_w0, *sh_w1, *sh_u;
  // FAM_DENSE with MAGNUS_TENSOR_SLICED: bf16 digits of the dense terms ([5][D][D], row exponents)
  // and of every vector set a dense matvec reads ([5][2 nvec][D], column exponents), and the
  // column-maximum slots of the slicing passes ([4][128], zero at launch: three rotate, the fourth
  // collects the maxima the tcgen05 path gathers in its epilogue)
  double2 *m6;  // M6 intermediate vectors, kM6Slots x [nvec][dim]
  // FAM_DENSE with MAGNUS_TENSOR_SLICED on tcgen05 (linear generators and M4): 4 x 8-bit digits
  int tc;                         // tcgen05 digit products: 1 linear generators, 2 M4
  int tc_ndense, tc_slots, tc_T;
  long long tc_N;
  long long tc_spins;             // spin budget of every mbarrier wait
  int tc_dslot[kMaxTerms];        // dense term k -> its index among the dense terms
  const void *tc_hd;              // dense-term digits, tiled [ndense][dim/128][dim/8][4][128][8]
  const int *tc_eh;               // row exponents [ndense][dim]
  void *tc_wd;                    // vector-set digits, tiled [3 + nterms][dim/8][4][128][8] (sets: substep input, w0, w1, u_k)
  int *tc_ex;                     // their column exponents [3 + nterms][128]
  double2 *tc_cacc;               // M4: the commutator sum of the current Leja iteration [nvec][dim]
  double *tc_P;                   // partial product tiles [grid][slots][128][128]
  // column-maximum slots of the slicing passes ([4][128], zero at launch): three rotate, the fourth
  // collects the maxima the tcgen05 path gathers in its epilogue
  unsigned long long *colmax;
  // exact fixed-point sums of pattern terms (FAM_CSR with pattern terms, FAM_MF): Z copies of the
  // substep input and of the two Leja vectors ([nvec][dim] each), headroom bits of the row sums,
  // and whether every term is real-valued (then |Re (X w)_r| <= ||X||_inf max |Re w|)
  longlong2 *zc, *zw0, *zw1;
  longlong2 *zu;  // M4 in fixed point: copies of u_k, [nterms][nvec][dim]
  int zfix, zhb, zreal;  // zfix: 0 FP64, 1 fixed-point linear generators, 2 fixed-point M4
  int stg;               // FAM_CSR, zfix 1: rows read from shared-memory slots the TMA fills per tile
};
enum { FAM_GENERIC = 0, FAM_CSR = 1, FAM_MF = 2, FAM_DENSE = 3 };
// a.zfix selects the instantiation with fixed-point sums and products: 1 for linear generators
// (M2, Cf4, Cf4:3), 2 for M4 (which also needs a.zu); never with M6.
cudaError_t launch_persistent(const PersistArgs &a, int grid, int block, bool m6, cudaStream_t st);
inline int persistent_fixed_kernel(const PersistArgs &a, bool m6) {
  return (!m6 && (a.fam == FAM_CSR || a.fam == FAM_MF)) ? a.zfix : 0;
}
int persistent_block_size();
cudaError_t persistent_max_blocks_per_sm(int fam, bool m6, int zf, int *n, bool stg = false);
// dynamic shared memory of the staged-rows instantiation (two slots per warp)
size_t persistent_stage_smem_bytes();
// Sliced rows of a CSR term (rowptr, col, and for a product term its mantissas fval; fval null for a
// pattern term), dim rows: fills hbase [ceil(dim/32)+1], hcol/hval [32 sum_s w_s] and, if some row
// has a tail, tptr [dim+1], tcol/tval (allocated here with cudaMalloc; *ntail = tail entries).
// Rows of a slice longer than 24 entries keep their CSR order.
struct SlicedRows {
  int64_t *hbase = nullptr;
  int32_t *hcol = nullptr;
  long long *hval = nullptr;
  int64_t *tptr = nullptr;
  int32_t *tcol = nullptr;
  long long *tval = nullptr;
  int64_t nhead = 0, ntail = 0;
};
cudaError_t build_sliced_rows(const int64_t *rowptr, const int32_t *col, const long long *fval, int64_t dim,
                              SlicedRows *out, cudaStream_t st);
void free_sliced_rows(SlicedRows *s);
// count (device, zeroed by the caller) += the 32-row tiles (rows [32 t, 32 t + 32)) of the CSR terms
// T[0..nt-1] whose runs do not fit one staging slot; such tiles are read from global memory
cudaError_t launch_stage_misfits(const Term *T, int nt, int64_t dim, unsigned long long *count, cudaStream_t st);

// Dense family (dense terms, optionally with a matrix-free field term): rows of all vectors per block.
int dense_block_size();
int dense_rows_per_unit(bool tiled);
cudaError_t dense_max_blocks_per_sm(int *n);
// partials must hold 4 * grid * nvec + 4 * nvec doubles
cudaError_t launch_dense_persistent(const PersistArgs &a, bool real_valued, int grid, cudaStream_t st);
// Dense term (real parts Hr[e * rs]) -> 4 x 8-bit digits in the tiled layout at `digits`, row
// exponents at rexp.
cudaError_t launch_slice_dense_tc(const double *Hr, int rs, int64_t D, void *digits, int *rexp, cudaStream_t st);
size_t dense_tc_smem_bytes();
int dense_tc_chunk(int64_t D);  // K per exact chunk of the tcgen05 digit products
int dense_tc_slots(int ndense, int64_t D, int grid);

// Dense term (complex128, real parts used) -> bf16 digits [5][D][D] and row exponents [D].

// H (real parts Hr[e * rs]) -> FP32 (hi, lo) pairs, n entries.
cudaError_t launch_split_dense(const double *Hr, int rs, float2 *out, int64_t n, cudaStream_t st);

// Adjoint: the augmented-block Leja kernel for one exponential and its helpers (adjoint.cu).
struct AugArgs {
  int64_t dim;
  int nterms, kd, m_max, fam, lbits;
  double tol_rel, tol_abs;
  const Term *terms;
  const ExpRec *rec;       // the exponential's record
  const double2 *dd;       // its divided differences [m_max+1]
  const double *xi;
  const double2 *v;        // input state
  double2 *out_a;          // L(Omega, -i H_kd) v
  double2 *acur, *bcur, *anxt, *bnxt, *wa0, *wb0, *wa1, *wb1;
  double *partials;        // [2][grid][6]: two sums and four maxima per block
  GridBar *bar;
  Counters *counters;
  long long spin_limit_ns;
  const double *dlo, *dhi;
  // fixed-point arithmetic (as in PersistArgs): copies of the substep input (zca, zcb) and of the
  // ping-pong vectors of both blocks
  int zfix, zhb, zreal;
  longlong2 *zca, *zcb, *zwa0, *zwb0, *zwa1, *zwb1;
};
int aug_block_size();
cudaError_t aug_max_blocks_per_sm(int *n);
cudaError_t launch_aug_persistent(const AugArgs &a, int grid, cudaStream_t st);
cudaError_t launch_negate_records(const ExpRec *in, const double2 *din, ExpRec *out, double2 *dout, int64_t nexp,
                                  int m_max, cudaStream_t st);
cudaError_t launch_dot(const double2 *x, const double2 *y, int64_t n, double2 *out, cudaStream_t st);
cudaError_t launch_adjoint_contract(const double2 *G, const double2 *z, const Coeff *coeff, int variant, double t0,
                                    double h, int64_t nsteps, double *grad, int ng, cudaStream_t st);

// Diagonal tables of a matrix-free XXZ term (FAM_MF), split at bit lbits.
cudaError_t launch_xxz_diag_tables(const Term *t_dev, int nspins, int lbits, double *dlo, double *dhi, cudaStream_t st);

// Builders.
cudaError_t launch_build_xxz_csr(int nspins, const double *J, const double *hz, double delta, int64_t *rowptr,
                                 int32_t *col, double2 *val, cudaStream_t st);
cudaError_t launch_build_field_x_csr(int nspins, int64_t *rowptr, int32_t *col, double2 *val, cudaStream_t st);
cudaError_t launch_build_longrange_dense(int nspins, double alpha, const double *hz, double delta, double2 *H,
                                         cudaStream_t st);
cudaError_t launch_build_field_x_dense(int nspins, double2 *H, cudaStream_t st);

}  // namespace mg
