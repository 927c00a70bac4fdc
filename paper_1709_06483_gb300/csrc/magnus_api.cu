// Host implementation of the C ABI declared in include/magnus.h.  Argument checking, device
// allocation, and launching the kernels of setup_kernels.cu and leja_persistent.cu; no part of
// the method's arithmetic runs on the host.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "magnus_internal.cuh"

using namespace mg;

struct magnus_plan_s {
  int device = 0;
  int num_sms = 0;
  int max_blocks_per_sm = 0;             // persistent kernel of the plan's family, linear / M4 generators
  int max_blocks_m6 = 0;                 // its M6 instantiation
  int max_blocks_zf = 0;                 // its instantiation with fixed-point sums and products
  int max_blocks_zf4 = 0;                // and that of fixed-point M4
  int max_blocks_stg = 0;                // and that of the staged-rows fixed-point CSR instantiation
  bool staged = false;                   // fixed-point CSR linear generators read staged rows
  cudaStream_t stream = nullptr;
  int64_t dim = 0;
  int nterms = 0;
  magnus_options opt{};
  Term terms_host[kMaxTerms]{};
  double term_ab_host[2 * kMaxTerms]{};
  // device
  Term *terms = nullptr;
  Coeff *coeffs = nullptr;
  double *term_ab = nullptr;
  double *xi = nullptr;
  double *cand = nullptr;
  unsigned *counter = nullptr;
  GridBar *bar = nullptr;
  Counters *counters = nullptr;
  double *partials = nullptr;
  int64_t partials_cap = 0;
  double2 *alt = nullptr, *w0 = nullptr, *w1 = nullptr, *u = nullptr;
  ExpRec *recs = nullptr;
  double2 *dd = nullptr;
  int64_t recs_cap = 0;
  int *mlog = nullptr;
  int64_t mlog_cap = 0;
  int fam = FAM_GENERIC;
  int dense_blocks_per_sm = 0;
  bool dense_real = true;
  float2 *hsplit[kMaxTerms] = {nullptr, nullptr, nullptr, nullptr};
  float4 *sh_cur = nullptr, *sh_w0 = nullptr, *sh_w1 = nullptr, *sh_u = nullptr;
  unsigned long long *colmax = nullptr;  // [4][128]: 3 rotating slicing slots + the epilogue's
  double2 *m6 = nullptr;                 // M6 intermediate vectors [kM6Slots][nvec][dim], on first use
  // MAGNUS_TENSOR_SLICED on tcgen05 (linear generators)
  uint16_t *tc_hd = nullptr;             // dense-term digits, tiled [ndense][dim/128][dim/8][4][128][8]
  int *tc_eh = nullptr;                  // their row exponents [ndense][dim]
  uint16_t *tc_wd = nullptr;             // vector-set digits, tiled [3 + nterms][dim/8][4][128][8]
  int *tc_ex = nullptr;                  // column exponents [3 + nterms][128]
  double2 *tc_cacc = nullptr;            // M4 commutator sums [nvec][dim]
  double *tc_P = nullptr;                // partial tiles [grid][slots][128][128]
  int tc_grid = 0, tc_slots = 0, tc_ndense = 0;
  int tc_dslot[kMaxTerms] = {0, 0, 0, 0};
  Coeff coeff_host[kMaxTerms];           // staging of magnus_set_coeff
  int lbits = 0;
  double *dlo = nullptr, *dhi = nullptr;
  // exact fixed-point sums of pattern terms: Z copies of the substep input and the Leja vectors
  longlong2 *zc = nullptr, *zw0 = nullptr, *zw1 = nullptr;
  longlong2 *zu = nullptr;  // M4 in fixed point: copies of u_k, on first use
  unsigned *zmax = nullptr;  // magnus_apply in fixed point: max |x| per state (high words)
  double *rcopy[kMaxTerms] = {nullptr, nullptr, nullptr, nullptr};  // real parts of complex-stored real CSR terms
  long long *fval[kMaxTerms] = {nullptr, nullptr, nullptr, nullptr};  // fixed-point values of real CSR terms
  int16_t *fexp[kMaxTerms] = {nullptr, nullptr, nullptr, nullptr};    // and their row exponents
  SlicedRows sliced[kMaxTerms];                                         // sliced rows of those terms
  unsigned long long rowmax[kMaxTerms] = {0, 0, 0, 0};                // longest row of each real CSR term
  int zhb = 0;
  bool zreal = true;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;
};

namespace {

std::string g_global_err;

magnus_status set_err(magnus_plan_t p, magnus_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
magnus_status set_err(magnus_plan_t p, magnus_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (p) p->err = buf; else g_global_err = buf;
  return s;
}

#define CUDA_TRY(plan, expr)                                                                        \
  do {                                                                                              \
    cudaError_t e_ = (expr);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      return set_err(plan, e_ == cudaErrorMemoryAllocation ? MAGNUS_ENOMEM : MAGNUS_ECUDA, "%s: %s", \
                     #expr, cudaGetErrorString(e_));                                                \
    }                                                                                               \
  } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t count) {
  return cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
}

void free_plan(magnus_plan_t p) {
  if (!p) return;
  void *bufs[] = {p->terms, p->coeffs, p->term_ab, p->xi, p->cand, p->counter, p->bar, p->counters, p->partials,
                  p->alt, p->w0, p->w1, p->u, p->recs, p->dd, p->mlog, p->dlo, p->dhi,
                  p->hsplit[0], p->hsplit[1], p->hsplit[2], p->hsplit[3], p->sh_cur, p->sh_w0, p->sh_w1, p->sh_u,
                  p->colmax, p->m6,
                  p->tc_hd, p->tc_eh, p->tc_wd, p->tc_ex, p->tc_P, p->tc_cacc, p->zc, p->zw0, p->zw1, p->zu, p->zmax,
                  p->rcopy[0], p->rcopy[1], p->rcopy[2], p->rcopy[3], p->fval[0], p->fval[1], p->fval[2],
                  p->fval[3], p->fexp[0], p->fexp[1], p->fexp[2], p->fexp[3]};
  for (void *b : bufs)
    if (b) cudaFree(b);
  for (int k = 0; k < kMaxTerms; k++) free_sliced_rows(&p->sliced[k]);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  delete p;
}

// the layout the fixed-point CSR rows of a launch read (0: not a fixed-point CSR launch)
int row_layout_of_call(magnus_plan_t p, const PersistArgs &a) {
  if (!a.zfix || p->fam != FAM_CSR) return 0;
  if (a.stg) return MAGNUS_ROWS_STAGED;
  for (int k = 0; k < p->nterms; k++)
    if (p->terms_host[k].hbase) return MAGNUS_ROWS_SLICED;
  return MAGNUS_ROWS_CSR;
}

bool is_pow2_dim(int64_t dim, int nspins) {
  return nspins >= 1 && nspins <= kMaxSpins && dim == ((int64_t)1 << nspins);
}

magnus_status ensure_exp_capacity(magnus_plan_t p, int64_t nexp) {
  if (nexp <= p->recs_cap) return MAGNUS_OK;
  if (p->recs) cudaFree(p->recs);
  if (p->dd) cudaFree(p->dd);
  p->recs = nullptr;
  p->dd = nullptr;
  p->recs_cap = 0;
  CUDA_TRY(p, dalloc(&p->recs, (size_t)nexp));
  CUDA_TRY(p, dalloc(&p->dd, (size_t)nexp * (p->opt.m_max + 1)));
  p->recs_cap = nexp;
  return MAGNUS_OK;
}

magnus_status ensure_mlog(magnus_plan_t p, int64_t cap) {
  if (cap <= p->mlog_cap) return MAGNUS_OK;
  if (p->mlog) cudaFree(p->mlog);
  p->mlog = nullptr;
  p->mlog_cap = 0;
  CUDA_TRY(p, dalloc(&p->mlog, (size_t)cap));
  p->mlog_cap = cap;
  return MAGNUS_OK;
}

// bounded wait at a grid barrier: the plan's barrier_timeout_s, default 4 s (far above any
// legitimate wait: one Leja iteration takes well under 100 ms)
long long spin_limit(magnus_plan_t p) {
  const double s = p->opt.barrier_timeout_s > 0.0 ? p->opt.barrier_timeout_s : 4.0;
  return (long long)(s * 1e9);
}

// grid: nvec * gv blocks, all co-resident (cooperative launch)
void choose_grid(magnus_plan_t p, int *grid, int *gv, bool m6 = false, int zf = 0, bool stg = false) {
  const int per_sm = m6 ? p->max_blocks_m6
                        : (zf == 2 ? p->max_blocks_zf4
                                   : (zf == 1 ? (stg ? p->max_blocks_stg : p->max_blocks_zf) : p->max_blocks_per_sm));
  const int maxg = p->num_sms * std::max(1, per_sm);
  const int nv = p->opt.nvec;
  int per_vec = std::max(1, maxg / nv);
  if (p->opt.ctas > 0) per_vec = std::max(1, std::min(per_vec, p->opt.ctas / nv));
  // at least 256 rows (a row per thread) per block: for small chains fewer, fuller blocks make the
  // per-iteration barrier and reduction cheaper (measured on 12 to 16 spins)
  int64_t by_rows = std::max<int64_t>(1, (p->dim + 255) / 256);
  if (p->opt.ctas <= 0) per_vec = (int)std::min<int64_t>(per_vec, by_rows);
  *gv = per_vec;
  *grid = per_vec * nv;
}

magnus_status run_persistent(magnus_plan_t p, void *psi, int64_t nexp, magnus_stats *stats, bool m6 = false,
                             bool m4 = false) {
  int grid, gv;
  size_t need;
  if (p->fam == FAM_DENSE) {
    const bool tiled = p->opt.nvec > 1 || p->opt.precision != MAGNUS_FP64;
    const int64_t units = (p->dim + dense_rows_per_unit(tiled) - 1) / dense_rows_per_unit(tiled);
    const int64_t maxg = (int64_t)p->num_sms * std::max(1, p->dense_blocks_per_sm);
    // the warp-per-row kernel handles 8 rows per block pass; give each block at least 8 rows
    const int64_t want = tiled ? units : (units + 7) / 8;
    grid = (int)std::max<int64_t>(1, std::min<int64_t>(p->opt.ctas > 0 ? p->opt.ctas : maxg, std::min(maxg, want)));
    gv = grid;
    need = (size_t)4 * grid * p->opt.nvec + (size_t)4 * p->opt.nvec;
  } else {
    choose_grid(p, &grid, &gv, m6, (p->zc != nullptr && !m6) ? (m4 ? 2 : 1) : 0, p->staged && !m6 && !m4);
    need = (size_t)8 * grid;  // two slots x grid x (two sums, two maxima)
  }
  if ((int64_t)need > p->partials_cap) {
    if (p->partials) cudaFree(p->partials);
    p->partials = nullptr;
    p->partials_cap = 0;
    CUDA_TRY(p, dalloc(&p->partials, need));
    p->partials_cap = (int64_t)need;
  }
  int64_t want_log = (stats && stats->m_log && stats->m_log_cap > 0) ? stats->m_log_cap : 0;
  if (want_log) {
    magnus_status s = ensure_mlog(p, want_log);
    if (s != MAGNUS_OK) return s;
  }
  CUDA_TRY(p, cudaMemsetAsync(p->bar, 0, sizeof(GridBar), p->stream));
  CUDA_TRY(p, cudaMemsetAsync(p->counters, 0, sizeof(Counters), p->stream));
  if (p->colmax) CUDA_TRY(p, cudaMemsetAsync(p->colmax, 0, sizeof(unsigned long long) * 4 * 128, p->stream));
  PersistArgs a{};
  a.dim = p->dim;
  a.nvec = p->opt.nvec;
  a.nterms = p->nterms;
  a.gv = gv;
  a.m_max = p->opt.m_max;
  a.nexp = nexp;
  a.tol_rel = p->opt.tol_rel;
  a.tol_abs = p->opt.tol_abs;
  a.norm_check = p->opt.norm_check;
  a.terms = p->terms;
  a.recs = p->recs;
  a.dd = p->dd;
  a.xi = p->xi;
  a.psi = (double2 *)psi;
  a.alt = p->alt;
  a.w0 = p->w0;
  a.w1 = p->w1;
  a.u = p->u;
  a.partials = p->partials;
  a.bar = p->bar;
  a.counters = p->counters;
  a.mlog = want_log ? p->mlog : nullptr;
  a.mlog_cap = want_log;
  a.spin_limit_ns = spin_limit(p);
  a.skip_arrival = p->opt.test_skip_arrival;
  a.fam = p->fam;
  a.lbits = p->lbits;
  a.dlo = p->dlo;
  a.dhi = p->dhi;
  a.split = p->opt.precision == MAGNUS_FP32_SPLIT;
  for (int k = 0; k < kMaxTerms; k++) a.hsplit[k] = p->hsplit[k];
  a.sh_cur = p->sh_cur;
  a.sh_w0 = p->sh_w0;
  a.sh_w1 = p->sh_w1;
  a.sh_u = p->sh_u;
  const bool tensor = p->opt.precision == MAGNUS_TENSOR_SLICED;
  a.tc = tensor ? (m4 ? 2 : 1) : 0;
  if (a.tc) {
    if (p->tc_grid != grid) {  // partial tiles for this grid
      if (p->tc_P) cudaFree(p->tc_P);
      p->tc_P = nullptr;
      p->tc_grid = 0;
      p->tc_slots = dense_tc_slots(p->tc_ndense, p->dim, grid);
      CUDA_TRY(p, dalloc(&p->tc_P, (size_t)grid * p->tc_slots * 128 * 128));
      p->tc_grid = grid;
    }
    a.tc_ndense = p->tc_ndense;
    a.tc_slots = p->tc_slots;
    a.tc_T = (int)(p->dim / 128);
    a.tc_N = (long long)p->tc_ndense * a.tc_T * (p->dim / dense_tc_chunk(p->dim));
    a.tc_spins = 1ll << 26;
    for (int k = 0; k < kMaxTerms; k++) a.tc_dslot[k] = p->tc_dslot[k];
    a.tc_hd = p->tc_hd;
    a.tc_eh = p->tc_eh;
    a.tc_wd = p->tc_wd;
    a.tc_ex = p->tc_ex;
    a.tc_P = p->tc_P;
    a.tc_cacc = p->tc_cacc;
  }
  a.colmax = p->colmax;
  a.m6 = p->m6;
  a.zfix = (p->zc != nullptr && !m6) ? (m4 ? 2 : 1) : 0;  // fixed-point linear generators (1) or M4 (2)
  if (a.zfix == 2 && !p->zu) CUDA_TRY(p, dalloc(&p->zu, (size_t)p->nterms * p->dim * p->opt.nvec));
  a.zu = p->zu;
  a.zc = p->zc;
  a.zw0 = p->zw0;
  a.zw1 = p->zw1;
  a.zhb = p->zhb;
  a.zreal = p->zreal;
  a.stg = p->staged && a.zfix == 1 && p->fam == FAM_CSR;
  CUDA_TRY(p, cudaEventRecord(p->ev0, p->stream));
  if (p->fam == FAM_DENSE) {
    NvtxRange nr("k_dense_persistent launch");
    CUDA_TRY(p, launch_dense_persistent(a, p->dense_real, grid, p->stream));
  } else {
    NvtxRange nr("k_magnus_persistent launch");
    CUDA_TRY(p, launch_persistent(a, grid, persistent_block_size(), m6, p->stream));
  }
  CUDA_TRY(p, cudaEventRecord(p->ev1, p->stream));
  Counters c{};
  CUDA_TRY(p, cudaMemcpyAsync(&c, p->counters, sizeof c, cudaMemcpyDeviceToHost, p->stream));
  if (want_log) {
    std::vector<int> tmp((size_t)want_log, 0);
    CUDA_TRY(p, cudaMemcpyAsync(tmp.data(), p->mlog, sizeof(int) * want_log, cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    memcpy(stats->m_log, tmp.data(), sizeof(int) * want_log);
  } else {
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
  }
  if (stats) {
    stats->n_exp = c.n_exp;
    stats->n_substeps = c.n_substeps;
    stats->n_matvec = c.n_matvec;
    stats->n_termapply = c.n_termapply;
    stats->max_m = c.max_m;
    stats->status = c.status;
    float ms = 0.f;
    CUDA_TRY(p, cudaEventElapsedTime(&ms, p->ev0, p->ev1));
    stats->kernel_ms = ms;
    stats->grid = grid;
    stats->block = p->fam == FAM_DENSE ? dense_block_size() : persistent_block_size();
    stats->fixed_sums = a.zfix != 0;
    stats->row_layout = row_layout_of_call(p, a);
    double drift;
    memcpy(&drift, &c.max_drift, sizeof drift);
    stats->norm_drift = drift;
  }
  if (c.status != MAGNUS_OK) {
    const char *what = c.status == MAGNUS_ENOCONV      ? "Leja interpolation did not converge within m_max"
                       : c.status == MAGNUS_ENONFINITE ? "non-finite norm in the Leja iteration"
                       : c.status == MAGNUS_ETIMEOUT   ? "grid barrier wait timed out"
                       : c.status == MAGNUS_EDRIFT     ? "a substep changed the state's norm beyond options.norm_check"
                                                       : "device error";
    return set_err(p, (magnus_status)c.status, "%s", what);
  }
  return MAGNUS_OK;
}

}  // namespace

namespace mg {
// Error text of the entry points that take no plan (read back with magnus_last_error(NULL)).
void noalloc_set_error(const char *msg) { g_global_err = msg; }
}  // namespace mg

extern "C" {

MAGNUS_API magnus_status magnus_real_parts(const void *z, int64_t n, double *out, void *stream) {
  if (n < 0 || (n > 0 && (!z || !out))) return set_err(nullptr, MAGNUS_EINVAL, "real_parts: bad arguments");
  if (n == 0) return MAGNUS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int *flag = nullptr;
  CUDA_TRY(nullptr, dalloc(&flag, 1));
  int fh = 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e == cudaSuccess) e = launch_real_parts((const double2 *)z, n, out, flag, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&fh, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(flag);
  CUDA_TRY(nullptr, e);
  if (fh) return set_err(nullptr, MAGNUS_EINVAL, "real_parts: some imaginary part is nonzero");
  return MAGNUS_OK;
}


const char *magnus_status_string(magnus_status s) {
  switch (s) {
    case MAGNUS_OK: return "MAGNUS_OK";
    case MAGNUS_EINVAL: return "MAGNUS_EINVAL";
    case MAGNUS_ENOMEM: return "MAGNUS_ENOMEM";
    case MAGNUS_ECUDA: return "MAGNUS_ECUDA";
    case MAGNUS_ENOCONV: return "MAGNUS_ENOCONV";
    case MAGNUS_ENONFINITE: return "MAGNUS_ENONFINITE";
    case MAGNUS_ETIMEOUT: return "MAGNUS_ETIMEOUT";
    case MAGNUS_EDRIFT: return "MAGNUS_EDRIFT";
  }
  return "MAGNUS_UNKNOWN";
}

const char *magnus_last_error(magnus_plan_t plan) { return plan ? plan->err.c_str() : g_global_err.c_str(); }

magnus_status magnus_plan_create(magnus_plan_t *out, int64_t dim, int32_t nterms, const magnus_term *terms,
                                 const magnus_coeff *coeffs, const magnus_options *opt, void *stream) {
  if (!out) return set_err(nullptr, MAGNUS_EINVAL, "plan pointer is null");
  *out = nullptr;
  if (dim < 1 || dim > ((int64_t)1 << 31)) return set_err(nullptr, MAGNUS_EINVAL, "dim %lld out of range", (long long)dim);
  if (nterms < 1 || nterms > kMaxTerms) return set_err(nullptr, MAGNUS_EINVAL, "nterms must be 1..%d", kMaxTerms);
  if (!terms || !coeffs) return set_err(nullptr, MAGNUS_EINVAL, "terms/coeffs are null");
  magnus_options o{1e-10, 1e-10, 4.0, 100, 1, 0, MAGNUS_FP64};
  o.fixed_sums = 1;
  if (opt) o = *opt;
  if (!(o.tol_rel >= 0.0) || !(o.tol_abs >= 0.0) || !(o.tol_rel + o.tol_abs > 0.0))
    return set_err(nullptr, MAGNUS_EINVAL, "tolerances must be >= 0 and not both 0");
  if (o.fixed_sums != 0 && o.fixed_sums != 1) return set_err(nullptr, MAGNUS_EINVAL, "fixed_sums must be 0 or 1");
  if (o.row_layout < MAGNUS_ROWS_AUTO || o.row_layout > MAGNUS_ROWS_SLICED)
    return set_err(nullptr, MAGNUS_EINVAL, "row_layout must be MAGNUS_ROWS_AUTO, _STAGED, _CSR or _SLICED");
  if (o.plain_values != 0 && o.plain_values != 1) return set_err(nullptr, MAGNUS_EINVAL, "plain_values must be 0 or 1");
  if (!(o.norm_check >= 0.0) || !std::isfinite(o.norm_check))
    return set_err(nullptr, MAGNUS_EINVAL, "norm_check must be finite and >= 0 (0 = off)");
  if (!(o.rho_max > 0.0)) return set_err(nullptr, MAGNUS_EINVAL, "rho_max must be > 0");
  if (!(o.barrier_timeout_s >= 0.0) || o.barrier_timeout_s > 600.0)
    return set_err(nullptr, MAGNUS_EINVAL, "barrier_timeout_s must be in [0, 600]");
  if (o.m_max < 2 || o.m_max > kMmaxLimit) return set_err(nullptr, MAGNUS_EINVAL, "m_max must be 2..%d", kMmaxLimit);
  if (o.nvec < 1 || o.nvec > 64) return set_err(nullptr, MAGNUS_EINVAL, "nvec must be 1..64");
  if (o.interval != MAGNUS_INTERVAL_GERSHGORIN && o.interval != MAGNUS_INTERVAL_LANCZOS)
    return set_err(nullptr, MAGNUS_EINVAL, "interval must be MAGNUS_INTERVAL_GERSHGORIN or MAGNUS_INTERVAL_LANCZOS");
  if (o.precision != MAGNUS_FP64 && o.precision != MAGNUS_FP32_SPLIT && o.precision != MAGNUS_TENSOR_SLICED)
    return set_err(nullptr, MAGNUS_EINVAL, "precision must be MAGNUS_FP64, MAGNUS_FP32_SPLIT or MAGNUS_TENSOR_SLICED");
  for (int k = 0; k < nterms; k++) {
    const magnus_term &t = terms[k];
    const magnus_coeff &c = coeffs[k];
    if (c.nmodes < 0 || c.nmodes > kMaxModes || (c.nmodes > 0 && !c.om))
      return set_err(nullptr, MAGNUS_EINVAL, "coefficient %d: nmodes must be 0..%d with om given", k, kMaxModes);
    switch (t.kind) {
      case MAGNUS_TERM_CSR:
        if (!t.rowptr || !t.col || !t.val || t.nnz < 0)
          return set_err(nullptr, MAGNUS_EINVAL, "term %d: CSR arrays missing", k);
        if (((uintptr_t)t.val) % 16) return set_err(nullptr, MAGNUS_EINVAL, "term %d: CSR values must be 16-byte aligned", k);
        break;
      case MAGNUS_TERM_CSR_REAL:
        if (!t.rowptr || !t.col || !t.val || t.nnz < 0)
          return set_err(nullptr, MAGNUS_EINVAL, "term %d: CSR arrays missing", k);
        if (((uintptr_t)t.val) % 8) return set_err(nullptr, MAGNUS_EINVAL, "term %d: real CSR values must be 8-byte aligned", k);
        break;
      case MAGNUS_TERM_DENSE:
      case MAGNUS_TERM_DENSE_REAL:
        if (!t.val) return set_err(nullptr, MAGNUS_EINVAL, "term %d: dense matrix missing", k);
        if (((uintptr_t)t.val) % (t.kind == MAGNUS_TERM_DENSE ? 16 : 8))
          return set_err(nullptr, MAGNUS_EINVAL, "term %d: dense values misaligned", k);
        if (dim > 65536) return set_err(nullptr, MAGNUS_EINVAL, "term %d: dense terms need dim <= 65536", k);
        break;
      case MAGNUS_TERM_XXZ:
        if (!is_pow2_dim(dim, t.nspins) || t.nspins < 2 || !t.J || !t.hz)
          return set_err(nullptr, MAGNUS_EINVAL, "term %d: XXZ needs dim = 2^nspins, nspins >= 2, J and hz", k);
        break;
      case MAGNUS_TERM_FIELD_X:
        if (!is_pow2_dim(dim, t.nspins)) return set_err(nullptr, MAGNUS_EINVAL, "term %d: FIELD_X needs dim = 2^nspins", k);
        break;
      default: return set_err(nullptr, MAGNUS_EINVAL, "term %d: unknown kind %d", k, t.kind);
    }
  }

  magnus_plan_t p = new magnus_plan_s();
  p->stream = (cudaStream_t)stream;
  p->dim = dim;
  p->nterms = nterms;
  p->opt = o;
  auto fail = [&](magnus_status s) {
    g_global_err = p->err;
    free_plan(p);
    return s;
  };
#define PLAN_TRY(expr)                                            \
  do {                                                            \
    cudaError_t e_ = (expr);                                      \
    if (e_ != cudaSuccess) {                                      \
      set_err(p, e_ == cudaErrorMemoryAllocation ? MAGNUS_ENOMEM : MAGNUS_ECUDA, "%s: %s", #expr, \
              cudaGetErrorString(e_));                            \
      return fail(e_ == cudaErrorMemoryAllocation ? MAGNUS_ENOMEM : MAGNUS_ECUDA); \
    }                                                             \
  } while (0)

  PLAN_TRY(cudaGetDevice(&p->device));
  PLAN_TRY(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
  PLAN_TRY(cudaEventCreate(&p->ev0));
  PLAN_TRY(cudaEventCreate(&p->ev1));

  std::vector<Coeff> ch(nterms);
  for (int k = 0; k < nterms; k++) {
    const magnus_term &t = terms[k];
    Term &T = p->terms_host[k];
    memset(&T, 0, sizeof T);
    set_term_storage(T, t);
    T.nspins = t.nspins;
    T.nnz = t.nnz;
    T.rowptr = t.rowptr;
    T.col = t.col;
    T.delta = t.delta;
    if (t.kind == MAGNUS_TERM_XXZ) {
      for (int i = 0; i < t.nspins - 1; i++) T.J[i] = t.J[i];
      for (int i = 0; i < t.nspins; i++) T.hz[i] = t.hz[i];
    }
    Coeff &C = ch[k];
    memset(&C, 0, sizeof C);
    C.a0 = coeffs[k].a0;
    C.nmodes = coeffs[k].nmodes;
    for (int m = 0; m < C.nmodes; m++) {
      C.ac[m] = coeffs[k].ac ? coeffs[k].ac[m] : 0.0;
      C.as[m] = coeffs[k].as ? coeffs[k].as[m] : 0.0;
      C.om[m] = coeffs[k].om[m];
    }
  }
  const size_t nd = (size_t)dim * o.nvec;
  PLAN_TRY(dalloc(&p->terms, nterms));
  PLAN_TRY(dalloc(&p->coeffs, nterms));
  PLAN_TRY(dalloc(&p->term_ab, 2 * nterms));
  PLAN_TRY(dalloc(&p->xi, o.m_max + 1));
  PLAN_TRY(dalloc(&p->cand, 2 * (o.m_max + 1)));
  PLAN_TRY(dalloc(&p->counter, 1));
  PLAN_TRY(dalloc(&p->bar, 1));
  PLAN_TRY(dalloc(&p->counters, 1));
  PLAN_TRY(dalloc(&p->alt, nd));
  PLAN_TRY(dalloc(&p->w0, nd));
  PLAN_TRY(dalloc(&p->w1, nd));
  PLAN_TRY(dalloc(&p->u, nd * nterms));
  PLAN_TRY(cudaMemcpyAsync(p->coeffs, ch.data(), sizeof(Coeff) * nterms, cudaMemcpyHostToDevice, p->stream));

  // real-valued CSR values: only the real parts need multiplying
  int *flag = nullptr;
  PLAN_TRY(dalloc(&flag, kMaxTerms));
  PLAN_TRY(cudaMemsetAsync(flag, 0, sizeof(int) * kMaxTerms, p->stream));
  for (int k = 0; k < nterms; k++) {
    if (p->terms_host[k].rs == 1) continue;  // real storage
    if (p->terms_host[k].kind == MAGNUS_TERM_CSR && p->terms_host[k].nnz > 0)
      PLAN_TRY(launch_imag_check(p->terms_host[k].val, p->terms_host[k].nnz, flag + k, p->stream));
    if (p->terms_host[k].kind == MAGNUS_TERM_DENSE)
      PLAN_TRY(launch_imag_check(p->terms_host[k].val, dim * dim, flag + k, p->stream));
  }
  int fh[kMaxTerms] = {0, 0, 0, 0};
  PLAN_TRY(cudaMemcpyAsync(fh, flag, sizeof fh, cudaMemcpyDeviceToHost, p->stream));
  PLAN_TRY(cudaStreamSynchronize(p->stream));
  cudaFree(flag);
  // (plain_values: complex-stored values stay complex, multiplied in place as complex128)
  for (int k = 0; k < nterms; k++)
    p->terms_host[k].real_valued =
        (p->terms_host[k].kind == MAGNUS_TERM_CSR || p->terms_host[k].kind == MAGNUS_TERM_DENSE) && !fh[k] &&
        !(o.plain_values && p->terms_host[k].rs == 2);
  for (int k = 0; k < nterms; k++)
    if (p->terms_host[k].kind == MAGNUS_TERM_DENSE && !p->terms_host[k].real_valued) p->dense_real = false;
  // real-valued CSR terms stored as complex128: a compact float64 copy of the real parts (the only
  // part any kernel multiplies), so that a pass reads 8 B per value instead of the 16 B a complex
  // value's sectors carry
  for (int k = 0; k < nterms; k++) {
    Term &T = p->terms_host[k];
    if (T.kind != MAGNUS_TERM_CSR || !T.real_valued || T.rs != 2 || T.nnz <= 0) continue;
    int *rflag = nullptr;
    PLAN_TRY(dalloc(&p->rcopy[k], (size_t)T.nnz));
    PLAN_TRY(dalloc(&rflag, 1));
    PLAN_TRY(launch_real_parts(T.val, T.nnz, p->rcopy[k], rflag, p->stream));
    PLAN_TRY(cudaStreamSynchronize(p->stream));
    cudaFree(rflag);
    T.rv = p->rcopy[k];
    T.rs = 1;
  }
  // pattern terms: real CSR terms with one stored value (summed in fixed point when fixed_sums)
  {
    int *pflag = nullptr;
    unsigned long long *prow = nullptr;
    PLAN_TRY(dalloc(&pflag, kMaxTerms));
    PLAN_TRY(dalloc(&prow, kMaxTerms));
    PLAN_TRY(cudaMemsetAsync(pflag, 0, sizeof(int) * kMaxTerms, p->stream));
    PLAN_TRY(cudaMemsetAsync(prow, 0, sizeof(unsigned long long) * kMaxTerms, p->stream));
    double v0[kMaxTerms] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < nterms; k++) {
      const Term &T = p->terms_host[k];
      if (T.kind != MAGNUS_TERM_CSR || !T.real_valued || T.nnz <= 0) continue;
      PLAN_TRY(launch_pattern_check(T.rowptr, T.rv, T.rs, dim, pflag + k, prow + k, p->stream));
      PLAN_TRY(cudaMemcpyAsync(v0 + k, T.rv, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    }
    int pf[kMaxTerms] = {1, 1, 1, 1};
    unsigned long long *pr = p->rowmax;
    PLAN_TRY(cudaMemcpyAsync(pf, pflag, sizeof pf, cudaMemcpyDeviceToHost, p->stream));
    PLAN_TRY(cudaMemcpyAsync(pr, prow, sizeof(unsigned long long) * kMaxTerms, cudaMemcpyDeviceToHost, p->stream));
    PLAN_TRY(cudaStreamSynchronize(p->stream));
    cudaFree(pflag);
    cudaFree(prow);
    for (int k = 0; k < nterms; k++) {
      Term &T = p->terms_host[k];
      if (T.kind != MAGNUS_TERM_CSR || !T.real_valued || T.nnz <= 0 || (pf[k] & 1)) continue;
      int bits = 0;
      while (bits < 40 && (1ull << bits) < pr[k]) bits++;
      T.pattern = 1;
      T.pbits = bits;
      T.pval = v0[k];
      T.plen = (pf[k] & 2) || pr[k] > (1u << 20) ? 0 : (int)pr[k];
    }
  }
  PLAN_TRY(cudaMemcpyAsync(p->terms, p->terms_host, sizeof(Term) * nterms, cudaMemcpyHostToDevice, p->stream));

  // operator family of the persistent kernel
  {
    bool all_csr = true;
    for (int k = 0; k < nterms; k++) all_csr &= (p->terms_host[k].kind == MAGNUS_TERM_CSR);
    const bool mf = nterms == 2 && p->terms_host[0].kind == MAGNUS_TERM_XXZ &&
                    p->terms_host[1].kind == MAGNUS_TERM_FIELD_X && p->terms_host[0].nspins == p->terms_host[1].nspins;
    if (all_csr) p->fam = FAM_CSR;
    bool any_dense = false, dense_ok = true;
    for (int k = 0; k < nterms; k++) {
      any_dense |= p->terms_host[k].kind == MAGNUS_TERM_DENSE;
      dense_ok &= p->terms_host[k].kind == MAGNUS_TERM_DENSE || p->terms_host[k].kind == MAGNUS_TERM_FIELD_X;
    }
    if (any_dense && !dense_ok) {
      set_err(p, MAGNUS_EINVAL, "dense terms can only be combined with MAGNUS_TERM_FIELD_X terms");
      return fail(MAGNUS_EINVAL);
    }
    if (any_dense) {
      p->fam = FAM_DENSE;
      PLAN_TRY(dense_max_blocks_per_sm(&p->dense_blocks_per_sm));
    }
    if (o.precision == MAGNUS_FP32_SPLIT) {
      if (p->fam != FAM_DENSE || !p->dense_real) {
        set_err(p, MAGNUS_EINVAL, "MAGNUS_FP32_SPLIT needs real-valued dense terms");
        return fail(MAGNUS_EINVAL);
      }
      for (int k = 0; k < nterms; k++)
        if (p->terms_host[k].kind == MAGNUS_TERM_DENSE) {
          PLAN_TRY(dalloc(&p->hsplit[k], (size_t)dim * dim));
          PLAN_TRY(launch_split_dense(p->terms_host[k].rv, p->terms_host[k].rs, p->hsplit[k], dim * dim, p->stream));
        }
      PLAN_TRY(dalloc(&p->sh_cur, nd));
      PLAN_TRY(dalloc(&p->sh_w0, nd));
      PLAN_TRY(dalloc(&p->sh_w1, nd));
      PLAN_TRY(dalloc(&p->sh_u, nd * nterms));
    }
    if (o.precision == MAGNUS_TENSOR_SLICED) {
      if (p->fam != FAM_DENSE || !p->dense_real || dim % 128 != 0) {
        set_err(p, MAGNUS_EINVAL, "MAGNUS_TENSOR_SLICED needs real-valued dense terms and dim a multiple of 128");
        return fail(MAGNUS_EINVAL);
      }
      // tcgen05 path: 4 x 8-bit digits of every dense term and of the vector sets (substep input,
      // w0, w1 and, for M4, one u_k per term), tiled in the order the tensor cores read them
      // (columns beyond 2 nvec stay zero)
      int nden = 0;
      for (int k = 0; k < nterms; k++)
        if (p->terms_host[k].kind == MAGNUS_TERM_DENSE) p->tc_dslot[k] = nden++;
      p->tc_ndense = nden;
      const size_t dd = (size_t)dim * dim;
      PLAN_TRY(dalloc(&p->tc_hd, (size_t)nden * 4 * dd));
      PLAN_TRY(dalloc(&p->tc_eh, (size_t)nden * dim));
      for (int k = 0; k < nterms; k++)
        if (p->terms_host[k].kind == MAGNUS_TERM_DENSE)
          PLAN_TRY(launch_slice_dense_tc(p->terms_host[k].rv, p->terms_host[k].rs, dim, p->tc_hd + (size_t)p->tc_dslot[k] * 4 * dd,
                                         p->tc_eh + (size_t)p->tc_dslot[k] * dim, p->stream));
      const size_t wset = (size_t)4 * 128 * dim;
      const size_t nsets = 3 + (size_t)nterms;
      PLAN_TRY(dalloc(&p->tc_wd, nsets * wset));
      PLAN_TRY(dalloc(&p->tc_ex, nsets * 128));
      PLAN_TRY(cudaMemsetAsync(p->tc_wd, 0, sizeof(uint16_t) * nsets * wset, p->stream));
      PLAN_TRY(cudaMemsetAsync(p->tc_ex, 0, sizeof(int) * nsets * 128, p->stream));
      PLAN_TRY(dalloc(&p->tc_cacc, nd));
      PLAN_TRY(dalloc(&p->colmax, (size_t)4 * 128));
    }
    if (mf) {
      const int n = p->terms_host[0].nspins;
      p->fam = FAM_MF;
      p->lbits = std::max(1, n / 2);
      PLAN_TRY(dalloc(&p->dlo, (size_t)1 << (p->lbits + 1)));
      PLAN_TRY(dalloc(&p->dhi, (size_t)1 << (n - p->lbits)));
      PLAN_TRY(launch_xxz_diag_tables(p->terms, n, p->lbits, p->dlo, p->dhi, p->stream));
    }
  }

  if (p->fam != FAM_DENSE) {
    PLAN_TRY(persistent_max_blocks_per_sm(p->fam, false, 0, &p->max_blocks_per_sm));
    PLAN_TRY(persistent_max_blocks_per_sm(p->fam, true, 0, &p->max_blocks_m6));
    PLAN_TRY(persistent_max_blocks_per_sm(p->fam, false, 1, &p->max_blocks_zf));
    PLAN_TRY(persistent_max_blocks_per_sm(p->fam, false, 2, &p->max_blocks_zf4));
  }

  // Gershgorin enclosures (one pass over every term) and the Leja points
  const int gblk = std::max(1, std::min(p->num_sms * 4, (int)((dim + 255) / 256)));
  double *gscratch = nullptr;
  PLAN_TRY(dalloc(&gscratch, 2 * gblk));
  for (int k = 0; k < nterms; k++)
    PLAN_TRY(launch_gershgorin(p->terms + k, p->terms_host[k], dim, gscratch, gblk, p->term_ab + 2 * k, p->stream));
  double gab[2 * kMaxTerms] = {0.0};  // the Gershgorin enclosures, before Lanczos narrows them
  PLAN_TRY(cudaMemcpyAsync(gab, p->term_ab, sizeof(double) * 2 * nterms, cudaMemcpyDeviceToHost, p->stream));
  if (o.interval == MAGNUS_INTERVAL_LANCZOS)
    for (int k = 0; k < nterms; k++)
      PLAN_TRY(lanczos_interval(p->terms + k, p->terms_host[k], dim, kLanczosSteps, p->term_ab + 2 * k, p->stream));
  PLAN_TRY(launch_leja_points(p->xi, o.m_max, p->cand, p->counter, p->stream));
  PLAN_TRY(cudaMemcpyAsync(p->term_ab_host, p->term_ab, sizeof(double) * 2 * nterms, cudaMemcpyDeviceToHost, p->stream));
  PLAN_TRY(cudaStreamSynchronize(p->stream));
  cudaFree(gscratch);
  for (int k = 0; k < nterms; k++)
    if (!(p->term_ab_host[2 * k] <= p->term_ab_host[2 * k + 1])) {
      set_err(p, MAGNUS_EINVAL, "term %d: spectral enclosure is not finite (NaN/Inf in the matrix?)", k);
      return fail(MAGNUS_EINVAL);
    }
  // ||H_k||_inf = max_r (|Re H_rr| + sum_{c != r} |H_rc|) = max(|a_k|, |b_k|) of the Gershgorin
  // enclosure (real diagonal), widened by 2^-40 for its rounding
  for (int k = 0; k < nterms; k++)
    p->terms_host[k].gnorm = std::max(std::fabs(gab[2 * k]), std::fabs(gab[2 * k + 1])) * (1.0 + 0x1p-40);
  // fixed-point arithmetic: CSR plans with a pattern term (exact sums) or another real CSR term
  // (products of 62-bit value mantissas and Z), and the matrix-free chain's field
  if (o.fixed_sums && (p->fam == FAM_CSR || p->fam == FAM_MF)) {
    int zhb = 0;  // headroom bits of Z: |Z| < 2^(62 - zhb)
    bool any = false;
    if (p->fam == FAM_MF) {
      Term &F = p->terms_host[1];
      int bits = 0;
      while ((1 << bits) < F.nspins) bits++;
      F.pattern = 1;
      F.pbits = bits;
      F.pval = 1.0;
      zhb = bits + 1;
      any = true;
    } else {
      for (int k = 0; k < nterms; k++) {
        Term &T = p->terms_host[k];
        if (!T.real_valued || T.nnz <= 0) continue;
        int bits = 0;  // ceil(log2(longest row))
        while (bits < 40 && (1ull << bits) < p->rowmax[k]) bits++;
        if (bits > 30) continue;
        if (T.pattern) {
          zhb = std::max(zhb, bits + 1);  // row sums of up to 2^bits entries of |Z| < 2^(61-bits) stay below 2^61
          any = true;
        } else {
          // products: |fval Z| / 2^64 < 2^(60 - zhb); rows of up to 2^bits entries stay below 2^63
          zhb = std::max(zhb, bits - 2);
          any = true;
        }
      }
      zhb = std::max(zhb, 1);
    }
    if (any) {
      p->zhb = zhb;
      for (int k = 0; k < nterms; k++) p->zreal &= p->fam == FAM_MF || p->terms_host[k].real_valued != 0;
      PLAN_TRY(dalloc(&p->zc, nd));
      PLAN_TRY(dalloc(&p->zw0, nd));
      PLAN_TRY(dalloc(&p->zw1, nd));
      PLAN_TRY(dalloc(&p->zmax, o.nvec));
      // fixed-point values of the real CSR terms that are not patterns
      if (p->fam == FAM_CSR)
        for (int k = 0; k < nterms; k++) {
          Term &T = p->terms_host[k];
          if (!T.real_valued || T.pattern || T.nnz <= 0 || p->rowmax[k] > (1ull << 30)) continue;
          int *wide = nullptr;
          PLAN_TRY(dalloc(&p->fval[k], (size_t)T.nnz));
          PLAN_TRY(dalloc(&p->fexp[k], (size_t)dim));
          PLAN_TRY(dalloc(&wide, 1));
          PLAN_TRY(cudaMemsetAsync(wide, 0, sizeof(int), p->stream));
          PLAN_TRY(launch_fixed_values(T.rowptr, T.rv, T.rs, dim, p->fval[k], p->fexp[k], wide, p->stream));
          int wh = 0;
          PLAN_TRY(cudaMemcpyAsync(&wh, wide, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
          PLAN_TRY(cudaStreamSynchronize(p->stream));
          cudaFree(wide);
          if (wh) {  // values beyond the scales' range: this term keeps FP64 products
            cudaFree(p->fval[k]);
            cudaFree(p->fexp[k]);
            p->fval[k] = nullptr;
            p->fexp[k] = nullptr;
            continue;
          }
          T.fval = p->fval[k];
          T.fexp = p->fexp[k];
        }
    }
  }
  PLAN_TRY(cudaMemcpyAsync(p->terms, p->terms_host, sizeof(Term) * nterms, cudaMemcpyHostToDevice, p->stream));
  // staged rows: every term a pattern or a product term with 16-byte aligned arrays, and at most
  // 1/64 of the 32-row tiles too large for a slot
  // row layout of the fixed-point CSR rows: the CSR arrays as given by default (MAGNUS_ROWS_AUTO:
  // measured fastest on the 20-spin chain, 694 steps/s against 552 sliced and 468 staged)
  const int layout = o.row_layout == MAGNUS_ROWS_AUTO ? MAGNUS_ROWS_CSR : o.row_layout;
  if (p->fam == FAM_CSR && p->zc && (layout == MAGNUS_ROWS_SLICED || layout == MAGNUS_ROWS_STAGED) &&
      dim <= ((int64_t)1 << 28)) {
    bool changed = false;
    for (int k = 0; k < nterms; k++) {
      Term &T = p->terms_host[k];
      if (!(T.pattern || T.fval) || T.nnz <= 0) continue;
      PLAN_TRY(build_sliced_rows(T.rowptr, T.col, T.fval, dim, &p->sliced[k], p->stream));
      const SlicedRows &S = p->sliced[k];
      T.hbase = S.hbase;
      T.hcol = S.hcol;
      T.hval = S.hval;
      T.tptr = S.tptr;
      T.tcol = S.tcol;
      T.tval = S.tval;
      changed = true;
    }
    if (changed)
      PLAN_TRY(cudaMemcpyAsync(p->terms, p->terms_host, sizeof(Term) * nterms, cudaMemcpyHostToDevice, p->stream));
  }
  if (p->fam == FAM_CSR && p->zc && layout == MAGNUS_ROWS_STAGED) {
    bool ok = nterms <= 2;  // two terms at most, each sliced (a pattern or a product term), CSR columns aligned
    for (int k = 0; k < nterms; k++) {
      const Term &T = p->terms_host[k];
      ok &= T.hbase != nullptr && T.nnz > 0 && ((uintptr_t)T.col % 16) == 0;
    }
    if (ok) {
      unsigned long long *cnt = nullptr, mis = 0;
      PLAN_TRY(dalloc(&cnt, 1));
      PLAN_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), p->stream));
      PLAN_TRY(launch_stage_misfits(p->terms, nterms, dim, cnt, p->stream));
      PLAN_TRY(cudaMemcpyAsync(&mis, cnt, sizeof mis, cudaMemcpyDeviceToHost, p->stream));
      PLAN_TRY(cudaStreamSynchronize(p->stream));
      cudaFree(cnt);
      const unsigned long long ntile = (unsigned long long)((dim + 31) / 32);
      if (mis * 64 <= ntile) {
        PLAN_TRY(persistent_max_blocks_per_sm(FAM_CSR, false, 1, &p->max_blocks_stg, true));
        p->staged = p->max_blocks_stg >= 1;
      }
    }
  }
  PLAN_TRY(cudaStreamSynchronize(p->stream));
#undef PLAN_TRY
  *out = p;
  return MAGNUS_OK;
}

magnus_status magnus_plan_destroy(magnus_plan_t plan) {
  if (!plan) return MAGNUS_OK;
  cudaStreamSynchronize(plan->stream);
  free_plan(plan);
  return MAGNUS_OK;
}

magnus_status magnus_propagate(magnus_plan_t p, void *psi, double t0, double h, int64_t nsteps, int32_t variant,
                               magnus_stats *stats) {
  NvtxRange nvtx_range("magnus_propagate");
  if (!p) return set_err(nullptr, MAGNUS_EINVAL, "plan is null");
  p->err.clear();
  if (!psi) return set_err(p, MAGNUS_EINVAL, "psi is null");
  if (((uintptr_t)psi) % 16) return set_err(p, MAGNUS_EINVAL, "psi must be 16-byte aligned");
  if (nsteps < 0) return set_err(p, MAGNUS_EINVAL, "nsteps < 0");
  const int per = exps_per_step(variant);
  if (per == 0) return set_err(p, MAGNUS_EINVAL, "unknown variant %d", variant);
  if (!(h == h) || !(t0 == t0)) return set_err(p, MAGNUS_EINVAL, "t0/h is NaN");
  if (stats) {
    int32_t *log = stats->m_log;
    int64_t cap = stats->m_log_cap;
    memset(stats, 0, sizeof *stats);
    stats->m_log = log;
    stats->m_log_cap = cap;
  }
  if (variant == MAGNUS_M6 && p->fam == FAM_DENSE)
    return set_err(p, MAGNUS_EINVAL, "MAGNUS_M6 takes CSR and matrix-free terms, not dense terms");
  if (nsteps == 0) return MAGNUS_OK;
  const int64_t nexp = nsteps * per;
  magnus_status s = ensure_exp_capacity(p, nexp);
  if (s != MAGNUS_OK) return s;
  if (variant == MAGNUS_M6 && !p->m6) CUDA_TRY(p, dalloc(&p->m6, (size_t)kM6Slots * p->dim * p->opt.nvec));
  CUDA_TRY(p, launch_exp_setup(variant, t0, h, nsteps, p->nterms, p->coeffs, p->term_ab, p->xi, p->opt.m_max,
                               p->opt.rho_max, p->recs, p->dd, nexp, p->stream));
  return run_persistent(p, psi, nexp, stats, variant == MAGNUS_M6, variant == MAGNUS_M4);
}

magnus_status leja_expv(magnus_plan_t p, const double *beta, const void *v, void *out, magnus_stats *stats) {
  NvtxRange nvtx_range("leja_expv");
  if (!p) return set_err(nullptr, MAGNUS_EINVAL, "plan is null");
  p->err.clear();
  if (!beta || !v || !out) return set_err(p, MAGNUS_EINVAL, "null argument");
  if (((uintptr_t)v) % 16 || ((uintptr_t)out) % 16) return set_err(p, MAGNUS_EINVAL, "vectors must be 16-byte aligned");
  for (int k = 0; k < p->nterms; k++)
    if (!(beta[k] == beta[k]) || beta[k] - beta[k] != 0.0) return set_err(p, MAGNUS_EINVAL, "beta[%d] not finite", k);
  if (stats) {
    int32_t *log = stats->m_log;
    int64_t cap = stats->m_log_cap;
    memset(stats, 0, sizeof *stats);
    stats->m_log = log;
    stats->m_log_cap = cap;
  }
  magnus_status s = ensure_exp_capacity(p, 1);
  if (s != MAGNUS_OK) return s;
  if (out != v)
    CUDA_TRY(p, cudaMemcpyAsync(out, v, sizeof(double2) * (size_t)p->dim * p->opt.nvec, cudaMemcpyDeviceToDevice,
                                p->stream));
  CUDA_TRY(p, launch_exp_setup_beta(beta, p->nterms, p->term_ab, p->xi, p->opt.m_max, p->opt.rho_max, p->recs, p->dd,
                                    p->stream));
  return run_persistent(p, out, 1, stats);
}

magnus_status magnus_set_coeff(magnus_plan_t p, int32_t k, const magnus_coeff *c) {
  if (!p) return set_err(nullptr, MAGNUS_EINVAL, "plan is null");
  p->err.clear();
  if (!c || k < 0 || k >= p->nterms) return set_err(p, MAGNUS_EINVAL, "bad term index or null coefficient");
  if (c->nmodes < 0 || c->nmodes > kMaxModes || (c->nmodes > 0 && !c->om))
    return set_err(p, MAGNUS_EINVAL, "nmodes must be 0..%d with om given", kMaxModes);
  Coeff &C = p->coeff_host[k];
  memset(&C, 0, sizeof C);
  C.a0 = c->a0;
  C.nmodes = c->nmodes;
  for (int m = 0; m < C.nmodes; m++) {
    C.ac[m] = c->ac ? c->ac[m] : 0.0;
    C.as[m] = c->as ? c->as[m] : 0.0;
    C.om[m] = c->om[m];
  }
  // stream-ordered: launches issued after this call see the new coefficients (pageable source:
  // the copy is staged before the call returns)
  CUDA_TRY(p, cudaMemcpyAsync(p->coeffs + k, &C, sizeof(Coeff), cudaMemcpyHostToDevice, p->stream));
  return MAGNUS_OK;
}

magnus_status magnus_apply(magnus_plan_t p, const double *beta, const void *x, void *y) {
  NvtxRange nvtx_range("magnus_apply");
  if (!p) return set_err(nullptr, MAGNUS_EINVAL, "plan is null");
  p->err.clear();
  if (!beta || !x || !y) return set_err(p, MAGNUS_EINVAL, "null argument");
  if (x == y) return set_err(p, MAGNUS_EINVAL, "x and y must be distinct buffers");
  if (((uintptr_t)x) % 16 || ((uintptr_t)y) % 16) return set_err(p, MAGNUS_EINVAL, "vectors must be 16-byte aligned");
  for (int k = 0; k < p->nterms; k++)
    if (!(beta[k] == beta[k]) || beta[k] - beta[k] != 0.0) return set_err(p, MAGNUS_EINVAL, "beta[%d] not finite", k);
  CUDA_TRY(p, launch_apply(p->fam, p->terms, p->nterms, beta, p->lbits, p->dlo, p->dhi, (const double2 *)x,
                           (double2 *)y, p->dim, p->opt.nvec, p->zc, p->zmax, p->zhb, p->num_sms, p->stream));
  return MAGNUS_OK;
}

magnus_status magnus_term_interval(magnus_plan_t p, int32_t k, double *a, double *b) {
  if (!p || !a || !b || k < 0 || k >= p->nterms) return set_err(p, MAGNUS_EINVAL, "bad argument");
  *a = p->term_ab_host[2 * k];
  *b = p->term_ab_host[2 * k + 1];
  return MAGNUS_OK;
}

magnus_status magnus_leja_points(magnus_plan_t p, double *xi, int32_t count) {
  if (!p || !xi || count < 1 || count > p->opt.m_max + 1) return set_err(p, MAGNUS_EINVAL, "bad argument");
  CUDA_TRY(p, cudaMemcpyAsync(xi, p->xi, sizeof(double) * count, cudaMemcpyDeviceToHost, p->stream));
  CUDA_TRY(p, cudaStreamSynchronize(p->stream));
  return MAGNUS_OK;
}

magnus_status magnus_divided_differences(magnus_plan_t p, double rho, void *d, int32_t count) {
  if (!p || !d || count < 1 || count > p->opt.m_max + 1 || !(rho >= 0.0))
    return set_err(p, MAGNUS_EINVAL, "bad argument");
  double2 *dev = nullptr;
  CUDA_TRY(p, dalloc(&dev, (size_t)count));
  cudaError_t e = launch_divided_differences(p->xi, count - 1, rho, dev, p->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, dev, sizeof(double2) * count, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  cudaFree(dev);
  if (e != cudaSuccess) return set_err(p, MAGNUS_ECUDA, "divided differences: %s", cudaGetErrorString(e));
  return MAGNUS_OK;
}

magnus_status magnus_adjoint_grad(magnus_plan_t p, const void *psi0, const void *phi, double t0, double h,
                                  int64_t nsteps, int32_t variant, int32_t kd, int32_t ckpt_every, double *F,
                                  double *grad, magnus_stats *stats) {
  NvtxRange nvtx_range("magnus_adjoint_grad");
  if (!p) return set_err(nullptr, MAGNUS_EINVAL, "plan is null");
  p->err.clear();
  if (!psi0 || !phi || !F || !grad) return set_err(p, MAGNUS_EINVAL, "null argument");
  if (((uintptr_t)psi0) % 16 || ((uintptr_t)phi) % 16) return set_err(p, MAGNUS_EINVAL, "vectors must be 16-byte aligned");
  if (variant != MAGNUS_CF4 && variant != MAGNUS_CF4_3 && variant != MAGNUS_M2)
    return set_err(p, MAGNUS_EINVAL, "the adjoint needs a commutator-free variant (CF4, CF4_3 or M2)");
  if (p->opt.nvec != 1) return set_err(p, MAGNUS_EINVAL, "the adjoint takes plans with nvec = 1");
  if (p->fam == FAM_DENSE) return set_err(p, MAGNUS_EINVAL, "the adjoint takes CSR or matrix-free terms");
  if (kd < 0 || kd >= p->nterms) return set_err(p, MAGNUS_EINVAL, "kd out of range");
  if (ckpt_every < 1 || nsteps < 1) return set_err(p, MAGNUS_EINVAL, "need nsteps >= 1 and ckpt_every >= 1");
  if (stats) memset(stats, 0, sizeof *stats);
  const int per = exps_per_step(variant);
  const int64_t D = p->dim, nexp = nsteps * per, seg_exps = (int64_t)ckpt_every * per;
  const int64_t nseg = (nexp + seg_exps - 1) / seg_exps;
  const int m1 = p->opt.m_max + 1;
  magnus_status s = ensure_exp_capacity(p, nexp);
  if (s != MAGNUS_OK) return s;
  // workspace (freed at the end of the call)
  std::vector<void *> tmp;
  auto grab = [&](void **ptr, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
    if (e == cudaSuccess) tmp.push_back(*ptr);
    return e;
  };
  struct Free {
    std::vector<void *> &t;
    ~Free() { for (void *q : t) cudaFree(q); }
  } freer{tmp};
  ExpRec *nrecs = nullptr;
  double2 *ndd = nullptr, *ckpt = nullptr, *seg = nullptr, *lam = nullptr, *aug = nullptr, *G = nullptr, *z = nullptr,
          *a_out = nullptr;
  double *gradd = nullptr, *apart = nullptr;
  Coeff *cdev = nullptr;
  int nm = 0;
  {
    Coeff ch{};
    CUDA_TRY(p, cudaMemcpyAsync(&ch, p->coeffs + kd, sizeof(Coeff), cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    nm = ch.nmodes;
  }
  const int ngrad = 1 + 2 * nm;
  int aug_per_sm = 0;
  CUDA_TRY(p, aug_max_blocks_per_sm(&aug_per_sm));
  const int agrid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)p->num_sms * std::max(1, aug_per_sm), (D + 31) / 32));
  CUDA_TRY(p, grab((void **)&nrecs, sizeof(ExpRec) * nexp));
  CUDA_TRY(p, grab((void **)&ndd, sizeof(double2) * nexp * m1));
  CUDA_TRY(p, grab((void **)&ckpt, sizeof(double2) * nseg * D));
  CUDA_TRY(p, grab((void **)&seg, sizeof(double2) * seg_exps * D));
  CUDA_TRY(p, grab((void **)&lam, sizeof(double2) * D));
  CUDA_TRY(p, grab((void **)&aug, sizeof(double2) * 8 * D));
  CUDA_TRY(p, grab((void **)&a_out, sizeof(double2) * D));
  CUDA_TRY(p, grab((void **)&G, sizeof(double2) * nexp));
  CUDA_TRY(p, grab((void **)&z, sizeof(double2)));
  CUDA_TRY(p, grab((void **)&gradd, sizeof(double) * ngrad));
  CUDA_TRY(p, grab((void **)&apart, sizeof(double) * 12 * agrid));  // two slots x agrid x (2 sums, 4 maxima)
  longlong2 *zaug = nullptr;  // fixed-point copies of the augmented vectors (substep input, ping-pong)
  if (p->zc) CUDA_TRY(p, grab((void **)&zaug, sizeof(longlong2) * 6 * D));
  cdev = p->coeffs + kd;

  int grid, gv;
  choose_grid(p, &grid, &gv, false, p->zc != nullptr ? 1 : 0);  // linear generators: the fixed-point kernel
  if ((int64_t)8 * grid > p->partials_cap) {
    if (p->partials) cudaFree(p->partials);
    p->partials = nullptr;
    p->partials_cap = 0;
    CUDA_TRY(p, dalloc(&p->partials, (size_t)8 * grid));
    p->partials_cap = (int64_t)8 * grid;
  }
  cudaStream_t st = p->stream;
  CUDA_TRY(p, launch_exp_setup(variant, t0, h, nsteps, p->nterms, p->coeffs, p->term_ab, p->xi, p->opt.m_max,
                               p->opt.rho_max, p->recs, p->dd, nexp, st));
  CUDA_TRY(p, launch_negate_records(p->recs, p->dd, nrecs, ndd, nexp, p->opt.m_max, st));
  CUDA_TRY(p, cudaMemsetAsync(p->bar, 0, sizeof(GridBar), st));
  CUDA_TRY(p, cudaMemsetAsync(p->counters, 0, sizeof(Counters), st));
  PersistArgs a{};
  a.dim = D;
  a.nvec = 1;
  a.nterms = p->nterms;
  a.gv = gv;
  a.m_max = p->opt.m_max;
  a.tol_rel = p->opt.tol_rel;
  a.tol_abs = p->opt.tol_abs;
  a.terms = p->terms;
  a.xi = p->xi;
  a.alt = p->alt;
  a.w0 = p->w0;
  a.w1 = p->w1;
  a.u = p->u;
  a.partials = p->partials;
  a.bar = p->bar;
  a.counters = p->counters;
  a.spin_limit_ns = spin_limit(p);
  a.fam = p->fam;
  a.lbits = p->lbits;
  a.dlo = p->dlo;
  a.dhi = p->dhi;
  a.zfix = p->zc != nullptr ? 1 : 0;
  a.zc = p->zc;
  a.zw0 = p->zw0;
  a.zw1 = p->zw1;
  a.zhb = p->zhb;
  a.zreal = p->zreal;
  auto persist = [&](double2 *x, const ExpRec *R, const double2 *DD, int64_t cnt) -> cudaError_t {
    PersistArgs q = a;
    q.recs = R;
    q.dd = DD;
    q.nexp = cnt;
    q.psi = x;
    return launch_persistent(q, grid, persistent_block_size(), false, st);
  };
  AugArgs g{};
  g.dim = D;
  g.nterms = p->nterms;
  g.kd = kd;
  g.m_max = p->opt.m_max;
  g.fam = p->fam;
  g.lbits = p->lbits;
  g.tol_rel = p->opt.tol_rel;
  g.tol_abs = p->opt.tol_abs;
  g.terms = p->terms;
  g.xi = p->xi;
  g.out_a = a_out;
  g.acur = aug; g.bcur = aug + D; g.anxt = aug + 2 * D; g.bnxt = aug + 3 * D;
  g.wa0 = aug + 4 * D; g.wb0 = aug + 5 * D; g.wa1 = aug + 6 * D; g.wb1 = aug + 7 * D;
  g.partials = apart;
  g.bar = p->bar;
  g.counters = p->counters;
  g.spin_limit_ns = spin_limit(p);
  g.dlo = p->dlo;
  g.dhi = p->dhi;
  g.zfix = zaug != nullptr;
  g.zhb = p->zhb;
  g.zreal = p->zreal;
  if (zaug) {
    g.zca = zaug; g.zcb = zaug + D; g.zwa0 = zaug + 2 * D; g.zwb0 = zaug + 3 * D; g.zwa1 = zaug + 4 * D;
    g.zwb1 = zaug + 5 * D;
  }

  // forward with a checkpoint at the start of every segment; the final state ends in p->alt's partner
  double2 *psiw = lam;  // lam doubles as the forward work vector until the backward pass starts
  CUDA_TRY(p, cudaMemcpyAsync(psiw, psi0, sizeof(double2) * D, cudaMemcpyDeviceToDevice, st));
  for (int64_t sgi = 0; sgi < nseg; sgi++) {
    const int64_t e0 = sgi * seg_exps, cnt = std::min(seg_exps, nexp - e0);
    CUDA_TRY(p, cudaMemcpyAsync(ckpt + sgi * D, psiw, sizeof(double2) * D, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(p, persist(psiw, p->recs + e0, p->dd + e0 * m1, cnt));
  }
  CUDA_TRY(p, launch_dot((const double2 *)phi, psiw, D, z, st));
  CUDA_TRY(p, cudaMemcpyAsync(lam, phi, sizeof(double2) * D, cudaMemcpyDeviceToDevice, st));
  // backward, segment by segment
  for (int64_t sgi = nseg - 1; sgi >= 0; sgi--) {
    const int64_t e0 = sgi * seg_exps, cnt = std::min(seg_exps, nexp - e0);
    CUDA_TRY(p, cudaMemcpyAsync(seg, ckpt + sgi * D, sizeof(double2) * D, cudaMemcpyDeviceToDevice, st));
    for (int64_t i = 1; i < cnt; i++) {
      CUDA_TRY(p, cudaMemcpyAsync(seg + i * D, seg + (i - 1) * D, sizeof(double2) * D, cudaMemcpyDeviceToDevice, st));
      CUDA_TRY(p, persist(seg + i * D, p->recs + e0 + i - 1, p->dd + (e0 + i - 1) * m1, 1));
    }
    for (int64_t i = cnt - 1; i >= 0; i--) {
      const int64_t e = e0 + i;
      g.rec = p->recs + e;
      g.dd = p->dd + e * m1;
      g.v = seg + i * D;
      CUDA_TRY(p, launch_aug_persistent(g, agrid, st));
      CUDA_TRY(p, launch_dot(lam, a_out, D, G + e, st));
      CUDA_TRY(p, persist(lam, nrecs + e, ndd + e * m1, 1));
    }
  }
  CUDA_TRY(p, launch_adjoint_contract(G, z, cdev, variant, t0, h, nsteps, gradd, ngrad, st));
  double2 zh{};
  Counters c{};
  CUDA_TRY(p, cudaMemcpyAsync(&zh, z, sizeof zh, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(p, cudaMemcpyAsync(grad, gradd, sizeof(double) * ngrad, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(p, cudaMemcpyAsync(&c, p->counters, sizeof c, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(p, cudaStreamSynchronize(st));
  *F = zh.x * zh.x + zh.y * zh.y;
  if (stats) {
    stats->n_matvec = c.n_matvec;
    stats->max_m = c.max_m;
    stats->status = c.status;
    stats->n_exp = nexp;
  }
  if (c.status != MAGNUS_OK) return set_err(p, (magnus_status)c.status, "adjoint: device status %d", c.status);
  return MAGNUS_OK;
}

int64_t magnus_xxz_nnz(int32_t nspins) {
  if (nspins < 2 || nspins > kMaxSpins) return -1;
  const int64_t D = (int64_t)1 << nspins;
  return D + (int64_t)(nspins - 1) * (D / 2);
}

magnus_status magnus_build_xxz_csr(int32_t nspins, const double *J, const double *hz, double delta, int64_t *rowptr,
                                   int32_t *col, void *val, void *stream) {
  if (nspins < 2 || nspins > kMaxSpins || !J || !hz || !rowptr || !col || !val)
    return set_err(nullptr, MAGNUS_EINVAL, "build_xxz_csr: bad argument");
  CUDA_TRY(nullptr, launch_build_xxz_csr(nspins, J, hz, delta, rowptr, col, (double2 *)val, (cudaStream_t)stream));
  return MAGNUS_OK;
}

magnus_status magnus_build_field_x_csr(int32_t nspins, int64_t *rowptr, int32_t *col, void *val, void *stream) {
  if (nspins < 1 || nspins > kMaxSpins || !rowptr || !col || !val)
    return set_err(nullptr, MAGNUS_EINVAL, "build_field_x_csr: bad argument");
  CUDA_TRY(nullptr, launch_build_field_x_csr(nspins, rowptr, col, (double2 *)val, (cudaStream_t)stream));
  return MAGNUS_OK;
}

magnus_status magnus_build_longrange_dense(int32_t nspins, double alpha, const double *hz, double delta, void *H,
                                           void *stream) {
  if (nspins < 2 || nspins > 15 || !hz || !H) return set_err(nullptr, MAGNUS_EINVAL, "build_longrange_dense: bad argument");
  CUDA_TRY(nullptr, launch_build_longrange_dense(nspins, alpha, hz, delta, (double2 *)H, (cudaStream_t)stream));
  return MAGNUS_OK;
}

magnus_status magnus_build_field_x_dense(int32_t nspins, void *H, void *stream) {
  if (nspins < 1 || nspins > 15 || !H) return set_err(nullptr, MAGNUS_EINVAL, "build_field_x_dense: bad argument");
  CUDA_TRY(nullptr, launch_build_field_x_dense(nspins, (double2 *)H, (cudaStream_t)stream));
  return MAGNUS_OK;
}

}  // extern "C"
