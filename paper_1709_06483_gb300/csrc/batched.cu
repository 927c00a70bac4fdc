// Many independent problems in one persistent launch: each CTA takes whole problems from a work
// queue (largest first) and runs their complete Magnus propagation (arXiv:1709.06483, Sec. 2) with
// the Leja recurrence of Sec. 3, synchronising only within the CTA -- a problem of up to 2^14 rows
// is about one SM's share of the whole batch, so no grid barrier is needed.  The per-problem setup
// launches and the persistent kernel are captured once into a CUDA graph and replayed; the CTA
// size is chosen by timing the candidates on the first call (the batch's own autotuner).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "magnus_internal.cuh"
#include "persist_common.cuh"
#include "rows.cuh"

namespace cg = cooperative_groups;

namespace mg {

struct BatchItem {
  int64_t dim;
  int nterms;
  int lbits;
  const Term *terms;      // device [nterms]
  const double *dlo, *dhi;
  const ExpRec *recs;     // device [nexp]
  const double2 *dd;      // device [nexp][m_max+1]
  double2 *psi;           // the caller's state
  double2 *alt, *w0, *w1, *u;
  int *mlog;              // degrees of the substeps, [mlog_cap]
  int mlog_cap;
  int zhb;                // fixed-point pattern sums: headroom bits of the row sums
  longlong2 *zc, *zw0, *zw1;  // their copies of the substep input and the Leja vectors (null: FP64 sums)
  int zreal;              // every term real-valued
  int _pad;
};

struct BatchArgs {
  int count;
  int m_max;
  int64_t nexp;
  double tol_rel, tol_abs;
  const double *xi;
  const BatchItem *items;
  const int *order;       // processing order (largest first)
  unsigned *next;         // queue heads, zero before the launch: [0] items shared by a cluster, [1] the rest
  int nbig;               // the first nbig items (in processing order) are shared by the CTAs of a cluster
  Counters *counters;
};

namespace {

using namespace rows;

// One problem per thread-block cluster: the cluster's CTAs split the problem's rows, exchange their
// partial norms through distributed shared memory and synchronise with the hardware cluster
// barrier (release/acquire at cluster scope), so a large chain runs on several SMs at once.  Only
// the problems larger than one CTA's fair share of all rows are shared so (the first A.nbig in
// the largest-first order); after them every CTA takes the remaining problems alone from a second
// queue.  Cluster size 1 is the plain CTA-per-problem case.  ZF: the instantiation for linear generators
// whose pattern terms are summed in fixed point (as in the single-problem kernel); it also
// tracks the largest component of every vector, from which the fixed-point scales follow.
template <int FAM, int BS, bool ZF>
__global__ void __launch_bounds__(BS) k_batched(BatchArgs A) {
  __shared__ int s_next;            // rank 0: the problem index taken from the queue
  __shared__ int s_item;            // every CTA: its copy of that index
  __shared__ BatchItem sI;
  __shared__ Term sT[kMaxTerms];
  __shared__ ExpRec sR;
  __shared__ double s_jb[kMaxSpins], s_j2[kMaxSpins];
  __shared__ double s_red[2][BS / 32];
  __shared__ unsigned s_rmx[2][BS / 32];
  __shared__ double s_part[2][4];   // this CTA's partial sums and maxima, two slots (alternating reductions)
  __shared__ double s_tot[4];       // cluster totals: two sums, then bounds of the two maxima
  __shared__ double s_wz[kMaxTerms];
  __shared__ long long s_cb[kMaxSpins];  // ZF, FAM_MF: bond weights as 62-bit mantissas
  __shared__ int s_cbe;

  cg::cluster_group cl = cg::this_cluster();
  const unsigned crank = cl.block_rank(), csize = cl.num_blocks();
  // solo: after the shared items, every CTA takes the remaining (small) items alone, from a queue
  // of their own, with CTA-local synchronisation only
  bool solo = false;
  auto csync = [&]() {
    if (solo) __syncthreads(); else cl.sync();
  };
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned slot = 0;
  // sums of two values over all threads of the cluster, identical in every thread afterwards
  // (fixed order: warps, then CTAs by rank), and (ZF) bounds of two maxima given as abshi high
  // words; the cluster barrier also publishes this CTA's vector writes to the other CTAs of the
  // cluster
  auto cluster_sums = [&](double x0, double x1, unsigned m0 = 0u, unsigned m1 = 0u) {
    x0 = warp_sum(x0);
    x1 = warp_sum(x1);
    if (ZF) {
      m0 = __reduce_max_sync(kFull, m0);
      m1 = __reduce_max_sync(kFull, m1);
    }
    if (lane == 0) {
      s_red[0][warp] = x0;
      s_red[1][warp] = x1;
      if (ZF) { s_rmx[0][warp] = m0; s_rmx[1][warp] = m1; }
    }
    __syncthreads();
    if (tid == 0) {
      double y0 = 0.0, y1 = 0.0;
      unsigned n0 = 0, n1 = 0;
      for (int w = 0; w < BS / 32; w++) {
        y0 += s_red[0][w];
        y1 += s_red[1][w];
        if (ZF) { n0 = max(n0, s_rmx[0][w]); n1 = max(n1, s_rmx[1][w]); }
      }
      s_part[slot][0] = y0;
      s_part[slot][1] = y1;
      s_part[slot][2] = __hiloint2double((int)n0, 0);
      s_part[slot][3] = __hiloint2double((int)n1, 0);
    }
    csync();
    if (tid == 0) {
      double y0 = 0.0, y1 = 0.0;
      unsigned n0 = 0, n1 = 0;
      for (unsigned q = 0; q < (solo ? 1u : csize); q++) {
        const double *rp = solo ? &s_part[slot][0] : cl.map_shared_rank(&s_part[slot][0], q);
        y0 += rp[0];
        y1 += rp[1];
        if (ZF) { n0 = max(n0, (unsigned)__double2hiint(rp[2])); n1 = max(n1, (unsigned)__double2hiint(rp[3])); }
      }
      s_tot[0] = y0;
      s_tot[1] = y1;
      s_tot[2] = abshi_bound(n0);
      s_tot[3] = abshi_bound(n1);
    }
    __syncthreads();
    slot ^= 1u;
  };

  for (;;) {
    int q = A.count;
    if (!solo) {
      cl.sync();
      if (crank == 0 && tid == 0) s_next = (int)atomicAdd(A.next, 1u);
      cl.sync();
      if (tid == 0) s_item = *cl.map_shared_rank(&s_next, 0);
      cl.sync();  // every CTA has read rank 0's index before any CTA may leave or go solo
      q = s_item;
      if (q >= A.nbig) solo = true;  // the same decision in every CTA of the cluster
    }
    if (solo) {
      __syncthreads();
      if (tid == 0) s_item = A.nbig + (int)atomicAdd(A.next + 1, 1u);
      __syncthreads();
      q = s_item;
    }
    if (q >= A.count) break;
    const unsigned cr = solo ? 0u : crank, cn = solo ? 1u : csize;  // this CTA's share of the item
    if (tid == 0) sI = A.items[A.order[q]];
    __syncthreads();
    const int64_t D = sI.dim;
    const int nt = sI.nterms;
    // this CTA's rows: whole warps of consecutive rows
    const int64_t rows_per = (((D + cn - 1) / cn) + 31) & ~(int64_t)31;
    const int64_t lo = min(D, (int64_t)cr * rows_per), hi = min(D, lo + rows_per);
    for (int i = tid; i < nt * (int)sizeof(Term) / 4; i += BS)
      reinterpret_cast<int *>(sT)[i] = reinterpret_cast<const int *>(sI.terms)[i];
    __syncthreads();
    Ctx cx{};
    cx.T = sT;
    cx.nt = nt;
    cx.n = sT[0].nspins;
    cx.lbits = sI.lbits;
    cx.lomask = ((int64_t)1 << (sI.lbits + 1)) - 1;
    cx.dlo = sI.dlo;
    cx.dhi = sI.dhi;
    cx.jb = s_jb;
    cx.j2 = s_j2;
    cx.cb = (ZF && FAM == FAM_MF) ? s_cb : nullptr;
    if (FAM == FAM_MF)
      for (int p = 1 + tid; p < cx.n; p += BS) s_j2[p - 1] = 2.0 * sT[0].J[cx.n - p - 1];

    double s0 = 0.0;
    unsigned m0 = 0;
    for (int64_t r = lo + tid; r < hi; r += BS) {
      const double2 v = sI.psi[r];
      s0 += cabs2(v);
      if (ZF) m0 = max(m0, abshi(v));
    }
    cluster_sums(s0, 0.0, m0, 0u);
    double vn = sqrt(s_tot[0]);
    double vm = s_tot[2];  // ZF: bound of the largest component of the substep input

    double2 *cur = sI.psi, *nxt = sI.alt;
    int sub_counter = 0;
    int status = MAGNUS_OK;
    for (int64_t e = 0; e < A.nexp && status == MAGNUS_OK; e++) {
      __syncthreads();
      if (tid == 0) sR = sI.recs[e];
      __syncthreads();
      const ExpRec &R = sR;
      if (ZF && R.mode != MODE_LINEAR) { status = MAGNUS_EINVAL; break; }  // ZF runs linear generators only
      if (FAM == FAM_MF) {
        for (int p = 1 + tid; p < cx.n; p += BS) s_jb[p - 1] = s_j2[p - 1] * R.bg[0];
        __syncthreads();
      }
      double opnorm = 0.0;  // ZF: sum_k |bg_k| ||H_k||_inf
      if (ZF) {
        if (tid < nt) s_wz[tid] = R.bg[tid] * sT[tid].pval;
        for (int k = 0; k < nt; k++) opnorm = fma(fabs(R.bg[k]), sT[k].gnorm, opnorm);
        if (FAM == FAM_MF && tid == 0) {  // bond weights 2 J bg_0 as mantissas: max |w| < 2^s_cbe
          double wmax = 0.0;
          for (int p = 0; p < cx.n - 1; p++) wmax = fmax(wmax, fabs(s_jb[p]));
          int E = 0;
          if (wmax > 0.0) frexp(wmax, &E);
          E = max(-400, min(400, E));
          for (int p = 0; p < cx.n - 1; p++) s_cb[p] = llrint(ldexp(s_jb[p], 62 - E));
          s_cbe = E;
        }
        __syncthreads();
        cx.cbe = s_cbe;
      }
      const double2 *d = sI.dd + e * (int64_t)(A.m_max + 1);
      if (!(R.gamma > 0.0)) {
        const double2 ph = d[0];
        for (int64_t r = lo + tid; r < hi; r += BS) nxt[r] = cmul(ph, cur[r]);
        csync();
        vm *= sqrt(cabs2(ph)) * (1.0 + 0x1p-40);
        double2 *tmp = cur; cur = nxt; nxt = tmp;
        continue;
      }
      const double2 d0 = d[0];
      for (int sub = 0; sub < R.s && status == MAGNUS_OK; sub++) {
        double ep = sqrt(cabs2(d0)) * vn, pn = vn, pm = vm, wm = vm;
        int m = 0;
        int zs_src = 0;
        if (ZF) {  // fixed-point copy of the substep input
          zs_src = fix_scale(vm, sI.zhb);
          for (int64_t r = lo + tid; r < hi; r += BS) sI.zc[r] = fix2(cur[r], zs_src);
          csync();
        }
        for (int j = 1; j <= A.m_max; j++) {
          const double2 *src = (j == 1) ? cur : (((j - 2) & 1) ? sI.w1 : sI.w0);
          double2 *dst = ((j - 1) & 1) ? sI.w1 : sI.w0;
          const double shift = R.cg + A.xi[j - 1];
          const double2 dj = d[j];
          if constexpr (ZF) {
            // |Re w_j|, |Im w_j| <= ||X - shift||_inf max(|Re w_{j-1}|, |Im w_{j-1}|) (x2 for complex terms)
            const int zs_dst = fix_scale((opnorm + fabs(shift)) * (sI.zreal ? 1.0 : 2.0) * wm * (1.0 + 0x1p-20), sI.zhb);
            const longlong2 *zsrc = (j == 1) ? sI.zc : (((j - 2) & 1) ? sI.zw1 : sI.zw0);
            longlong2 *zdst = ((j - 1) & 1) ? sI.zw1 : sI.zw0;
            double sw = 0.0, sp = 0.0;
            unsigned mw = 0, mp = 0;
            for (int64_t r = lo + tid; r < hi; r += BS) {
              double2 wr;
              const double2 y = Op<FAM>::combo_z(cx, R, s_wz, shift, src, zsrc, zs_src, r, wr);
              dst[r] = y;
              zdst[r] = fix2(y, zs_dst);
              double2 pr = (j == 1) ? cmul(d0, wr) : nxt[r];
              pr = cfma(dj, y, pr);
              nxt[r] = pr;
              sw = fma(y.x, y.x, fma(y.y, y.y, sw));
              sp = fma(pr.x, pr.x, fma(pr.y, pr.y, sp));
              mw = max(mw, abshi(y));
              mp = max(mp, abshi(pr));
            }
            cluster_sums(sw, sp, mw, mp);
            zs_src = zs_dst;
            wm = s_tot[2];
            pm = s_tot[3];
            const double ej = sqrt(cabs2(dj)) * sqrt(s_tot[0]);
            pn = sqrt(s_tot[1]);
            if (!isfinite(ej) || !isfinite(pn)) { status = MAGNUS_ENONFINITE; m = j; break; }
            if (ej + ep <= A.tol_abs + A.tol_rel * pn) { m = j; break; }
            ep = ej;
            continue;
          }
          if (R.mode == MODE_M4) {
            for (int64_t r = lo + tid; r < hi; r += BS)
              for (int k = 0; k < nt; k++) sI.u[(size_t)k * D + r] = Op<FAM>::term(cx, k, src, r);
            csync();
          }
          double sw = 0.0, sp = 0.0;
          for (int64_t r = lo + tid; r < hi; r += BS) {
            double2 y, wr;
            if (R.mode == MODE_M4) {
              y = make_double2(0.0, 0.0);
              double2 z = make_double2(0.0, 0.0);
              int pi = 0;
              for (int k = 0; k < nt; k++) {
                y = rfma(R.bg[k], sI.u[(size_t)k * D + r], y);
                for (int l = k + 1; l < nt; l++, pi++) {
                  const double2 hkul = Op<FAM>::term(cx, k, sI.u + (size_t)l * D, r);
                  const double2 hluk = Op<FAM>::term(cx, l, sI.u + (size_t)k * D, r);
                  z = rfma(R.kg[pi], make_double2(hkul.x - hluk.x, hkul.y - hluk.y), z);
                }
              }
              y.x += z.y;
              y.y -= z.x;
              wr = ldv(src + r);
              y = rfma(-shift, wr, y);
            } else {
              y = Op<FAM>::combo(cx, R, shift, src, r, wr);
            }
            dst[r] = y;
            double2 pr = (j == 1) ? cmul(d0, wr) : nxt[r];
            pr = cfma(dj, y, pr);
            nxt[r] = pr;
            sw = fma(y.x, y.x, fma(y.y, y.y, sw));
            sp = fma(pr.x, pr.x, fma(pr.y, pr.y, sp));
          }
          cluster_sums(sw, sp);
          const double ej = sqrt(cabs2(dj)) * sqrt(s_tot[0]);
          pn = sqrt(s_tot[1]);
          if (!isfinite(ej) || !isfinite(pn)) { status = MAGNUS_ENONFINITE; m = j; break; }
          if (ej + ep <= A.tol_abs + A.tol_rel * pn) { m = j; break; }
          ep = ej;
        }
        if (status == MAGNUS_OK && m == 0) { status = MAGNUS_ENOCONV; m = A.m_max; }
        if (cr == 0 && tid == 0) {
          atomicAdd((unsigned long long *)&A.counters->n_matvec, (unsigned long long)m);
          atomicAdd((unsigned long long *)&A.counters->n_termapply,
                    (unsigned long long)m * nt * (R.mode == MODE_M4 ? 2 : 1));
          atomicAdd((unsigned long long *)&A.counters->n_substeps, 1ULL);
          atomicMax(&A.counters->max_m, m);
          if (sI.mlog && sub_counter < sI.mlog_cap) sI.mlog[sub_counter] = m;
        }
        sub_counter++;
        vn = pn;
        vm = pm;
        double2 *tmp = cur; cur = nxt; nxt = tmp;
      }
      if (cr == 0 && tid == 0) atomicAdd((unsigned long long *)&A.counters->n_exp, 1ULL);
    }
    if (status != MAGNUS_OK) {
      if (cr == 0 && tid == 0) atomicCAS(&A.counters->status, 0, status);
    } else if (cur != sI.psi) {
      for (int64_t r = lo + tid; r < hi; r += BS) sI.psi[r] = cur[r];
    }
  }
}

template <int BS>
const void *batched_kernel(int fam, bool zf) {
  if (zf && fam == FAM_CSR) return (const void *)k_batched<FAM_CSR, BS, true>;
  if (zf && fam == FAM_MF) return (const void *)k_batched<FAM_MF, BS, true>;
  switch (fam) {
    case FAM_CSR: return (const void *)k_batched<FAM_CSR, BS, false>;
    case FAM_MF: return (const void *)k_batched<FAM_MF, BS, false>;
    default: return (const void *)k_batched<FAM_GENERIC, BS, false>;
  }
}

const void *batched_kernel_for(int fam, int bs, bool zf) {
  switch (bs) {
    case 128: return batched_kernel<128>(fam, zf);
    case 512: return batched_kernel<512>(fam, zf);
    case 1024: return batched_kernel<1024>(fam, zf);
    default: return batched_kernel<256>(fam, zf);
  }
}

}  // namespace
}  // namespace mg

// ============================================================================ host side
using namespace mg;

struct magnus_batch_s {
  cudaStream_t stream = nullptr;  // the batch's own stream (graphs are captured on it)
  int count = 0;
  int fam = FAM_GENERIC;
  int num_sms = 0;
  magnus_options opt{};
  std::vector<int64_t> dims;
  std::vector<int> nterms;
  int *nterms_dev = nullptr;      // [count]
  std::vector<std::vector<Term>> terms_host;
  std::vector<std::vector<Coeff>> coeffs_host;
  std::vector<int> lbits;
  std::vector<void *> allocs;     // every device allocation, freed at destroy
  Term *terms = nullptr;          // [count][kMaxTerms]
  Coeff *coeffs = nullptr;        // [count][kMaxTerms]
  double *term_ab = nullptr;      // [count][2 kMaxTerms]
  std::vector<const double *> dlo, dhi;
  double *xi = nullptr, *cand = nullptr;
  unsigned *counter = nullptr, *next = nullptr;
  Counters *counters = nullptr;
  double2 *scratch = nullptr;     // alt, w0, w1, u per item
  std::vector<size_t> scratch_off;
  bool zf = false;                // linear generators sum pattern terms in fixed point
  longlong2 *zscratch = nullptr;  // their copies: substep input, w0, w1 per item (at 3 scratch_z_off[i])
  std::vector<size_t> zoff;
  std::vector<int> zhb, zreal;
  int *order = nullptr;
  std::vector<int> order_host;    // the processing order (largest first)
  BatchItem *items_dev = nullptr;
  std::vector<BatchItem> items_host;
  ExpRec *recs = nullptr;
  double2 *dd = nullptr;
  int64_t recs_cap = 0;           // per item
  int *mlog = nullptr;
  int64_t mlog_cap = 0;           // per item
  // graph cache
  cudaGraphExec_t graph = nullptr;
  double g_t0 = 0, g_h = 0;
  int64_t g_nsteps = -1;
  int g_variant = 0, g_bs = 0, g_mlog = 0;
  int tuned_bs = 0;
  int tuned_cs = 1;
  std::vector<double> tune_ms;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;
};

namespace {

std::string g_batch_err;

magnus_status berr(magnus_batch_t b, magnus_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) b->err = buf; else g_batch_err = buf;
  return s;
}

#define BTRY(b, expr)                                                                                   \
  do {                                                                                                  \
    cudaError_t e_ = (expr);                                                                            \
    if (e_ != cudaSuccess)                                                                              \
      return berr(b, e_ == cudaErrorMemoryAllocation ? MAGNUS_ENOMEM : MAGNUS_ECUDA, "%s: %s", #expr,     \
                  cudaGetErrorString(e_));                                                              \
  } while (0)

template <class T>
cudaError_t balloc(magnus_batch_t b, T **p, size_t count) {
  cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
  if (e == cudaSuccess) b->allocs.push_back((void *)*p);
  return e;
}

void batch_free(magnus_batch_t b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void *p : b->allocs) cudaFree(p);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

magnus_status enqueue_run(magnus_batch_t b, int variant, double t0, double h, int64_t nsteps, int bs, int cs,
                          const BatchItem *items_dev) {
  const int64_t nexp = nsteps * exps_per_step(variant);
  const bool zf = b->zf && variant != MAGNUS_M4;
  BTRY(b, launch_exp_setup_batch(variant, t0, h, nsteps, b->count, b->nterms_dev, b->coeffs, b->term_ab, b->xi,
                                 b->opt.m_max, b->opt.rho_max, b->recs, b->dd, b->recs_cap, b->stream));
  BTRY(b, cudaMemsetAsync(b->next, 0, 2 * sizeof(unsigned), b->stream));
  BTRY(b, cudaMemsetAsync(b->counters, 0, sizeof(Counters), b->stream));
  BatchArgs A{};
  A.count = b->count;
  A.m_max = b->opt.m_max;
  A.nexp = nexp;
  A.tol_rel = b->opt.tol_rel;
  A.tol_abs = b->opt.tol_abs;
  A.xi = b->xi;
  A.items = items_dev;
  A.order = b->order;
  A.next = b->next;
  A.counters = b->counters;
  A.nbig = b->count;
  int per_sm = 0;
  BTRY(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel_for(b->fam, bs, zf), bs, 0));
  int grid = b->num_sms * std::max(1, per_sm);
  if (b->opt.ctas > 0) grid = std::min(grid, b->opt.ctas);
  grid = std::min(grid, b->count * cs);
  grid = std::max(cs, grid - grid % cs);
  if (cs > 1) {
    // a cluster shares only the items larger than one CTA's fair share of all rows; after them its
    // CTAs take the rest alone (splitting small items only adds cluster barriers)
    int64_t total = 0;
    for (int i = 0; i < b->count; i++) total += b->dims[i];
    const int64_t fair = total / grid;
    int nbig = 0;
    while (nbig < b->count && b->dims[b->order_host[nbig]] > fair) nbig++;
    A.nbig = nbig;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(bs);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void *args[] = {&A};
  BTRY(b, cudaLaunchKernelExC(&cfg, batched_kernel_for(b->fam, bs, zf), args));
  return MAGNUS_OK;
}

}  // namespace

extern "C" {

MAGNUS_API const char *magnus_batch_last_error(magnus_batch_t b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

MAGNUS_API magnus_status magnus_batch_create(magnus_batch_t *out, int32_t count, const magnus_batch_item *items,
                                             const magnus_options *opt, void *stream) {
  (void)stream;
  if (!out) return berr(nullptr, MAGNUS_EINVAL, "batch pointer is null");
  *out = nullptr;
  if (count < 1 || !items) return berr(nullptr, MAGNUS_EINVAL, "count must be >= 1 with items given");
  magnus_options o{1e-10, 1e-10, 4.0, 100, 1, 0, MAGNUS_FP64};
  o.fixed_sums = 1;
  if (opt) o = *opt;
  if (o.nvec != 1) return berr(nullptr, MAGNUS_EINVAL, "batch items carry one state each (nvec = 1)");
  if (o.fixed_sums != 0 && o.fixed_sums != 1) return berr(nullptr, MAGNUS_EINVAL, "fixed_sums must be 0 or 1");
  if (o.precision != MAGNUS_FP64) return berr(nullptr, MAGNUS_EINVAL, "batches use MAGNUS_FP64");
  if (o.interval != MAGNUS_INTERVAL_GERSHGORIN)
    return berr(nullptr, MAGNUS_EINVAL, "batches use MAGNUS_INTERVAL_GERSHGORIN");
  if (o.m_max < 2 || o.m_max > kMmaxLimit || !(o.rho_max > 0.0) || !(o.tol_rel + o.tol_abs > 0.0))
    return berr(nullptr, MAGNUS_EINVAL, "bad options");
  magnus_batch_t b = new magnus_batch_s();
  b->count = count;
  b->opt = o;
  auto fail = [&](magnus_status s) {
    g_batch_err = b->err;
    batch_free(b);
    return s;
  };
#define BCREATE(expr)                                             \
  do {                                                            \
    magnus_status s_ = (magnus_status)0;                          \
    cudaError_t e_ = (expr);                                      \
    if (e_ != cudaSuccess) {                                      \
      s_ = berr(b, e_ == cudaErrorMemoryAllocation ? MAGNUS_ENOMEM : MAGNUS_ECUDA, "%s: %s", #expr, \
                cudaGetErrorString(e_));                          \
      return fail(s_);                                            \
    }                                                             \
  } while (0)
  int dev = 0;
  BCREATE(cudaGetDevice(&dev));
  BCREATE(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev));
  BCREATE(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
  BCREATE(cudaEventCreate(&b->ev0));
  BCREATE(cudaEventCreate(&b->ev1));
  b->dims.resize(count);
  b->nterms.resize(count);
  b->terms_host.resize(count);
  b->coeffs_host.resize(count);
  b->lbits.assign(count, 1);
  int fam_all = -1;
  for (int i = 0; i < count; i++) {
    const magnus_batch_item &it = items[i];
    if (it.dim < 2 || it.dim > ((int64_t)1 << 24) || it.nterms < 1 || it.nterms > kMaxTerms || !it.terms || !it.coeffs) {
      berr(b, MAGNUS_EINVAL, "item %d: bad dim/nterms", i);
      return fail(MAGNUS_EINVAL);
    }
    b->dims[i] = it.dim;
    b->nterms[i] = it.nterms;
    b->terms_host[i].assign(kMaxTerms, Term{});
    b->coeffs_host[i].assign(kMaxTerms, Coeff{});
    bool all_csr = true;
    for (int k = 0; k < it.nterms; k++) {
      const magnus_term &t = it.terms[k];
      Term &T = b->terms_host[i][k];
      memset(&T, 0, sizeof T);
      set_term_storage(T, t);
      T.nspins = t.nspins;
      T.nnz = t.nnz;
      T.rowptr = t.rowptr;
      T.col = t.col;
      T.delta = t.delta;
      const bool pow2 = t.nspins >= 1 && t.nspins <= kMaxSpins && it.dim == ((int64_t)1 << t.nspins);
      if (t.kind == MAGNUS_TERM_CSR || t.kind == MAGNUS_TERM_CSR_REAL) {
        if (!t.rowptr || !t.col || !t.val) { berr(b, MAGNUS_EINVAL, "item %d term %d: CSR arrays missing", i, k); return fail(MAGNUS_EINVAL); }
      } else if (t.kind == MAGNUS_TERM_XXZ) {
        if (!pow2 || t.nspins < 2 || !t.J || !t.hz) { berr(b, MAGNUS_EINVAL, "item %d term %d: bad XXZ term", i, k); return fail(MAGNUS_EINVAL); }
        for (int s = 0; s < t.nspins - 1; s++) T.J[s] = t.J[s];
        for (int s = 0; s < t.nspins; s++) T.hz[s] = t.hz[s];
      } else if (t.kind == MAGNUS_TERM_FIELD_X) {
        if (!pow2) { berr(b, MAGNUS_EINVAL, "item %d term %d: FIELD_X needs dim = 2^nspins", i, k); return fail(MAGNUS_EINVAL); }
      } else {
        berr(b, MAGNUS_EINVAL, "item %d term %d: batches take CSR, XXZ and FIELD_X terms", i, k);
        return fail(MAGNUS_EINVAL);
      }
      all_csr &= T.kind == MAGNUS_TERM_CSR;
      const magnus_coeff &c = it.coeffs[k];
      if (c.nmodes < 0 || c.nmodes > kMaxModes || (c.nmodes > 0 && !c.om)) {
        berr(b, MAGNUS_EINVAL, "item %d coefficient %d: bad modes", i, k);
        return fail(MAGNUS_EINVAL);
      }
      Coeff &C = b->coeffs_host[i][k];
      C.a0 = c.a0;
      C.nmodes = c.nmodes;
      for (int q = 0; q < c.nmodes; q++) {
        C.ac[q] = c.ac ? c.ac[q] : 0.0;
        C.as[q] = c.as ? c.as[q] : 0.0;
        C.om[q] = c.om[q];
      }
    }
    const bool mf = it.nterms == 2 && it.terms[0].kind == MAGNUS_TERM_XXZ && it.terms[1].kind == MAGNUS_TERM_FIELD_X &&
                    it.terms[0].nspins == it.terms[1].nspins;
    const int fam = all_csr ? FAM_CSR : (mf ? FAM_MF : FAM_GENERIC);
    fam_all = (fam_all < 0 || fam_all == fam) ? fam : FAM_GENERIC;
    if (mf) b->lbits[i] = std::max(1, it.terms[0].nspins / 2);
  }
  b->fam = fam_all;

  BCREATE(balloc(b, &b->terms, (size_t)count * kMaxTerms));
  BCREATE(balloc(b, &b->coeffs, (size_t)count * kMaxTerms));
  BCREATE(balloc(b, &b->term_ab, (size_t)count * 2 * kMaxTerms));
  BCREATE(balloc(b, &b->xi, o.m_max + 1));
  BCREATE(balloc(b, &b->cand, 2 * (o.m_max + 1)));
  BCREATE(balloc(b, &b->counter, 1));
  BCREATE(balloc(b, &b->next, 2));
  BCREATE(balloc(b, &b->counters, 1));
  BCREATE(balloc(b, &b->order, count));
  BCREATE(balloc(b, &b->nterms_dev, count));
  BCREATE(balloc(b, &b->items_dev, count));
  size_t total = 0;
  b->scratch_off.resize(count);
  for (int i = 0; i < count; i++) {
    b->scratch_off[i] = total;
    total += (size_t)b->dims[i] * (3 + b->nterms[i]);
  }
  BCREATE(balloc(b, &b->scratch, total));

  // real-valued flags of CSR terms, terms and coefficients to the device
  int *flags = nullptr;
  BCREATE(balloc(b, &flags, (size_t)count * kMaxTerms));
  BCREATE(cudaMemsetAsync(flags, 0, sizeof(int) * count * kMaxTerms, b->stream));
  for (int i = 0; i < count; i++)
    for (int k = 0; k < b->nterms[i]; k++)
      if (b->terms_host[i][k].kind == MAGNUS_TERM_CSR && b->terms_host[i][k].rs == 2 && b->terms_host[i][k].nnz > 0)
        BCREATE(launch_imag_check(b->terms_host[i][k].val, b->terms_host[i][k].nnz, flags + i * kMaxTerms + k, b->stream));
  std::vector<int> fh((size_t)count * kMaxTerms);
  BCREATE(cudaMemcpyAsync(fh.data(), flags, sizeof(int) * fh.size(), cudaMemcpyDeviceToHost, b->stream));
  BCREATE(cudaStreamSynchronize(b->stream));
  std::vector<Term> tflat((size_t)count * kMaxTerms);
  std::vector<Coeff> cflat((size_t)count * kMaxTerms);
  // real-valued CSR terms stored as complex128 get a compact float64 copy of their real parts (one
  // allocation for the whole batch), as plans do
  size_t ncopy = 0;
  for (int i = 0; i < count; i++)
    for (int k = 0; k < kMaxTerms; k++) {
      Term &T = b->terms_host[i][k];
      T.real_valued = T.kind == MAGNUS_TERM_CSR && (T.rs == 1 || !fh[(size_t)i * kMaxTerms + k]);
      if (T.real_valued && T.rs == 2 && T.nnz > 0) ncopy += (size_t)T.nnz;
    }
  if (ncopy) {
    double *rc = nullptr;
    BCREATE(balloc(b, &rc, ncopy));
    int *rflag = nullptr;
    BCREATE(balloc(b, &rflag, 1));
    size_t off = 0;
    for (int i = 0; i < count; i++)
      for (int k = 0; k < kMaxTerms; k++) {
        Term &T = b->terms_host[i][k];
        if (!(T.real_valued && T.rs == 2 && T.nnz > 0)) continue;
        BCREATE(launch_real_parts(T.val, T.nnz, rc + off, rflag, b->stream));
        T.rv = rc + off;
        T.rs = 1;
        off += (size_t)T.nnz;
      }
  }
  for (int i = 0; i < count; i++)
    for (int k = 0; k < kMaxTerms; k++) {
      tflat[(size_t)i * kMaxTerms + k] = b->terms_host[i][k];
      cflat[(size_t)i * kMaxTerms + k] = b->coeffs_host[i][k];
    }
  BCREATE(cudaMemcpyAsync(b->terms, tflat.data(), sizeof(Term) * tflat.size(), cudaMemcpyHostToDevice, b->stream));
  BCREATE(cudaMemcpyAsync(b->coeffs, cflat.data(), sizeof(Coeff) * cflat.size(), cudaMemcpyHostToDevice, b->stream));

  // per item: Gershgorin enclosures, diagonal tables of matrix-free chains; shared Leja points
  double *gscratch = nullptr;
  const int gblk = 256;
  BCREATE(balloc(b, &gscratch, 2 * gblk));
  b->dlo.assign(count, nullptr);
  b->dhi.assign(count, nullptr);
  for (int i = 0; i < count; i++) {
    const int64_t D = b->dims[i];
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(gblk, (D + 255) / 256));
    for (int k = 0; k < b->nterms[i]; k++)
      BCREATE(launch_gershgorin(b->terms + (size_t)i * kMaxTerms + k, b->terms_host[i][k], D, gscratch, nb,
                                b->term_ab + (size_t)i * 2 * kMaxTerms + 2 * k, b->stream));
    if (b->fam == FAM_MF) {
      const int n = b->terms_host[i][0].nspins, L = b->lbits[i];
      double *lo_ = nullptr, *hi_ = nullptr;
      BCREATE(balloc(b, &lo_, (size_t)1 << (L + 1)));
      BCREATE(balloc(b, &hi_, (size_t)1 << (n - L)));
      BCREATE(launch_xxz_diag_tables(b->terms + (size_t)i * kMaxTerms, n, L, lo_, hi_, b->stream));
      b->dlo[i] = lo_;
      b->dhi[i] = hi_;
    }
  }
  BCREATE(launch_leja_points(b->xi, o.m_max, b->cand, b->counter, b->stream));
  // largest problems first (longest-processing-time order)
  std::vector<int> ord(count);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return b->dims[x] > b->dims[y]; });
  BCREATE(cudaMemcpyAsync(b->order, ord.data(), sizeof(int) * count, cudaMemcpyHostToDevice, b->stream));
  b->order_host = ord;
  BCREATE(cudaMemcpyAsync(b->nterms_dev, b->nterms.data(), sizeof(int) * count, cudaMemcpyHostToDevice, b->stream));
  std::vector<double> ab((size_t)count * 2 * kMaxTerms);
  BCREATE(cudaMemcpyAsync(ab.data(), b->term_ab, sizeof(double) * ab.size(), cudaMemcpyDeviceToHost, b->stream));
  BCREATE(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < count; i++)
    for (int k = 0; k < b->nterms[i]; k++)
      if (!(ab[(size_t)i * 2 * kMaxTerms + 2 * k] <= ab[(size_t)i * 2 * kMaxTerms + 2 * k + 1])) {
        berr(b, MAGNUS_EINVAL, "item %d term %d: spectral enclosure not finite", i, k);
        return fail(MAGNUS_EINVAL);
      }

  // fixed-point pattern sums (as for plans): ||H_k||_inf from the Gershgorin enclosures, the
  // pattern terms (matrix-free transverse fields; real CSR terms with one stored value), and per
  // item the headroom bits and three Z vectors
  if (o.fixed_sums && (b->fam == FAM_CSR || b->fam == FAM_MF)) {
    int *pflag = nullptr;
    unsigned long long *prow = nullptr;
    BCREATE(balloc(b, &pflag, (size_t)count * kMaxTerms));
    BCREATE(balloc(b, &prow, (size_t)count * kMaxTerms));
    BCREATE(cudaMemsetAsync(pflag, 0, sizeof(int) * count * kMaxTerms, b->stream));
    BCREATE(cudaMemsetAsync(prow, 0, sizeof(unsigned long long) * count * kMaxTerms, b->stream));
    std::vector<double> v0((size_t)count * kMaxTerms, 0.0);
    for (int i = 0; i < count; i++)
      for (int k = 0; k < b->nterms[i]; k++) {
        const Term &T = b->terms_host[i][k];
        if (b->fam != FAM_CSR) continue;
        const size_t q = (size_t)i * kMaxTerms + k;
        if (T.kind != MAGNUS_TERM_CSR || !T.real_valued) continue;  // real-valued CSR only
        if (T.nnz <= 0) continue;
        BCREATE(launch_pattern_check(T.rowptr, T.rv, T.rs, b->dims[i], pflag + q, prow + q, b->stream));
        BCREATE(cudaMemcpyAsync(v0.data() + q, T.rv, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
      }
    std::vector<int> pf((size_t)count * kMaxTerms);
    std::vector<unsigned long long> pr((size_t)count * kMaxTerms);
    BCREATE(cudaMemcpyAsync(pf.data(), pflag, sizeof(int) * pf.size(), cudaMemcpyDeviceToHost, b->stream));
    BCREATE(cudaMemcpyAsync(pr.data(), prow, sizeof(unsigned long long) * pr.size(), cudaMemcpyDeviceToHost, b->stream));
    BCREATE(cudaStreamSynchronize(b->stream));
    b->zhb.assign(count, 1);
    b->zreal.assign(count, 1);
    b->zoff.resize(count);
    size_t ztotal = 0, ftotal = 0, etotal = 0;
    std::vector<size_t> foff((size_t)count * kMaxTerms, SIZE_MAX), eoff((size_t)count * kMaxTerms, 0);
    for (int i = 0; i < count; i++) {
      int zhb = 1;
      for (int k = 0; k < b->nterms[i]; k++) {
        Term &T = b->terms_host[i][k];
        const size_t q = (size_t)i * kMaxTerms + k;
        T.gnorm = std::max(std::fabs(ab[2 * q]), std::fabs(ab[2 * q + 1])) * (1.0 + 0x1p-40);
        int bits = 0;
        if (b->fam == FAM_MF && k == 1) {
          while ((1 << bits) < T.nspins) bits++;
          T.pattern = 1;
          T.pval = 1.0;
          T.pbits = bits;
        } else if (b->fam == FAM_CSR) {
          b->zreal[i] &= T.real_valued ? 1 : 0;
          if (T.real_valued && T.nnz > 0) {
            while (bits < 40 && (1ull << bits) < pr[q]) bits++;
            if (!(pf[q] & 1)) {
              T.pattern = 1;
              T.pval = v0[q];
              T.pbits = bits;
              T.plen = (pf[q] & 2) || pr[q] > (1u << 20) ? 0 : (int)pr[q];
            } else if (bits <= 30) {  // fixed-point products: mantissas at offset foff, exponents at eoff
              foff[q] = ftotal;
              eoff[q] = etotal;
              ftotal += (size_t)T.nnz;
              etotal += (size_t)b->dims[i];
              zhb = std::max(zhb, bits - 2);
            }
          }
        }
        if (T.pattern) zhb = std::max(zhb, std::min(T.pbits, 30) + 1);
      }
      b->zhb[i] = zhb;
      b->zoff[i] = ztotal;
      ztotal += (size_t)3 * b->dims[i];
      for (int k = 0; k < kMaxTerms; k++) tflat[(size_t)i * kMaxTerms + k] = b->terms_host[i][k];
    }
    BCREATE(balloc(b, &b->zscratch, ztotal));
    if (ftotal) {  // row-scaled mantissas of the real CSR terms that are not patterns
      long long *fv = nullptr;
      int16_t *fe = nullptr;
      int *wide = nullptr;
      BCREATE(balloc(b, &fv, ftotal));
      BCREATE(balloc(b, &fe, etotal));
      BCREATE(balloc(b, &wide, (size_t)count * kMaxTerms));
      BCREATE(cudaMemsetAsync(wide, 0, sizeof(int) * count * kMaxTerms, b->stream));
      for (int i = 0; i < count; i++)
        for (int k = 0; k < b->nterms[i]; k++) {
          const size_t q = (size_t)i * kMaxTerms + k;
          if (foff[q] == SIZE_MAX) continue;
          const Term &T = b->terms_host[i][k];
          BCREATE(launch_fixed_values(T.rowptr, T.rv, T.rs, b->dims[i], fv + foff[q], fe + eoff[q], wide + q, b->stream));
        }
      std::vector<int> wh((size_t)count * kMaxTerms);
      BCREATE(cudaMemcpyAsync(wh.data(), wide, sizeof(int) * wh.size(), cudaMemcpyDeviceToHost, b->stream));
      BCREATE(cudaStreamSynchronize(b->stream));
      for (int i = 0; i < count; i++)
        for (int k = 0; k < b->nterms[i]; k++) {
          const size_t q = (size_t)i * kMaxTerms + k;
          if (foff[q] == SIZE_MAX || wh[q]) continue;  // out-of-range values keep FP64 products
          Term &T = b->terms_host[i][k];
          T.fval = fv + foff[q];
          T.fexp = fe + eoff[q];
          tflat[q] = T;
        }
    }
    BCREATE(cudaMemcpyAsync(b->terms, tflat.data(), sizeof(Term) * tflat.size(), cudaMemcpyHostToDevice, b->stream));
    BCREATE(cudaStreamSynchronize(b->stream));
    b->zf = true;
  }
#undef BCREATE
  *out = b;
  return MAGNUS_OK;
}

MAGNUS_API magnus_status magnus_batch_destroy(magnus_batch_t b) {
  batch_free(b);
  return MAGNUS_OK;
}

MAGNUS_API magnus_status magnus_batch_propagate(magnus_batch_t b, void *const *psi, double t0, double h,
                                                int64_t nsteps, int32_t variant, magnus_batch_stats *stats) {
  NvtxRange nvtx_range("magnus_batch_propagate");
  if (!b) return berr(nullptr, MAGNUS_EINVAL, "batch is null");
  b->err.clear();
  if (!psi) return berr(b, MAGNUS_EINVAL, "psi array is null");
  for (int i = 0; i < b->count; i++)
    if (!psi[i] || ((uintptr_t)psi[i]) % 16) return berr(b, MAGNUS_EINVAL, "psi[%d] null or not 16-byte aligned", i);
  const int per = exps_per_step(variant);
  if (per == 0) return berr(b, MAGNUS_EINVAL, "unknown variant %d", variant);
  if (variant == MAGNUS_M6) return berr(b, MAGNUS_EINVAL, "batches take M2, M4, CF4 and CF4_3");
  if (nsteps < 0 || !(h == h) || !(t0 == t0)) return berr(b, MAGNUS_EINVAL, "bad nsteps / t0 / h");
  int32_t *ulog = stats ? stats->m_log : nullptr;
  const int64_t ucap = stats ? stats->m_log_cap_per_item : 0;
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->m_log = ulog;
    stats->m_log_cap_per_item = ucap;
  }
  if (nsteps == 0) return MAGNUS_OK;
  const int64_t nexp = nsteps * per;
  if (nexp > b->recs_cap) {
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    BTRY(b, balloc(b, &b->recs, (size_t)b->count * nexp));
    BTRY(b, balloc(b, &b->dd, (size_t)b->count * nexp * (b->opt.m_max + 1)));
    b->recs_cap = nexp;
  }
  const int want_log = (ulog && ucap > 0) ? 1 : 0;
  if (want_log && ucap > b->mlog_cap) {
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    BTRY(b, balloc(b, &b->mlog, (size_t)b->count * ucap));
    b->mlog_cap = ucap;
  }
  // item descriptors (the caller's state pointers may change between calls)
  b->items_host.resize(b->count);
  for (int i = 0; i < b->count; i++) {
    BatchItem &I = b->items_host[i];
    const int64_t D = b->dims[i];
    double2 *base = b->scratch + b->scratch_off[i];
    I.dim = D;
    I.nterms = b->nterms[i];
    I.lbits = b->lbits[i];
    I.terms = b->terms + (size_t)i * kMaxTerms;
    I.dlo = b->dlo[i];
    I.dhi = b->dhi[i];
    I.recs = b->recs + (size_t)i * b->recs_cap;
    I.dd = b->dd + (size_t)i * b->recs_cap * (b->opt.m_max + 1);
    I.psi = (double2 *)psi[i];
    I.alt = base;
    I.w0 = base + D;
    I.w1 = base + 2 * D;
    I.u = base + 3 * D;
    I.mlog = want_log ? b->mlog + (size_t)i * b->mlog_cap : nullptr;
    I.mlog_cap = want_log ? (int)std::min<int64_t>(b->mlog_cap, 1 << 30) : 0;
    I.zc = b->zf ? b->zscratch + b->zoff[i] : nullptr;
    I.zw0 = b->zf ? I.zc + D : nullptr;
    I.zw1 = b->zf ? I.zc + 2 * D : nullptr;
    I.zhb = b->zf ? b->zhb[i] : 0;
    I.zreal = b->zf ? b->zreal[i] : 1;
  }
  BTRY(b, cudaMemcpyAsync(b->items_dev, b->items_host.data(), sizeof(BatchItem) * b->count, cudaMemcpyHostToDevice,
                          b->stream));
  // autotune the CTA size once: time each candidate on copies of the states, first steps only
  if (!b->tuned_bs) {
    if (b->opt.ctas < 0) {
      b->tuned_bs = (-b->opt.ctas) & 0xffff;            // forced CTA size (testing)
      b->tuned_cs = std::max(1, (-b->opt.ctas) >> 16);  // and cluster size in the high bits
    } else {
      size_t total = 0;
      for (int i = 0; i < b->count; i++) total += (size_t)b->dims[i];
      double2 *tune = nullptr;
      BTRY(b, balloc(b, &tune, total));
      std::vector<BatchItem> ti = b->items_host;
      size_t off = 0;
      for (int i = 0; i < b->count; i++) {
        BTRY(b, cudaMemcpyAsync(tune + off, psi[i], sizeof(double2) * b->dims[i], cudaMemcpyDeviceToDevice, b->stream));
        ti[i].psi = tune + off;
        ti[i].mlog = nullptr;
        ti[i].mlog_cap = 0;
        off += (size_t)b->dims[i];
      }
      BatchItem *tdev = nullptr;
      BTRY(b, balloc(b, &tdev, b->count));
      BTRY(b, cudaMemcpyAsync(tdev, ti.data(), sizeof(BatchItem) * b->count, cudaMemcpyHostToDevice, b->stream));
      const int cands[4] = {128, 256, 512, 1024};
      const int clusters[3] = {1, 2, 4};
      const int64_t tsteps = std::min<int64_t>(nsteps, 2);
      double best = 1e30;
      b->tune_ms.clear();
      for (int cs : clusters)
        for (int bs : cands) {
          BTRY(b, cudaEventRecord(b->ev0, b->stream));
          magnus_status s = enqueue_run(b, variant, t0, h, tsteps, bs, cs, tdev);
          if (s != MAGNUS_OK) return s;
          BTRY(b, cudaEventRecord(b->ev1, b->stream));
          BTRY(b, cudaStreamSynchronize(b->stream));
          float ms = 0.f;
          BTRY(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
          b->tune_ms.push_back(ms);
          if (ms < best) { best = ms; b->tuned_bs = bs; b->tuned_cs = cs; }
        }
    }
  }
  // graph of (setup launches + persistent kernel), captured once per (t0, h, nsteps, variant)
  const bool same = b->graph && b->g_t0 == t0 && b->g_h == h && b->g_nsteps == nsteps && b->g_variant == variant &&
                    b->g_bs == b->tuned_bs && b->g_mlog == want_log;  // tuning happens once, before any graph
  if (!same) {
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    cudaGraph_t g = nullptr;
    BTRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    magnus_status s = enqueue_run(b, variant, t0, h, nsteps, b->tuned_bs, b->tuned_cs, b->items_dev);
    cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
    if (s != MAGNUS_OK) { if (g) cudaGraphDestroy(g); return s; }
    BTRY(b, ce);
    cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    BTRY(b, ie);
    b->g_t0 = t0; b->g_h = h; b->g_nsteps = nsteps; b->g_variant = variant; b->g_bs = b->tuned_bs; b->g_mlog = want_log;
  }
  BTRY(b, cudaEventRecord(b->ev0, b->stream));
  BTRY(b, cudaGraphLaunch(b->graph, b->stream));
  BTRY(b, cudaEventRecord(b->ev1, b->stream));
  Counters c{};
  BTRY(b, cudaMemcpyAsync(&c, b->counters, sizeof c, cudaMemcpyDeviceToHost, b->stream));
  BTRY(b, cudaStreamSynchronize(b->stream));
  if (stats) {
    float ms = 0.f;
    BTRY(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    stats->n_exp = c.n_exp;
    stats->n_substeps = c.n_substeps;
    stats->n_matvec = c.n_matvec;
    stats->n_termapply = c.n_termapply;
    stats->max_m = c.max_m;
    stats->status = c.status;
    stats->graph_ms = ms;
    stats->block = b->tuned_bs;
    stats->cluster = b->tuned_cs;
    stats->fixed_sums = b->zf && variant != MAGNUS_M4;
    if (want_log) {
      std::vector<int> tmp((size_t)b->count * b->mlog_cap);
      BTRY(b, cudaMemcpyAsync(tmp.data(), b->mlog, sizeof(int) * tmp.size(), cudaMemcpyDeviceToHost, b->stream));
      BTRY(b, cudaStreamSynchronize(b->stream));
      for (int i = 0; i < b->count; i++)
        memcpy(ulog + (size_t)i * ucap, tmp.data() + (size_t)i * b->mlog_cap, sizeof(int) * ucap);
    }
  }
  if (c.status != MAGNUS_OK)
    return berr(b, (magnus_status)c.status, "%s",
                c.status == MAGNUS_ENOCONV ? "Leja interpolation did not converge within m_max" : "non-finite norm");
  return MAGNUS_OK;
}

}  // extern "C"
