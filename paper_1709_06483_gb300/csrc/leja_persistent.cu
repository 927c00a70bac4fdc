// The hot path: one persistent, cooperative launch runs a whole Magnus propagation
// (arXiv:1709.06483, Sec. 2, Y_{n+1} = exp(Omega_n) Y_n) with every exponential applied by the
// Newton-form Leja recurrence of Sec. 3:
//     w = v, p = d_0 v;   for j = 1..m:  w <- X w - xi_{j-1} w,  p <- p + d_j w,
// X = (K - cI)/gamma, stopped early once |d_j| ||w_j|| + |d_{j-1}| ||w_{j-1}|| <= tol_abs + tol_rel ||p||.
// The paper runs this loop on the CPU and only the vector operations on the GPU (Sec. 3); here
// the loop control stays on the device: each Leja iteration is one fused pass (matvec of every
// term + shift + Newton update of p + partial norms), followed by one grid barrier after which
// every block reads the same per-block partial sums in the same order and so takes the same
// stop decision.  M4 (Sec. 2, Method M4) applies its commutator matrix-free,
// [H_2, H_1] w = sum_{k<l} coef_kl (H_k (H_l w) - H_l (H_k w)), with one extra barrier between
// the two term applications.
//
// On GB300 the FP64 pipe (2 FMA/clk/SM) is the tighter limit for these matvecs, so the kernel is
// specialised at compile time per operator family to keep the FP64 instruction count per row
// minimal and many independent loads in flight:
//   FAM_CSR     every term CSR (real-valued values multiply only the real parts);
//   FAM_MF      matrix-free XXZ chain + transverse field, diagonal from two small tables;
//   FAM_GENERIC any mix of CSR and matrix-free terms;
// and per arithmetic: ZF = 0 FP64 throughout; ZF = 1 (linear generators) and ZF = 2 (M4) take the
// matvecs in fixed point on int64 copies of the vectors (exact sums of pattern terms, products of
// row-scaled value mantissas, rows.cuh), which leaves 14 FP64 instructions per row.
// Vectors written by other blocks between barriers are read with ordinary (coherent, L1-cached)
// loads; only the immutable matrices use the read-only path.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "magnus_internal.cuh"
#include "persist_common.cuh"
#include "rows.cuh"
#include "csr_stage.cuh"

namespace mg {

namespace {

using namespace rows;

constexpr int kBlock = 256;
// Resident CTAs per SM the register budget targets: 4 (64 registers) for the CSR family with
// fixed-point pattern sums, whose time goes to gather latency that more warps hide; 3 (80
// registers) for the matrix-free family, which is FP64-bound and spills at 64, and for the others.
#ifndef MG_CSR_MIN_BLOCKS
#define MG_CSR_MIN_BLOCKS 4
#endif
template <int FAM, bool HM6, int ZF>
constexpr int min_blocks() {
  return (FAM == FAM_CSR && ZF == 1) ? MG_CSR_MIN_BLOCKS : 3;
}
constexpr int kMaxVec = 64;


// M6 intermediate vectors (slots of PersistArgs::m6), named by the operator word applied to w, u
// or v: e.g. PQW = P(Q w).
enum {
  S_PW, S_QW, S_RW, S_PQW, S_QPW, S_PRW, S_RPW, S_PPW, S_U, S_V, S_PU, S_QU, S_RU, S_PV, S_QV, S_RV,
  S_PQU, S_QPU, S_PRU, S_RPU, S_PPU, S_PQV, S_QPV
};
static_assert(S_QPV + 1 == kM6Slots, "M6 slot count");

__device__ __forceinline__ double2 mul_i(double2 z) { return make_double2(-z.y, z.x); }  // i z
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 sub2(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 scal2(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// --------------------------------------------------------------------- kernel
// HM6: the instantiation that also carries Method M6 (launched only for MAGNUS_M6, so that its
// extra code does not weigh on the register budget of the other methods).  ZF: the instantiations
// with fixed-point sums and products (options.fixed_sums): 1 for linear generators (M2, Cf4, Cf4:3),
// which carries only that path, 2 for M4 (its two phases on fixed-point copies of w and of u_k).
// STG: the fixed-point CSR instantiation whose rows read the sliced matrix from shared memory,
// staged per warp tile by the TMA bulk engine (csr_stage.cuh); two CTAs of 8 warps per SM hold the
// slots.
template <int FAM, bool HM6, int ZF, bool STG = false>
__global__ void __launch_bounds__(kBlock, (STG ? 2 : min_blocks<FAM, HM6, ZF>())) k_magnus_persistent(PersistArgs a) {
  static_assert(!STG || (FAM == FAM_CSR && ZF == 1 && !HM6), "staged rows: fixed-point CSR linear generators");
  extern __shared__ __align__(128) unsigned char s_dyn[];
  __shared__ __align__(8) uint64_t s_sbar[STG ? 2 * stage::kWarps : 1];
  __shared__ Term sT[kMaxTerms];
  __shared__ ExpRec sR;
  __shared__ double s_jb[kMaxSpins], s_j2[kMaxSpins];
  __shared__ double s_vn[kMaxVec], s_ep[kMaxVec], s_pn[kMaxVec];
  // largest component max(|Re|, |Im|) of the substep input, of p at the stop and of the last w
  __shared__ double s_vm[kMaxVec], s_pm[kMaxVec], s_wm[kMaxVec];
  __shared__ double s_wz[kMaxTerms];  // weights of the fixed-point pattern sums: bg_k v_k
  __shared__ long long s_cb[kMaxSpins];  // FAM_MF fixed point: bond weights as 62-bit mantissas
  __shared__ int s_cbe;
  __shared__ long long s_c2[kMaxSpins];  // FAM_MF fixed-point M4: the unscaled weights 2 J likewise
  __shared__ int s_c2e;
  __shared__ int s_act[kMaxVec], s_m[kMaxVec];
  __shared__ double s_red[2][kBlock / 32];
  __shared__ unsigned s_rmx[2][kBlock / 32];
  __shared__ int s_flag;
  __shared__ int s_drift;  // the norm check of the last substep failed
  __shared__ int s_kp;  // staged rows: the pattern term whose rows of one length are read as 16-byte loads

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned G = gridDim.x;
  const int b = blockIdx.x;
  const int vec = b / a.gv, chunk = b % a.gv;
  const int64_t D = a.dim;
  // rows per block rounded up to whole warps, so that each warp owns 32 consecutive rows
  const int64_t rows_per = (((D + a.gv - 1) / a.gv) + 31) & ~(int64_t)31;
  const int64_t lo = min(D, (int64_t)chunk * rows_per), hi = min(D, lo + rows_per);
  // The row loops take r = r_lo + tid, r_lo + tid + r_step, ... below r_hi.  Except for the staged
  // rows (whose warp tiles need [lo, hi)), the vector's blocks take its rows in interleaved passes
  // of blockDim.x rows, so that each block's rows come from the whole range: row lengths follow the
  // high bits of the row index in spin-chain terms, and a contiguous range would give blocks whole
  // regions of long or short rows (measured on the 20-spin chain: the slowest block's rows took 12 %
  // longer than the mean; interleaved, the Leja iteration takes 101 instead of 106 us).
  const bool ilv = !STG;
  const int64_t r_lo = ilv ? (int64_t)chunk * blockDim.x : lo;
  const int64_t r_hi = ilv ? D : hi;
  const int64_t r_step = ilv ? (int64_t)a.gv * blockDim.x : (int64_t)blockDim.x;
  const int64_t base = (int64_t)vec * D;
  const int nt = a.nterms, nv = a.nvec;

  for (int i = tid; i < nt * (int)sizeof(Term) / 4; i += blockDim.x)
    reinterpret_cast<int *>(sT)[i] = reinterpret_cast<const int *>(a.terms)[i];
  if (tid == 0) {
    s_kp = -1;
    for (int k = 0; k < nt; k++)
      if (s_kp < 0 && sT[k].pattern && sT[k].plen > 0 && sT[k].plen <= 20 && (sT[k].plen & 3) == 0) s_kp = k;
  }
  __syncthreads();
  Ctx cx{};
  cx.T = sT;
  cx.nt = nt;
  cx.n = sT[0].nspins;
  cx.lbits = a.lbits;
  cx.lomask = ((int64_t)1 << (a.lbits + 1)) - 1;
  cx.dlo = a.dlo;
  cx.dhi = a.dhi;
  cx.jb = s_jb;
  cx.j2 = s_j2;
  cx.cb = (ZF && FAM == FAM_MF) ? s_cb : nullptr;
  cx.cbe = 0;
  cx.c2 = (ZF == 2 && FAM == FAM_MF) ? s_c2 : nullptr;
  cx.c2e = 0;
  if (FAM == FAM_MF) {
    // bond at bits (p, p-1) couples spins s = n-p and s+1 with J[s-1] = J[n-p-1]
    for (int p = 1 + tid; p < cx.n; p += blockDim.x) s_j2[p - 1] = 2.0 * sT[0].J[cx.n - p - 1];
    if (ZF == 2) {
      __syncthreads();
      if (tid == 0) {
        double wmax = 0.0;
        for (int p = 0; p < cx.n - 1; p++) wmax = fmax(wmax, fabs(s_j2[p]));
        int E = 0;
        if (wmax > 0.0) frexp(wmax, &E);
        E = max(-400, min(400, E));
        for (int p = 0; p < cx.n - 1; p++) s_c2[p] = llrint(ldexp(s_j2[p], 62 - E));
        s_c2e = E;
      }
      __syncthreads();
      cx.c2e = s_c2e;
    }
  }

  unsigned it = 0;  // slot counter of the partial sums: consecutive reductions alternate slots
  // per block: two sums and two maxima (high words of non-negative doubles, abshi)
  auto block_reduce_store = [&](double x0, double x1, unsigned m0, unsigned m1) {
    x0 = warp_sum(x0);
    x1 = warp_sum(x1);
    m0 = __reduce_max_sync(kFull, m0);
    m1 = __reduce_max_sync(kFull, m1);
    if (lane == 0) { s_red[0][warp] = x0; s_red[1][warp] = x1; s_rmx[0][warp] = m0; s_rmx[1][warp] = m1; }
    __syncthreads();
    if (tid == 0) {
      double y0 = 0.0, y1 = 0.0;
      unsigned n0 = 0, n1 = 0;
      for (int w = 0; w < kBlock / 32; w++) {
        y0 += s_red[0][w];
        y1 += s_red[1][w];
        n0 = max(n0, s_rmx[0][w]);
        n1 = max(n1, s_rmx[1][w]);
      }
      double *slot = a.partials + (size_t)(it & 1u) * G * 4;
      slot[4 * b] = y0;
      slot[4 * b + 1] = y1;
      slot[4 * b + 2] = __hiloint2double((int)n0, 0);
      slot[4 * b + 3] = __hiloint2double((int)n1, 0);
    }
  };
  // totals of vector v from the current slot, identical in every block (fixed order), and upper
  // bounds of its two maxima
  auto vector_totals = [&](int v, double &t0, double &t1, double *mx0 = nullptr, double *mx1 = nullptr) {
    const double *slot = a.partials + (size_t)(it & 1u) * G * 4;
    double y0 = 0.0, y1 = 0.0;
    unsigned n0 = 0, n1 = 0;
    for (int q = lane; q < a.gv; q += 32) {
      const double *pq = slot + 4 * (v * a.gv + q);
      y0 += pq[0];
      y1 += pq[1];
      n0 = max(n0, (unsigned)__double2hiint(pq[2]));
      n1 = max(n1, (unsigned)__double2hiint(pq[3]));
    }
    t0 = warp_sum(y0);
    t1 = warp_sum(y1);
    if (mx0) *mx0 = abshi_bound(__reduce_max_sync(kFull, n0));
    if (mx1) *mx1 = abshi_bound(__reduce_max_sync(kFull, n1));
  };
  auto fail = [&](int status) {
    if (tid == 0) atomicCAS(&a.counters->status, 0, status);
  };
  // staged rows: the warp's copy pipeline (its copies run across Leja iterations)
  stage::Pipe P{};
  if constexpr (STG) stage::init(P, s_dyn, s_sbar, warp, lane, lo, hi);
  // leave the kernel: report the status and wait for the copies still in flight
  auto bail = [&](int status) {
    fail(status);
    if constexpr (STG) stage::drain(P, a.spin_limit_ns);
  };

  // ||psi|| and the largest component of every vector
  {
    double s = 0.0;
    unsigned mx = 0;
    for (int64_t r = r_lo + tid; r < r_hi; r += r_step) {
      const double2 v = a.psi[base + r];
      s += cabs2(v);
      mx = max(mx, abshi(v));
    }
    block_reduce_store(s, 0.0, mx, 0);
    // testing hook: CTA 0 leaves before its first barrier (a participant that never arrives), so
    // that every other CTA's bounded wait runs out
    if (a.skip_arrival && b == 0) return;
    if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { bail(MAGNUS_ETIMEOUT); return; }
    if (warp == 0)
      for (int v = 0; v < nv; v++) {
        double t0, t1, m0;
        vector_totals(v, t0, t1, &m0);
        if (lane == 0) {
          s_vn[v] = sqrt(t0);
          s_vm[v] = m0;
        }
      }
    __syncthreads();
    it++;
  }

  double2 *cur = a.psi, *nxt = a.alt;
  long long sub_counter = 0;
  for (int64_t e = 0; e < a.nexp; e++) {
    __syncthreads();
    if (tid == 0) sR = a.recs[e];
    __syncthreads();
    const ExpRec &R = sR;
    if (FAM == FAM_MF)
      for (int p = 1 + tid; p < cx.n; p += blockDim.x) s_jb[p - 1] = s_j2[p - 1] * R.bg[0];
    // fixed-point pattern sums: linear generators of the CSR and matrix-free families
    constexpr bool zf = ZF != 0 && FAM != FAM_GENERIC;
    // the host launches ZF = 1 for linear generators and ZF = 2 for M4 (whose records may be linear)
    if ((ZF == 1 && R.mode != MODE_LINEAR) || (ZF == 2 && R.mode != MODE_LINEAR && R.mode != MODE_M4)) {
      bail(MAGNUS_EINVAL);
      return;
    }
    // sum_k |bg_k| ||H_k||_inf (+ the M4 commutator's sum_{k<l} |kg| 2 ||H_k||_inf ||H_l||_inf): with
    // |shift|, a bound of ||X - shift||_inf
    double opnorm = 0.0;
    if (zf) {
      if (tid < nt) s_wz[tid] = R.bg[tid] * sT[tid].pval;
      for (int k = 0; k < nt; k++) opnorm = fma(fabs(R.bg[k]), sT[k].gnorm, opnorm);
      if (ZF == 2 && R.mode == MODE_M4)
        for (int k = 0, pi = 0; k < nt; k++)
          for (int l = k + 1; l < nt; l++, pi++) opnorm = fma(fabs(R.kg[pi]), 2.0 * sT[k].gnorm * sT[l].gnorm, opnorm);
      if (FAM == FAM_MF) {  // bond weights 2 J bg_0 as mantissas at one exponent: max |w| < 2^s_cbe
        __syncthreads();
        if (tid == 0) {
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
    }
    const double2 *d = a.dd + e * (int64_t)(a.m_max + 1);
    if (!(R.gamma > 0.0)) {  // scalar generator: a phase
      const double2 ph = d[0];
      for (int64_t r = r_lo + tid; r < r_hi; r += r_step) nxt[base + r] = cmul(ph, cur[base + r]);
      if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { bail(MAGNUS_ETIMEOUT); return; }
      if (tid < nv) s_vm[tid] *= sqrt(cabs2(ph)) * (1.0 + 0x1p-40);
      double2 *tmp = cur; cur = nxt; nxt = tmp;
      if (b == 0 && tid == 0) a.counters->n_exp++;
      continue;
    }
    const double2 d0 = d[0];
    for (int sub = 0; sub < R.s; sub++) {
      if (tid < nv) {
        s_act[tid] = 1;
        s_ep[tid] = sqrt(cabs2(d0)) * s_vn[tid];
        s_m[tid] = 0;
      }
      __syncthreads();
      int zs_src = 0;  // scale of the Z copy of this iteration's input
      if (zf) {        // Z copy of the substep input
        zs_src = fix_scale(s_vm[vec], a.zhb);
        for (int64_t r = r_lo + tid; r < r_hi; r += r_step) a.zc[base + r] = fix2(cur[base + r], zs_src);
        if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { bail(MAGNUS_ETIMEOUT); return; }
      }
      bool done = false;
      int j;
      for (j = 1; j <= a.m_max; j++) {
        const double2 *src = (j == 1) ? cur : (((j - 2) & 1) ? a.w1 : a.w0);
        double2 *dst = ((j - 1) & 1) ? a.w1 : a.w0;
        const double shift = R.cg + a.xi[j - 1];
        const double2 dj = d[j];
        const bool mine = s_act[vec] != 0;
        if (!ZF && R.mode == MODE_M4) {
          // phase 1: u_k = H_k w for this block's rows
          if (mine)
            for (int64_t r = r_lo + tid; r < r_hi; r += r_step)
              for (int k = 0; k < nt; k++) a.u[((size_t)k * nv) * D + base + r] = Op<FAM>::term(cx, k, src + base, r);
          if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { bail(MAGNUS_ETIMEOUT); return; }
        }
        // fixed-point M4, phase 1: u_k = H_k w from the copy of w, and the copy of u_k, scaled from
        // |u_k| <= ||H_k||_inf max|w| (x2 for complex terms)
        int zs_u[kMaxTerms] = {0, 0, 0, 0};
        if constexpr (ZF == 2 && zf) {
          if (R.mode == MODE_M4) {
            const double msrc = (j == 1) ? s_vm[vec] : s_wm[vec];
            const longlong2 *zw = ((j == 1) ? a.zc : (((j - 2) & 1) ? a.zw1 : a.zw0)) + base;
            for (int k = 0; k < nt; k++)
              zs_u[k] = fix_scale(sT[k].gnorm * (a.zreal ? 1.0 : 2.0) * msrc * (1.0 + 0x1p-20), a.zhb);
            if (mine)
              for (int64_t r = r_lo + tid; r < r_hi; r += r_step)
                for (int k = 0; k < nt; k++) {
                  const double2 hk = Op<FAM>::term_z(cx, k, src + base, zw, zs_src, r);
                  a.u[((size_t)k * nv) * D + base + r] = hk;
                  a.zu[((size_t)k * nv) * D + base + r] = fix2(hk, zs_u[k]);
                }
            if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { bail(MAGNUS_ETIMEOUT); return; }
          }
        }
        // Method M6: K w = P w + R w / 12 + (i/240) (U (V w) - V (U w)) with
        //   U = i(20 P + R) - [P, Q],   V = -i Q + [P, R]/30 - (i/60) [P, [P, Q]],
        // built in five passes over this block's rows, each followed by a grid barrier; every pass
        // applies the terms once per input vector and forms all combinations it needs.
        if (HM6 && R.mode == MODE_M6) {
          const size_t sl = (size_t)nv * D;
          auto V6 = [&](int k) { return a.m6 + (size_t)k * sl + base; };
          double2 t[kMaxTerms];
          auto terms_of = [&](const double2 *x, int64_t r) {
            for (int k = 0; k < nt; k++) t[k] = Op<FAM>::term(cx, k, x, r);
          };
          auto lc = [&](const double *c) {
            double2 z = make_double2(0.0, 0.0);
            for (int k = 0; k < nt; k++) z = rfma(c[k], t[k], z);
            return z;
          };
          const double *P6 = R.p6, *Q6 = R.q6, *R6 = R.r6;
          if (mine)  // pass 1: P w, Q w, R w
            for (int64_t r = r_lo + tid; r < r_hi; r += r_step) {
              terms_of(src + base, r);
              V6(S_PW)[r] = lc(P6);
              V6(S_QW)[r] = lc(Q6);
              V6(S_RW)[r] = lc(R6);
            }
          if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { bail(MAGNUS_ETIMEOUT); return; }
          if (mine)  // pass 2: P(Q w), Q(P w), R(P w), P(P w), P(R w)
            for (int64_t r = r_lo + tid; r < r_hi; r += r_step) {
              terms_of(V6(S_QW), r);
              V6(S_PQW)[r] = lc(P6);
              terms_of(V6(S_PW), r);
              V6(S_QPW)[r] = lc(Q6);
              V6(S_RPW)[r] = lc(R6);
              V6(S_PPW)[r] = lc(P6);
              terms_of(V6(S_RW), r);
              V6(S_PRW)[r] = lc(P6);
            }
          if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { bail(MAGNUS_ETIMEOUT); return; }
          if (mine)  // pass 3: u = U w, v = V w
            for (int64_t r = r_lo + tid; r < r_hi; r += r_step) {
              terms_of(V6(S_PQW), r);
              const double2 ppq = lc(P6);
              terms_of(V6(S_QPW), r);
              const double2 pqp = lc(P6);
              terms_of(V6(S_PPW), r);
              const double2 qpp = lc(Q6);
              const double2 pw = ldv(V6(S_PW) + r), qw = ldv(V6(S_QW) + r), rw = ldv(V6(S_RW) + r);
              const double2 pqw = ldv(V6(S_PQW) + r), qpw = ldv(V6(S_QPW) + r);
              const double2 prw = ldv(V6(S_PRW) + r), rpw = ldv(V6(S_RPW) + r);
              const double2 uw = sub2(mul_i(add2(scal2(20.0, pw), rw)), sub2(pqw, qpw));
              const double2 nest = add2(sub2(ppq, scal2(2.0, pqp)), qpp);  // [P,[P,Q]] w
              const double2 vw = sub2(add2(mul_i(scal2(-1.0, qw)), scal2(1.0 / 30.0, sub2(prw, rpw))),
                                      scal2(1.0 / 60.0, mul_i(nest)));
              V6(S_U)[r] = uw;
              V6(S_V)[r] = vw;
            }
          if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { bail(MAGNUS_ETIMEOUT); return; }
          if (mine)  // pass 4: P u, Q u, R u, P v, Q v, R v
            for (int64_t r = r_lo + tid; r < r_hi; r += r_step) {
              terms_of(V6(S_U), r);
              V6(S_PU)[r] = lc(P6);
              V6(S_QU)[r] = lc(Q6);
              V6(S_RU)[r] = lc(R6);
              terms_of(V6(S_V), r);
              V6(S_PV)[r] = lc(P6);
              V6(S_QV)[r] = lc(Q6);
              V6(S_RV)[r] = lc(R6);
            }
          if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { bail(MAGNUS_ETIMEOUT); return; }
          if (mine)  // pass 5: P(Q u), Q(P u), R(P u), P(P u), P(R u), P(Q v), Q(P v)
            for (int64_t r = r_lo + tid; r < r_hi; r += r_step) {
              terms_of(V6(S_QU), r);
              V6(S_PQU)[r] = lc(P6);
              terms_of(V6(S_PU), r);
              V6(S_QPU)[r] = lc(Q6);
              V6(S_RPU)[r] = lc(R6);
              V6(S_PPU)[r] = lc(P6);
              terms_of(V6(S_RU), r);
              V6(S_PRU)[r] = lc(P6);
              terms_of(V6(S_QV), r);
              V6(S_PQV)[r] = lc(P6);
              terms_of(V6(S_PV), r);
              V6(S_QPV)[r] = lc(Q6);
            }
          if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { bail(MAGNUS_ETIMEOUT); return; }
        }
        double sw = 0.0, sp = 0.0;
        unsigned mw = 0, mp = 0;
        int zs_dst = 0;
        if constexpr (zf) {
         if (mine) {  // linear generator with fixed-point pattern sums
          // |Re w_j|, |Im w_j| <= ||X - shift||_inf max(|Re w_{j-1}|, |Im w_{j-1}|) (x2 for complex terms)
          const double msrc = (j == 1) ? s_vm[vec] : s_wm[vec];
          zs_dst = fix_scale((opnorm + fabs(shift)) * (a.zreal ? 1.0 : 2.0) * msrc * (1.0 + 0x1p-20), a.zhb);
          const longlong2 *zsrc = ((j == 1) ? a.zc : (((j - 2) & 1) ? a.zw1 : a.zw0)) + base;
          longlong2 *zdst = (((j - 1) & 1) ? a.zw1 : a.zw0) + base;
          // p starts as d_0 v in the first iteration: its own loop, so that no other iteration
          // spends FP64 slots on that product
          auto rows_z = [&](auto first) {
            auto row = [&](int64_t r) {
              double2 wr;
              double2 y;
              double2 pold = make_double2(0.0, 0.0);
              if constexpr (!decltype(first)::value) pold = nxt[base + r];  // issued before the row's gathers
              if (ZF == 2 && R.mode == MODE_M4) {
                // phase 2: sum_k bg_k u_k + sum_{k<l} kg (H_k u_l - H_l u_k) (times -i) - shift w
                y = make_double2(0.0, 0.0);
                double2 zq = make_double2(0.0, 0.0);
                for (int k = 0, pi = 0; k < nt; k++) {
                  const size_t ok = ((size_t)k * nv) * D + base;
                  y = rfma(R.bg[k], ldv(a.u + ok + r), y);
                  for (int l = k + 1; l < nt; l++, pi++) {
                    const size_t ol = ((size_t)l * nv) * D + base;
                    const double2 hkul = Op<FAM>::term_z(cx, k, a.u + ol, a.zu + ol, zs_u[l], r);
                    const double2 hluk = Op<FAM>::term_z(cx, l, a.u + ok, a.zu + ok, zs_u[k], r);
                    zq = rfma(R.kg[pi], make_double2(hkul.x - hluk.x, hkul.y - hluk.y), zq);
                  }
                }
                y.x += zq.y;  // -i zq
                y.y -= zq.x;
                wr = ldv(src + base + r);
                y = rfma(-shift, wr, y);
              } else {
                y = Op<FAM>::combo_z(cx, R, s_wz, shift, src + base, zsrc, zs_src, r, wr);
              }
              dst[base + r] = y;
              zdst[r] = fix2(y, zs_dst);
              double2 pr;
              if constexpr (decltype(first)::value) pr = cmul(d0, wr); else pr = pold;
              pr = cfma(dj, y, pr);
              nxt[base + r] = pr;
              sw = fma(y.x, y.x, fma(y.y, y.y, sw));
              sp = fma(pr.x, pr.x, fma(pr.y, pr.y, sp));
              mw = max(mw, abshi(y));
              mp = max(mp, abshi(pr));
            };
            for (int64_t r = r_lo + tid; r < r_hi; r += r_step) row(r);
          };
          // the same rows, tile by tile: the sliced terms' heads and tails from the warp's
          // shared-memory slots (csr_stage.cuh), the rows of one length of pattern terms from global
          // memory; every term of this instantiation is a pattern or a product term
          auto rows_staged = [&](auto first) {
            using namespace stage;
            if (P.ntiles == 0) return;
            if (!P.primed) {  // first pass: the row data of tile 0 and the copies of the first two tiles
              P.primed = true;
              int64_t ra, rb;
              tile_rows(P, lo, hi, 0, ra, rb);
              load_rowdata(P, sT, nt, ra + lane, rb);
              if (lane == 0)
                for (long long n = 0; n < 2; n++) {
                  tile_rows(P, lo, hi, tile_ahead(P, (int)n), ra, rb);
                  Span S;
                  load_span(sT, nt, ra, rb, S);
                  issue(P, sT, nt, n, S);
                }
              P.issued = 2;
              __syncwarp();
            }
            for (int jt = 0; jt < P.ntiles; jt++) {
              const long long n = P.consumed;
              int64_t ra, rb;
              tile_rows(P, lo, hi, P.tc, ra, rb);
              const int64_t r = ra + lane;
              const bool valid = r < rb;
              long long t0[kTerms], t1[kTerms];
              int fe[kTerms];
#pragma unroll
              for (int k = 0; k < kTerms; k++) {
                t0[k] = P.nt0[k];
                t1[k] = P.nt1[k];
                fe[k] = P.nfe[k];
              }
              // columns of the rows of one length of a pattern term (no row pointer needed, at most
              // 20 entries, 16-byte aligned): issued first, as 16-byte loads
              int4 pc[5];
              const int kp = s_kp;
              const int p4 = kp >= 0 ? sT[kp].plen / 4 : 0;
              if (kp >= 0 && valid) {
                const int4 *c4 = reinterpret_cast<const int4 *>(sT[kp].col + r * sT[kp].plen);
#pragma unroll
                for (int q = 0; q < 5; q++)
                  if (q < p4) pc[q] = __ldg(c4 + q);
              }
              {  // row data of the next tile (the first tile of the next pass after the last)
                int64_t na, nb;
                tile_rows(P, lo, hi, tile_ahead(P, 1), na, nb);
                load_rowdata(P, sT, nt, na + lane, nb);
              }
              // lane 0: the runs of consumption n + 2, copied once this tile is done
              if (lane == 0) {
                int64_t qa, qb;
                tile_rows(P, lo, hi, tile_ahead(P, 2), qa, qb);
                load_span(sT, nt, qa, qb, *span_ptr(P));
              }
              const double2 wr = valid ? ldv(src + base + r) : make_double2(0.0, 0.0);
              double2 pold = make_double2(0.0, 0.0);
              if constexpr (!decltype(first)::value) pold = valid ? nxt[base + r] : pold;
              const int sl = (int)(n & 1);
              if (!wait_slot(P.bar + sl, (uint32_t)((n >> 1) & 1), a.spin_limit_ns)) {
                // the copy did not arrive: report it; every block leaves at the next barrier
                if (lane == 0) {
                  atomicCAS(&a.counters->status, 0, MAGNUS_ETIMEOUT);
                  atomicExch(&a.bar->error, 1);
                }
                break;
              }
              __syncwarp();
              const Desc &Dd = *desc_ptr(P, n);
              const unsigned char *slot = slot_ptr(P, n);
              const bool fits = Dd.fits != 0;
              double2 y = make_double2(0.0, 0.0);
              if (valid) {
                longlong2 acc[kTerms];
#pragma unroll
                for (int k = 0; k < kTerms; k++) {
                  acc[k] = make_longlong2(0, 0);
                  if (k >= nt) continue;
                  const Term &t = sT[k];
                  if (k == kp) {
#pragma unroll
                    for (int h = 0; h < 3; h++) {
                      if (2 * h >= p4) break;
                      longlong2 g[8];
#pragma unroll
                      for (int i = 0; i < 8; i++) {
                        const int4 v = pc[min(2 * h + i / 4, 4)];
                        const int cq = (i & 3) == 0 ? v.x : (i & 3) == 1 ? v.y : (i & 3) == 2 ? v.z : v.w;
                        g[i] = (2 * h + i / 4 < p4) ? ldz(zsrc + cq) : make_longlong2(0, 0);
                      }
#pragma unroll
                      for (int i = 0; i < 8; i++) zadd(acc[k], g[i]);
                    }
                  } else if (t.pattern && t.plen) {
                    acc[k] = csr_row_zsum(t, zsrc, r);
                  } else if (fits) {
                    const int32_t *hc = reinterpret_cast<const int32_t *>(slot + Dd.hc[k]) + lane;
                    const int tl = (int)(t1[k] - t0[k]);
                    const int32_t *tcp = reinterpret_cast<const int32_t *>(slot + Dd.tc[k]) +
                                         (t0[k] - (run_lo(Dd.t0[k], 4) >> 2));
                    if (t.pattern) {
                      acc[k] = zsum_staged(hc, Dd.w[k], tcp, tl, zsrc);
                    } else {
                      const long long *hv = reinterpret_cast<const long long *>(slot + Dd.hv[k]) + lane;
                      const long long *tvp = reinterpret_cast<const long long *>(slot + Dd.tv[k]) +
                                             (t0[k] - (run_lo(Dd.t0[k], 8) >> 3));
                      acc[k] = zprod_staged(hc, hv, Dd.w[k], tcp, tvp, tl, zsrc);
                    }
                  } else {
                    acc[k] = t.pattern ? sl_row_zsum(t, zsrc, r) : sl_row_zprod(t, zsrc, r);
                  }
                }
#pragma unroll
                for (int k = 0; k < kTerms; k++) {
                  if (k >= nt) continue;
                  y = sT[k].pattern ? rfma(s_wz[k], unfix2(acc[k], zs_src), y)
                                    : rfma(R.bg[k], unfix2(acc[k], zs_src - fe[k] - 2), y);
                }
                y = rfma(-shift, wr, y);
              }
              // the slot is free again: copy the runs of consumption n + 2 into it
              P.consumed = n + 1;
              P.tc = tile_ahead(P, 1);
              __syncwarp();
              if (lane == 0) {
                fence_proxy_async();
                issue(P, sT, nt, n + 2, *span_ptr(P));
              }
              P.issued = n + 3;
              if (valid) {
                dst[base + r] = y;
                zdst[r] = fix2(y, zs_dst);
                double2 pr;
                if constexpr (decltype(first)::value) pr = cmul(d0, wr); else pr = pold;
                pr = cfma(dj, y, pr);
                nxt[base + r] = pr;
                sw = fma(y.x, y.x, fma(y.y, y.y, sw));
                sp = fma(pr.x, pr.x, fma(pr.y, pr.y, sp));
                mw = max(mw, abshi(y));
                mp = max(mp, abshi(pr));
              }
            }
          };
          if constexpr (STG) {
            if (j == 1) rows_staged(std::true_type{}); else rows_staged(std::false_type{});
          } else {
            if (j == 1) rows_z(std::true_type{}); else rows_z(std::false_type{});
          }
         }
        } else if (mine) {
          for (int64_t r = r_lo + tid; r < r_hi; r += r_step) {

            double2 y, wr;
            if (HM6 && R.mode == MODE_M6) {  // pass 6: V u, U v and K w, fused with the Leja update
              const size_t sl = (size_t)nv * D;
              auto V6 = [&](int k) { return a.m6 + (size_t)k * sl + base; };
              double2 t6[kMaxTerms];
              double2 ppq = make_double2(0.0, 0.0), pqp = ppq, qpp = ppq;
              for (int k = 0; k < nt; k++) t6[k] = Op<FAM>::term(cx, k, V6(S_PQU), r);
              for (int k = 0; k < nt; k++) ppq = rfma(R.p6[k], t6[k], ppq);
              for (int k = 0; k < nt; k++) t6[k] = Op<FAM>::term(cx, k, V6(S_QPU), r);
              for (int k = 0; k < nt; k++) pqp = rfma(R.p6[k], t6[k], pqp);
              for (int k = 0; k < nt; k++) t6[k] = Op<FAM>::term(cx, k, V6(S_PPU), r);
              for (int k = 0; k < nt; k++) qpp = rfma(R.q6[k], t6[k], qpp);
              const double2 qu = ldv(V6(S_QU) + r), pru = ldv(V6(S_PRU) + r), rpu = ldv(V6(S_RPU) + r);
              const double2 nest = add2(sub2(ppq, scal2(2.0, pqp)), qpp);  // [P,[P,Q]] u
              const double2 vu = sub2(add2(mul_i(scal2(-1.0, qu)), scal2(1.0 / 30.0, sub2(pru, rpu))),
                                      scal2(1.0 / 60.0, mul_i(nest)));
              const double2 pv = ldv(V6(S_PV) + r), rv = ldv(V6(S_RV) + r);
              const double2 pqv = ldv(V6(S_PQV) + r), qpv = ldv(V6(S_QPV) + r);
              const double2 uv = sub2(mul_i(add2(scal2(20.0, pv), rv)), sub2(pqv, qpv));
              const double2 pw = ldv(V6(S_PW) + r), rw = ldv(V6(S_RW) + r);
              const double2 kw = add2(add2(pw, scal2(1.0 / 12.0, rw)), scal2(1.0 / 240.0, mul_i(sub2(uv, vu))));
              wr = ldv(src + base + r);
              y = rfma(-shift, wr, scal2(1.0 / R.gamma, kw));
            } else if (R.mode == MODE_M4) {
              y = make_double2(0.0, 0.0);
              double2 z = make_double2(0.0, 0.0);
              int pi = 0;
              for (int k = 0; k < nt; k++) {
                y = rfma(R.bg[k], a.u[((size_t)k * nv) * D + base + r], y);
                for (int l = k + 1; l < nt; l++, pi++) {
                  const double2 hkul = Op<FAM>::term(cx, k, a.u + ((size_t)l * nv) * D + base, r);
                  const double2 hluk = Op<FAM>::term(cx, l, a.u + ((size_t)k * nv) * D + base, r);
                  z = rfma(R.kg[pi], make_double2(hkul.x - hluk.x, hkul.y - hluk.y), z);
                }
              }
              y.x += z.y;  // -i z
              y.y -= z.x;
              wr = ldv(src + base + r);
              y = rfma(-shift, wr, y);
            } else {
              y = Op<FAM>::combo(cx, R, shift, src + base, r, wr);
            }
            dst[base + r] = y;
            double2 pr = (j == 1) ? cmul(d0, wr) : nxt[base + r];
            pr = cfma(dj, y, pr);
            nxt[base + r] = pr;
            sw = fma(y.x, y.x, fma(y.y, y.y, sw));
            sp = fma(pr.x, pr.x, fma(pr.y, pr.y, sp));
            mw = max(mw, abshi(y));  // kept on every path: a later linear generator scales from them
            mp = max(mp, abshi(pr));
          }
        }
        block_reduce_store(sw, sp, mw, mp);
        if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { bail(MAGNUS_ETIMEOUT); return; }
        if constexpr (STG) {  // a staged copy that did not arrive (its block may have arrived last)
          if (*(volatile int *)&a.bar->error) { bail(MAGNUS_ETIMEOUT); return; }
        }
        zs_src = zs_dst;
        if (warp == 0) {
          int any = 0, bad = 0;
          const double adj = sqrt(cabs2(dj));
          for (int v = 0; v < nv; v++) {
            if (!s_act[v]) continue;  // uniform across the warp
            double tw, tp, mxw, mxp;
            vector_totals(v, tw, tp, &mxw, &mxp);
            if (lane == 0) {
              const double ej = adj * sqrt(tw), pn = sqrt(tp);
              s_wm[v] = mxw;
              if (!isfinite(ej) || !isfinite(pn)) bad = 1;
              if (ej + s_ep[v] <= a.tol_abs + a.tol_rel * pn) {
                s_act[v] = 0;
                s_m[v] = j;
                s_pn[v] = pn;
                s_pm[v] = mxp;
              } else {
                s_ep[v] = ej;
                any = 1;
              }
            }
          }
          if (lane == 0) s_flag = bad ? 2 : (any ? 0 : 1);
        }
        __syncthreads();
        it++;
        if (s_flag == 2) { bail(MAGNUS_ENONFINITE); return; }
        if (s_flag == 1) { done = true; break; }
      }
      if (!done) { bail(MAGNUS_ENOCONV); return; }
      if (tid == 0) {  // a posteriori norm check of the substep (every block decides alike)
        int bad = 0;
        for (int v = 0; v < nv; v++)
          bad |= drift_fails(s_pn[v], s_vn[v], a.tol_abs, a.tol_rel, a.norm_check, a.counters, b == 0) ? 1 : 0;
        s_drift = bad;
      }
      __syncthreads();
      if (s_drift) { bail(MAGNUS_EDRIFT); return; }
      if (tid < nv) {
        s_vn[tid] = s_pn[tid];
        s_vm[tid] = s_pm[tid];
      }
      if (b == 0 && tid == 0) {
        Counters *c = a.counters;
        for (int v = 0; v < nv; v++) {
          const int m = s_m[v];
          c->n_matvec += m;
          c->n_termapply += (long long)m * nt * (R.mode == MODE_M4 ? 2 : (R.mode == MODE_M6 ? 17 : 1));
          if (m > c->max_m) c->max_m = m;
          if (a.mlog && sub_counter * nv + v < a.mlog_cap) a.mlog[sub_counter * nv + v] = m;
        }
        c->n_substeps += nv;
      }
      __syncthreads();
      sub_counter++;
      double2 *tmp = cur; cur = nxt; nxt = tmp;
    }
    if (b == 0 && tid == 0) a.counters->n_exp++;
  }
  if constexpr (STG) stage::drain(P, a.spin_limit_ns);
  if (cur != a.psi)
    for (int64_t r = r_lo + tid; r < r_hi; r += r_step) a.psi[base + r] = cur[base + r];
}

const void *kernel_for(int fam, bool m6, int zf, bool stg = false) {
  if (stg && !m6 && zf == 1 && fam == FAM_CSR) return (const void *)k_magnus_persistent<FAM_CSR, false, 1, true>;
  if (m6) {
    switch (fam) {
      case FAM_CSR: return (const void *)k_magnus_persistent<FAM_CSR, true, 0>;
      case FAM_MF: return (const void *)k_magnus_persistent<FAM_MF, true, 0>;
      default: return (const void *)k_magnus_persistent<FAM_GENERIC, true, 0>;
    }
  }
  if (zf == 1 && fam == FAM_CSR) return (const void *)k_magnus_persistent<FAM_CSR, false, 1>;
  if (zf == 1 && fam == FAM_MF) return (const void *)k_magnus_persistent<FAM_MF, false, 1>;
  if (zf == 2 && fam == FAM_CSR) return (const void *)k_magnus_persistent<FAM_CSR, false, 2>;
  if (zf == 2 && fam == FAM_MF) return (const void *)k_magnus_persistent<FAM_MF, false, 2>;
  switch (fam) {
    case FAM_CSR: return (const void *)k_magnus_persistent<FAM_CSR, false, 0>;
    case FAM_MF: return (const void *)k_magnus_persistent<FAM_MF, false, 0>;
    default: return (const void *)k_magnus_persistent<FAM_GENERIC, false, 0>;
  }
}

}  // namespace

int persistent_block_size() { return kBlock; }

// Resident CTAs per SM of the instantiation for this family (method M6, fixed-point linear
// generators, their staged-rows variant, or the rest): the largest cooperative grid of that launch.
cudaError_t persistent_max_blocks_per_sm(int fam, bool m6, int zf, int *n, bool stg) {
  const void *k = kernel_for(fam, m6, zf, stg);
  const size_t dyn = (stg && !m6 && zf == 1 && fam == FAM_CSR) ? stage::kSmemBytes : 0;
  if (dyn) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k, kBlock, dyn);
}

cudaError_t launch_persistent(const PersistArgs &a, int grid, int block, bool m6, cudaStream_t st) {
  PersistArgs copy = a;
  void *args[] = {&copy};
  const int zf = persistent_fixed_kernel(a, m6);
  const bool stg = a.stg && !m6 && zf == 1 && a.fam == FAM_CSR;
  return cudaLaunchCooperativeKernel(kernel_for(a.fam, m6, zf, stg), dim3(grid), dim3(block), args,
                                     stg ? stage::kSmemBytes : 0, st);
}

size_t persistent_stage_smem_bytes() { return stage::kSmemBytes; }

namespace {
__global__ void k_stage_misfits(const Term *Tg, int nt, int64_t dim, unsigned long long *count) {
  __shared__ Term sT[kMaxTerms];
  for (int i = threadIdx.x; i < nt * (int)sizeof(Term) / 4; i += blockDim.x)
    reinterpret_cast<int *>(sT)[i] = reinterpret_cast<const int *>(Tg)[i];
  __syncthreads();
  const int64_t ntile = (dim + stage::kTile - 1) / stage::kTile;
  unsigned long long mine = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntile; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ra = t * stage::kTile, rb = min(dim, ra + stage::kTile);
    stage::Span S;
    stage::load_span(sT, nt, ra, rb, S);
    stage::Desc L;
    stage::layout(sT, nt, S, L);
    mine += L.fits ? 0 : 1;
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(kFull, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
}
}  // namespace

cudaError_t launch_stage_misfits(const Term *T, int nt, int64_t dim, unsigned long long *count, cudaStream_t st) {
  const int64_t ntile = (dim + stage::kTile - 1) / stage::kTile;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (ntile + 255) / 256));
  k_stage_misfits<<<grid, 256, 0, st>>>(T, nt, dim, count);
  return cudaGetLastError();
}

}  // namespace mg
