// Setup kernels of the Magnus + Leja path (arXiv:1709.06483):
//  * Leja points on [-2,2] and divided differences of exp(-i rho x) (Sec. 3),
//  * per-exponential records: drive values at the Gauss nodes, Magnus weights (Sec. 2,
//    Methods M2, M4, Cf4, Cf4:3), spectral enclosure, shift/scale, substeps,
//  * Gershgorin enclosures of the stored terms (Sec. 3: the spectrum estimate),
//  * Hamiltonian builders for the spin chains of Sec. 4.
// All of it runs once per plan or once per propagation; none of it is in the Leja hot loop.
#include <math.h>

#include "magnus_internal.cuh"

namespace mg {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
  // fixed butterfly order: every lane ends with the same, deterministic value
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// ------------------------------------------------------------------ Leja points
// xi_j = argmax_{x in [-2,2]} prod_{k<j} |x - xi_k|.  With both endpoints already nodes the
// maximiser lies inside one gap between neighbouring nodes, where the log-product is strictly
// concave: its maximiser is the root of sum_k 1/(x - xi_k), bracketed by the gap and found by
// bisection to the last bit.  One block (one warp) per gap; the last block to finish picks the
// gap with the largest log-product, ties (within 1e-10) going to the larger x.
__global__ void k_leja_gap(double *xi, int j, double *cand, unsigned *counter) {
  __shared__ double sorted[kMmaxLimit + 1];
  __shared__ bool last;
  const int lane = threadIdx.x;
  const int g = blockIdx.x;
  // rank sort of xi[0..j-1] (distinct values)
  for (int a = lane; a < j; a += 32) {
    double v = xi[a];
    int r = 0;
    for (int b = 0; b < j; b++) r += (xi[b] < v);
    sorted[r] = v;
  }
  __syncwarp();
  double lo = sorted[g], hi = sorted[g + 1];
  double mid = 0.5 * (lo + hi);
  for (int it = 0; it < 2000; it++) {
    mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double s = 0.0;
    for (int k = lane; k < j; k += 32) s += 1.0 / (mid - xi[k]);
    s = warp_sum(s);
    if (s == 0.0) break;
    if (s > 0.0) lo = mid; else hi = mid;
  }
  double L = 0.0;
  for (int k = lane; k < j; k += 32) L += log(fabs(mid - xi[k]));
  L = warp_sum(L);
  if (lane == 0) {
    cand[2 * g] = mid;
    cand[2 * g + 1] = L;
    __threadfence();
    unsigned done = atomicAdd(counter, 1u);
    last = (done == (unsigned)(j - 2));
  }
  __syncwarp();
  if (last) {
    __threadfence();
    const int ng = j - 1;
    double best = -INFINITY;
    for (int q = lane; q < ng; q += 32) best = fmax(best, ((volatile double *)cand)[2 * q + 1]);
    best = warp_max(best);
    double pick = -INFINITY;
    for (int q = lane; q < ng; q += 32) {
      double x = ((volatile double *)cand)[2 * q], l = ((volatile double *)cand)[2 * q + 1];
      if (l >= best - 1e-10) pick = fmax(pick, x);
    }
    pick = warp_max(pick);
    if (lane == 0) {
      xi[j] = pick;
      *counter = 0u;
    }
  }
}

__global__ void k_leja_init(double *xi, int m, unsigned *counter) {
  xi[0] = 2.0;
  if (m >= 1) xi[1] = -2.0;  // maximiser of |x - 2| on [-2,2]
  *counter = 0u;
}

// --------------------------------------------------------- divided differences
// d_j = g[xi_0..xi_j] for g(x) = exp(-i rho x) is the first column of g(Z), Z the lower
// bidiagonal matrix with xi on the diagonal and ones below (Opitz).  Here the first column is
// propagated directly: d = exp(-i rho Z) e_0 = (exp(-i (rho/q) Z))^q e_0 with q chosen so that
// ||(rho/q) Z||_1 <= 1/2, each factor by its Taylor series acting on the vector.  One warp per
// table; entry j lives in lane j % 32, register j / 32.
static_assert(kMmaxLimit + 1 <= 8 * 32, "divided differences: at most 8 entries per lane");

template <int kDDRegs>
__device__ void warp_divided_differences_r(const double *xi, int m, double rho, double2 phase, double2 *d) {
  // lane l holds entries j = kDDRegs l + r, so that the bidiagonal product needs one value from the
  // neighbouring lane per term; convergence is tested every fourth term (each test is two warp
  // reductions, the latency that bounds this single-warp computation)
  const int lane = threadIdx.x & 31;
  double2 y[kDDRegs];
  double x[kDDRegs];
#pragma unroll
  for (int r = 0; r < kDDRegs; r++) {
    const int j = kDDRegs * lane + r;
    x[r] = (j <= m) ? xi[j] : 0.0;
    y[r] = make_double2((j == 0) ? 1.0 : 0.0, 0.0);
  }
  const double znorm = 3.0;  // ||Z||_1 <= max|xi| + 1
  int q = (int)ceil(rho * znorm / 0.5);
  if (q < 1) q = 1;
  const double t = rho / q;
  for (int piece = 0; piece < q; piece++) {
    double2 term[kDDRegs], sum[kDDRegs];
#pragma unroll
    for (int r = 0; r < kDDRegs; r++) { term[r] = y[r]; sum[r] = y[r]; }
    for (int k = 1; k <= 40; k++) {
      // term <- (-i t / k) Z term ;  (Z v)_j = xi_j v_j + v_{j-1}
      const double px = __shfl_up_sync(kFull, term[kDDRegs - 1].x, 1);
      const double py = __shfl_up_sync(kFull, term[kDDRegs - 1].y, 1);
      const double f = t / k;
#pragma unroll
      for (int r = kDDRegs - 1; r >= 0; r--) {  // high to low: term[r - 1] is still the old value
        const int j = kDDRegs * lane + r;
        const double bx = r > 0 ? term[r > 0 ? r - 1 : 0].x : (lane > 0 ? px : 0.0);
        const double by = r > 0 ? term[r > 0 ? r - 1 : 0].y : (lane > 0 ? py : 0.0);
        const double zx = fma(x[r], term[r].x, bx);
        const double zy = fma(x[r], term[r].y, by);
        // (-i f) (zx + i zy) = f zy - i f zx
        term[r] = (j <= m) ? make_double2(f * zy, -f * zx) : make_double2(0.0, 0.0);
        sum[r].x += term[r].x;
        sum[r].y += term[r].y;
      }
      if ((k & 3) == 0) {
        double tmax = 0.0, smax = 0.0;
#pragma unroll
        for (int r = 0; r < kDDRegs; r++) {
          tmax = fmax(tmax, fabs(term[r].x) + fabs(term[r].y));
          smax = fmax(smax, fabs(sum[r].x) + fabs(sum[r].y));
        }
        tmax = warp_max(tmax);
        smax = warp_max(smax);
        if (tmax <= 1e-18 * smax) break;
      }
    }
#pragma unroll
    for (int r = 0; r < kDDRegs; r++) y[r] = sum[r];
  }
#pragma unroll
  for (int r = 0; r < kDDRegs; r++) {
    const int j = kDDRegs * lane + r;
    if (j <= m) d[j] = cmul(phase, y[r]);
  }
}

// entries per lane: 4 (m <= 127, the default m_max = 100) or 8 (m <= 255); every entry a lane holds
// costs FP64 instructions whether or not it is used
__device__ void warp_divided_differences(const double *xi, int m, double rho, double2 phase, double2 *d) {
  if (m < 128)
    warp_divided_differences_r<4>(xi, m, rho, phase, d);
  else
    warp_divided_differences_r<8>(xi, m, rho, phase, d);
}

__global__ void k_divided_differences(const double *xi, int m, double rho, double2 *d) {
  warp_divided_differences(xi, m, rho, make_double2(1.0, 0.0), d);
}

// ------------------------------------------------------ per-exponential records
__device__ double coeff_eval(const Coeff &c, double t) {
  double f = c.a0;
  for (int q = 0; q < c.nmodes; q++) f += c.ac[q] * cos(c.om[q] * t) + c.as[q] * sin(c.om[q] * t);
  return f;
}

// Spectral enclosure of sum_k lin_k H_k (Minkowski sum of the scaled Gershgorin intervals,
// Weyl), widened by +-r for the M4 commutator.
__device__ void finish_record(ExpRec &R, const double *lin, int nterms, const double *term_ab, double r, double rho_max) {
  double lo = 0.0, hi = 0.0;
  for (int k = 0; k < nterms; k++) {
    double x1 = lin[k] * term_ab[2 * k], x2 = lin[k] * term_ab[2 * k + 1];
    lo += fmin(x1, x2);
    hi += fmax(x1, x2);
  }
  lo -= r;
  hi += r;
  R.a = lo;
  R.b = hi;
  R.c = 0.5 * (lo + hi);
  R.gamma = 0.25 * (hi - lo);
  int s = 1;
  if (R.gamma > 0.0) {
    s = (int)ceil(R.gamma / rho_max);
    if (s < 1) s = 1;
    for (int k = 0; k < kMaxTerms; k++) R.bg[k] = (k < nterms) ? lin[k] / R.gamma : 0.0;
    R.cg = R.c / R.gamma;
  } else {
    for (int k = 0; k < kMaxTerms; k++) R.bg[k] = 0.0;
    R.cg = 0.0;
  }
  R.s = s;
}

// One warp per exponential, in application order.  e -> (step n, stage).
//  M2:    stage 0: beta_k = h f_k(t_n + h/2).
//  M4:    lambda_k = h/2 (f_k(t1) + f_k(t2)),  kappa = sqrt(3) h^2 / 12,
//         coef_kl = f_k(t2) f_l(t1) - f_l(t2) f_k(t1)  ([H_2,H_1] = sum_{k<l} coef_kl [H_k,H_l]).
//  Cf4:   stage 0 (applied first): h (a2 f(t1) + a1 f(t2)), stage 1: h (a1 f(t1) + a2 f(t2)).
//  Cf4:3: stage 0 uses the third row of the alpha table, stage 2 the first.
//  M6:    one exponential; P, Q, R of the three Gauss nodes (see the branch below).
__device__ void exp_setup_warp(long long e, int variant, double t0, double h, int nterms, const Coeff *coeffs,
                               const double *term_ab, const double *xi, int m_max, double rho_max, ExpRec *recs,
                               double2 *dd, int per_step) {
  const int lane = threadIdx.x & 31;
  const long long n = e / per_step;
  const int stage = (int)(e % per_step);
  const double tn = t0 + (double)n * h;
  const double r3 = sqrt(3.0), r15 = sqrt(15.0);
  ExpRec R;
  for (int k = 0; k < kMaxPairs; k++) R.kg[k] = 0.0;
  for (int k = 0; k < kMaxTerms; k++) R.p6[k] = R.q6[k] = R.r6[k] = 0.0;
  double lin[kMaxTerms] = {0.0, 0.0, 0.0, 0.0};
  double r = 0.0;
  R.mode = MODE_LINEAR;
  if (variant == MAGNUS_M6) {
    // Method M6 with A_i = -i H(t_n + c_i h): B_1 = -iP, B_2 = -iQ, B_3 = -iR,
    //   P = h H(t2), Q = (sqrt(15)/3) h (H(t3) - H(t1)), R = (10/3) h (H(t3) - 2 H(t2) + H(t1)),
    // K = i Omega = P + R/12 + (i/240)[U, V]; the linear part P + R/12 gives the enclosure and
    // the commutator adds +-r (bound from the half-widths, S = 20 P + R, C = [P, Q]):
    //   r = (|[S,Q]| + 2 |S| |E| + 2 |C| (|Q| + |E|)) / 240,  |E| = (|[P,R]| + |P| |C|) / 30.
    R.mode = MODE_M6;
    const double c6[3] = {0.5 - r15 / 10.0, 0.5, 0.5 + r15 / 10.0};
    double hw[kMaxTerms], sk[kMaxTerms];
    for (int k = 0; k < nterms; k++) {
      const double f1 = coeff_eval(coeffs[k], tn + c6[0] * h);
      const double f2 = coeff_eval(coeffs[k], tn + c6[1] * h);
      const double f3 = coeff_eval(coeffs[k], tn + c6[2] * h);
      R.p6[k] = h * f2;
      R.q6[k] = r15 / 3.0 * h * (f3 - f1);
      R.r6[k] = 10.0 / 3.0 * h * (f3 - 2.0 * f2 + f1);
      lin[k] = R.p6[k] + R.r6[k] / 12.0;
      sk[k] = 20.0 * R.p6[k] + R.r6[k];
      hw[k] = 0.5 * (term_ab[2 * k + 1] - term_ab[2 * k]);
    }
    double pq = 0.0, pr = 0.0, sq = 0.0, pn = 0.0, sn = 0.0, qn = 0.0;
    for (int k = 0; k < nterms; k++) {
      pn += fabs(R.p6[k]) * hw[k];
      sn += fabs(sk[k]) * hw[k];
      qn += fabs(R.q6[k]) * hw[k];
      for (int l = k + 1; l < nterms; l++) {
        const double w2 = 2.0 * hw[k] * hw[l];
        pq += fabs(R.p6[k] * R.q6[l] - R.p6[l] * R.q6[k]) * w2;
        pr += fabs(R.p6[k] * R.r6[l] - R.p6[l] * R.r6[k]) * w2;
        sq += fabs(sk[k] * R.q6[l] - sk[l] * R.q6[k]) * w2;
      }
    }
    const double en = (pr + pn * pq) / 30.0;
    r = (sq + 2.0 * sn * en + 2.0 * pq * (qn + en)) / 240.0;
  } else if (variant == MAGNUS_M2) {
    for (int k = 0; k < nterms; k++) lin[k] = h * coeff_eval(coeffs[k], tn + 0.5 * h);
  } else if (variant == MAGNUS_CF4) {
    const double c1 = 0.5 - r3 / 6.0, c2 = 0.5 + r3 / 6.0;
    const double a1 = (3.0 - 2.0 * r3) / 12.0, a2 = (3.0 + 2.0 * r3) / 12.0;
    const double w1 = (stage == 0) ? a2 : a1, w2 = (stage == 0) ? a1 : a2;
    for (int k = 0; k < nterms; k++)
      lin[k] = h * (w1 * coeff_eval(coeffs[k], tn + c1 * h) + w2 * coeff_eval(coeffs[k], tn + c2 * h));
  } else if (variant == MAGNUS_CF4_3) {
    const double c[3] = {0.5 - r15 / 10.0, 0.5, 0.5 + r15 / 10.0};
    const double al[3][3] = {{37.0 / 240.0 - 10.0 * r15 / 261.0, -1.0 / 30.0, 37.0 / 240.0 + 10.0 * r15 / 261.0},
                             {-11.0 / 360.0, 23.0 / 45.0, -11.0 / 360.0},
                             {37.0 / 240.0 + 10.0 * r15 / 261.0, -1.0 / 30.0, 37.0 / 240.0 - 10.0 * r15 / 261.0}};
    const int row = 2 - stage;
    for (int k = 0; k < nterms; k++) {
      double s = 0.0;
      for (int q = 0; q < 3; q++) s += al[row][q] * coeff_eval(coeffs[k], tn + c[q] * h);
      lin[k] = h * s;
    }
  } else {  // MAGNUS_M4
    R.mode = MODE_M4;
    const double c1 = 0.5 - r3 / 6.0, c2 = 0.5 + r3 / 6.0;
    double f1[kMaxTerms], f2[kMaxTerms];
    for (int k = 0; k < nterms; k++) {
      f1[k] = coeff_eval(coeffs[k], tn + c1 * h);
      f2[k] = coeff_eval(coeffs[k], tn + c2 * h);
      lin[k] = 0.5 * h * (f1[k] + f2[k]);
    }
    const double kappa = r3 * h * h / 12.0;
    int pi = 0;
    for (int k = 0; k < nterms; k++)
      for (int l = k + 1; l < nterms; l++, pi++) {
        double coef = f2[k] * f1[l] - f2[l] * f1[k];
        double hwk = 0.5 * (term_ab[2 * k + 1] - term_ab[2 * k]);
        double hwl = 0.5 * (term_ab[2 * l + 1] - term_ab[2 * l]);
        r += fabs(coef) * 2.0 * hwk * hwl;
        R.kg[pi] = kappa * coef;  // divided by gamma below
      }
    r *= kappa;
  }
  finish_record(R, lin, nterms, term_ab, r, rho_max);
  if (R.gamma > 0.0)
    for (int p = 0; p < kMaxPairs; p++) R.kg[p] /= R.gamma;
  double2 *d = dd + e * (long long)(m_max + 1);
  if (R.gamma > 0.0) {
    // each substep's polynomial carries the phase e^{-i c / s}
    double ph = -R.c / R.s;
    warp_divided_differences(xi, m_max, R.gamma / R.s, make_double2(cos(ph), sin(ph)), d);
  } else {
    // K is enclosed by the scalar c: exp(-iK) = e^{-ic}; stored as d_0, no iteration
    if (lane == 0) d[0] = make_double2(cos(-R.c), sin(-R.c));
    for (int j = 1 + lane; j <= m_max; j += 32) d[j] = make_double2(0.0, 0.0);
  }
  if (lane == 0) recs[e] = R;
}

// one warp per exponential
__global__ void k_exp_setup(int variant, double t0, double h, int nterms, const Coeff *coeffs, const double *term_ab,
                            const double *xi, int m_max, double rho_max, ExpRec *recs, double2 *dd, long long nexp,
                            int per_step) {
  const long long e = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x / 32);
  if (e >= nexp) return;  // whole warp exits together
  exp_setup_warp(e, variant, t0, h, nterms, coeffs, term_ab, xi, m_max, rho_max, recs, dd, per_step);
}

// one warp per (problem, exponential) of a batch: problem i has nterms[i] terms, coefficients at
// coeffs + i kMaxTerms, enclosures at term_ab + 2 i kMaxTerms, records at recs + i rec_stride and
// tables at dd + i rec_stride (m_max + 1)
__global__ void k_exp_setup_batch(int variant, double t0, double h, int count, const int *nterms, const Coeff *coeffs,
                                  const double *term_ab, const double *xi, int m_max, double rho_max, ExpRec *recs,
                                  double2 *dd, long long nexp, long long rec_stride, int per_step) {
  const long long g = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x / 32);
  if (g >= (long long)count * nexp) return;
  const long long i = g / nexp, e = g % nexp;
  exp_setup_warp(e, variant, t0, h, nterms[i], coeffs + i * kMaxTerms, term_ab + i * 2 * kMaxTerms, xi, m_max,
                 rho_max, recs + i * rec_stride, dd + i * rec_stride * (m_max + 1), per_step);
}

struct BetaArg {
  double b[kMaxTerms];
};

__global__ void k_exp_setup_beta(BetaArg beta, int nterms, const double *term_ab, const double *xi,
                                 int m_max, double rho_max, ExpRec *recs, double2 *dd) {
  const int lane = threadIdx.x & 31;
  ExpRec R;
  for (int k = 0; k < kMaxPairs; k++) R.kg[k] = 0.0;
  double lin[kMaxTerms] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < nterms; k++) lin[k] = beta.b[k];
  R.mode = MODE_LINEAR;
  finish_record(R, lin, nterms, term_ab, 0.0, rho_max);
  if (R.gamma > 0.0) {
    double ph = -R.c / R.s;
    warp_divided_differences(xi, m_max, R.gamma / R.s, make_double2(cos(ph), sin(ph)), dd);
  } else {
    if (lane == 0) dd[0] = make_double2(cos(-R.c), sin(-R.c));
    for (int j = 1 + lane; j <= m_max; j += 32) dd[j] = make_double2(0.0, 0.0);
  }
  if (lane == 0) recs[0] = R;
}

// --------------------------------------------------------------- Gershgorin
// spec(H) within [min_i (Re H_ii - R_i), max_i (Re H_ii + R_i)], R_i = sum_{j != i} |H_ij|.
__device__ __forceinline__ double cabs_(double2 v) { return hypot(v.x, v.y); }
// entry e of a CSR / dense term in either storage
__device__ __forceinline__ double2 term_val(const Term &t, int64_t e) {
  return t.rs == 1 ? make_double2(t.rv[e], 0.0) : t.val[e];
}

__device__ void row_center_radius(const Term &t, int64_t dim, int64_t i, double &c, double &R) {
  c = 0.0;
  R = 0.0;
  if (t.kind == MAGNUS_TERM_CSR) {
    for (int64_t e = t.rowptr[i]; e < t.rowptr[i + 1]; e++) {
      double2 v = term_val(t, e);
      if (t.col[e] == i) c += v.x; else R += t.real_valued ? fabs(v.x) : cabs_(v);
    }
  } else if (t.kind == MAGNUS_TERM_XXZ) {
    const int n = t.nspins;
    for (int s = 1; s <= n; s++) {
      double zs = ((i >> (n - s)) & 1) ? -1.0 : 1.0;
      c += t.hz[s - 1] * zs;
      if (s < n) {
        double zn = ((i >> (n - s - 1)) & 1) ? -1.0 : 1.0;
        c += t.delta * t.J[s - 1] * zs * zn;
        if (zs != zn) R += fabs(2.0 * t.J[s - 1]);
      }
    }
  } else if (t.kind == MAGNUS_TERM_FIELD_X) {
    R = (double)t.nspins;
  }
}

__global__ void k_gershgorin_rows(const Term *tp, int64_t dim, double *part) {
  const Term &t = *tp;
  double lo = INFINITY, hi = -INFINITY;
  if (t.kind == MAGNUS_TERM_DENSE) {
    // one warp per row
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < dim; i += nwarps) {
      double c = 0.0, R = 0.0;
      for (int64_t j = lane; j < dim; j += 32) {
        double2 v = term_val(t, i * dim + j);
        if (j == i) c += v.x; else R += t.real_valued ? fabs(v.x) : cabs_(v);
      }
      c = warp_sum(c);
      R = warp_sum(R);
      lo = fmin(lo, c - R);
      hi = fmax(hi, c + R);
    }
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
      double c, R;
      row_center_radius(t, dim, i, c, R);
      lo = fmin(lo, c - R);
      hi = fmax(hi, c + R);
    }
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  __shared__ double slo[32], shi[32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { slo[w] = lo; shi[w] = hi; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    lo = (lane < nw) ? slo[lane] : INFINITY;
    hi = (lane < nw) ? shi[lane] : -INFINITY;
    lo = warp_min(lo);
    hi = warp_max(hi);
    if (lane == 0) { part[2 * blockIdx.x] = lo; part[2 * blockIdx.x + 1] = hi; }
  }
}

__global__ void k_gershgorin_final(const double *part, int nblk, double *out) {
  const int lane = threadIdx.x;
  double lo = INFINITY, hi = -INFINITY;
  for (int b = lane; b < nblk; b += 32) { lo = fmin(lo, part[2 * b]); hi = fmax(hi, part[2 * b + 1]); }
  lo = warp_min(lo);
  hi = warp_max(hi);
  if (lane == 0) { out[0] = lo; out[1] = hi; }
}

__global__ void k_imag_check(const double2 *val, int64_t n, int *flag) {
  bool any = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    any |= (val[i].y != 0.0);
  if (__any_sync(kFull, any) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// Pattern check of a real-valued CSR term: flag |= 1 if some stored value differs from the first
// (or is NaN), |= 2 if some row's length differs from the first row's or rowptr[0] != 0 (rows of
// one length then start at r * length); rowmax = longest row.
__global__ void k_pattern_check(const int64_t *rowptr, const double *rv, int rs, int64_t dim, int *flag,
                                unsigned long long *rowmax) {
  const double v0 = rv[0];
  const int64_t len0 = rowptr[1] - rowptr[0];
  bool differs = false, ragged = rowptr[0] != 0;
  unsigned long long lmax = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = rowptr[i], e1 = rowptr[i + 1];
    lmax = max(lmax, (unsigned long long)(e1 - e0));
    ragged |= (e1 - e0) != len0;
    for (int64_t e = e0; e < e1; e++) differs |= !(rv[e * rs] == v0);
  }
  if (__any_sync(kFull, differs) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
  if (__any_sync(kFull, ragged) && (threadIdx.x & 31) == 0) atomicOr(flag, 2);
  atomicMax(rowmax, lmax);
}

// one thread per row: the row's exponent, then its entries as 62-bit signed mantissas at that scale
__global__ void k_fixed_values(const int64_t *rowptr, const double *rv, int rs, int64_t dim, long long *fval,
                               int16_t *fexp, int *wide) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = rowptr[i], e1 = rowptr[i + 1];
    double amax = 0.0;
    for (int64_t e = e0; e < e1; e++) amax = fmax(amax, fabs(rv[e * rs]));
    int E = 0;
    if (amax > 0.0) {
      frexp(amax, &E);  // amax = f 2^E, f in [0.5, 1): amax < 2^E
    }
    if (E > 400 || E < -400 || !(amax <= 1.7e308)) atomicOr(wide, 1);  // outside the range the scales cover
    fexp[i] = (int16_t)max(-400, min(400, E));
    for (int64_t e = e0; e < e1; e++) fval[e] = llrint(ldexp(rv[e * rs], 62 - E));
  }
}

__global__ void k_real_parts(const double2 *z, int64_t n, double *out, int *flag) {
  bool any = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = z[i];
    out[i] = v.x;
    any |= (v.y != 0.0);
  }
  if (__any_sync(kFull, any) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// ------------------------------------------------------------------ builders
// Kronecker convention of Sec. 4: spin s (1-based) of n is bit (n - s); z_s = 1 - 2 b_s.
// sx_i sx_j + sy_i sy_j maps |x> to (1 - z_i z_j)|x ^ bit_i ^ bit_j>.
struct BuildParams {
  double J[kMaxSpins];
  double hz[kMaxSpins];
};

// Number of x' < x whose bits p and p-1 differ (anti-parallel neighbours at those bits): per
// period 2^(p+1) they differ exactly on [2^(p-1), 3*2^(p-1)).
__device__ __forceinline__ int64_t antiparallel_below(int64_t x, int p) {
  int64_t period = (int64_t)1 << (p + 1), half = (int64_t)1 << p, q = (int64_t)1 << (p - 1);
  int64_t full = (x >> (p + 1)) * half;
  int64_t rem = (x & (period - 1)) - q;
  rem = rem < 0 ? 0 : (rem > half ? half : rem);
  return full + rem;
}

__global__ void k_build_xxz_csr(int n, BuildParams P, double delta, int64_t *rowptr, int32_t *col, double2 *val) {
  const int64_t D = (int64_t)1 << n;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= D; x += (int64_t)gridDim.x * blockDim.x) {
    int64_t start = x;
    for (int s = 1; s < n; s++) start += antiparallel_below(x, n - s);
    rowptr[x] = start;
    if (x == D) continue;
    int64_t cc[kMaxSpins + 1];
    double cv[kMaxSpins + 1];
    int cnt = 0;
    double diag = 0.0;
    for (int s = 1; s <= n; s++) {
      double zs = ((x >> (n - s)) & 1) ? -1.0 : 1.0;
      diag += P.hz[s - 1] * zs;
      if (s < n) {
        double zn = ((x >> (n - s - 1)) & 1) ? -1.0 : 1.0;
        diag += delta * P.J[s - 1] * zs * zn;
        if (zs != zn) {
          cc[cnt] = x ^ ((int64_t)3 << (n - s - 1));
          cv[cnt] = 2.0 * P.J[s - 1];
          cnt++;
        }
      }
    }
    cc[cnt] = x;
    cv[cnt] = diag;
    cnt++;
    for (int a = 1; a < cnt; a++) {  // ascending columns
      int64_t c = cc[a];
      double v = cv[a];
      int b = a - 1;
      while (b >= 0 && cc[b] > c) { cc[b + 1] = cc[b]; cv[b + 1] = cv[b]; b--; }
      cc[b + 1] = c;
      cv[b + 1] = v;
    }
    for (int a = 0; a < cnt; a++) {
      col[start + a] = (int32_t)cc[a];
      val[start + a] = make_double2(cv[a], 0.0);
    }
  }
}

__global__ void k_build_field_x_csr(int n, int64_t *rowptr, int32_t *col, double2 *val) {
  const int64_t D = (int64_t)1 << n;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= D; x += (int64_t)gridDim.x * blockDim.x) {
    rowptr[x] = x * n;
    if (x == D) continue;
    // columns x ^ 2^b in ascending order: bits set in x lower the column, so they come first
    // from the highest such bit down, then the clear bits from the lowest up
    int a = 0;
    for (int b = n - 1; b >= 0; b--)
      if ((x >> b) & 1) { col[x * n + a] = (int32_t)(x ^ ((int64_t)1 << b)); val[x * n + a] = make_double2(1.0, 0.0); a++; }
    for (int b = 0; b < n; b++)
      if (!((x >> b) & 1)) { col[x * n + a] = (int32_t)(x ^ ((int64_t)1 << b)); val[x * n + a] = make_double2(1.0, 0.0); a++; }
  }
}

__global__ void k_build_longrange_dense(int n, double alpha, BuildParams P, double delta, double2 *H) {
  const int64_t D = (int64_t)1 << n;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < D; x += (int64_t)gridDim.x * blockDim.x) {
    double diag = 0.0;
    for (int i = 1; i <= n; i++) diag += P.hz[i - 1] * (((x >> (n - i)) & 1) ? -1.0 : 1.0);
    for (int i = 1; i <= n; i++)
      for (int j = i + 1; j <= n; j++) {
        double Jij = 1.0 / pow((double)(j - i), alpha);
        double zi = ((x >> (n - i)) & 1) ? -1.0 : 1.0, zj = ((x >> (n - j)) & 1) ? -1.0 : 1.0;
        diag += delta * Jij * zi * zj;
        if (zi != zj) {
          int64_t y = x ^ ((int64_t)1 << (n - i)) ^ ((int64_t)1 << (n - j));
          H[x * D + y] = make_double2(2.0 * Jij, 0.0);
        }
      }
    H[x * D + x] = make_double2(diag, 0.0);
  }
}

__global__ void k_build_field_x_dense(int n, double2 *H) {
  const int64_t D = (int64_t)1 << n;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < D; x += (int64_t)gridDim.x * blockDim.x)
    for (int b = 0; b < n; b++) H[x * D + (x ^ ((int64_t)1 << b))] = make_double2(1.0, 0.0);
}

// Diagonal of the open XXZ chain split at bit L: diag(x) = dhi[x >> L] + dlo[x & (2^(L+1) - 1)].
// Bit p holds spin n-p; the bond between bits p and p-1 has coupling J[n-p-1].  dlo holds the fields
// at bits 0..L-1 and the bonds (p, p-1) for p = 1..L; dhi the fields at bits L..n-1 and the bonds
// for p = L+1..n-1, so that every term of the diagonal is counted exactly once.
__global__ void k_xxz_diag_tables(const Term *tp, int n, int L, double *dlo, double *dhi) {
  const Term &t = *tp;
  const int64_t nlo = (int64_t)1 << (L + 1), nhi = (int64_t)1 << (n - L);
  const int64_t total = nlo > nhi ? nlo : nhi;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nlo) {
      double s = 0.0;
      for (int p = 0; p < L; p++) s += t.hz[n - p - 1] * (((i >> p) & 1) ? -1.0 : 1.0);
      for (int p = 1; p <= L; p++)
        s += t.delta * t.J[n - p - 1] * ((((i >> p) ^ (i >> (p - 1))) & 1) ? -1.0 : 1.0);
      dlo[i] = s;
    }
    if (i < nhi) {
      const int64_t x = i << L;
      double s = 0.0;
      for (int p = L; p < n; p++) s += t.hz[n - p - 1] * (((x >> p) & 1) ? -1.0 : 1.0);
      for (int p = L + 1; p < n; p++)
        s += t.delta * t.J[n - p - 1] * ((((x >> p) ^ (x >> (p - 1))) & 1) ? -1.0 : 1.0);
      dhi[i] = s;
    }
  }
}

int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

int exps_per_step(int variant) {
  switch (variant) {
    case MAGNUS_CF4: return 2;
    case MAGNUS_CF4_3: return 3;
    case MAGNUS_M4: return 1;
    case MAGNUS_M2: return 1;
    case MAGNUS_M6: return 1;
    default: return 0;
  }
}

cudaError_t launch_leja_points(double *xi, int m, double *cand, unsigned *counter, cudaStream_t st) {
  k_leja_init<<<1, 1, 0, st>>>(xi, m, counter);
  for (int j = 2; j <= m; j++) k_leja_gap<<<j - 1, 32, 0, st>>>(xi, j, cand, counter);
  return cudaGetLastError();
}

cudaError_t launch_divided_differences(const double *xi, int m, double rho, double2 *d, cudaStream_t st) {
  k_divided_differences<<<1, 32, 0, st>>>(xi, m, rho, d);
  return cudaGetLastError();
}

cudaError_t launch_gershgorin(const Term *t_dev, const Term &t_host, int64_t dim, double *scratch, int nblk,
                              double *out, cudaStream_t st) {
  (void)t_host;
  k_gershgorin_rows<<<nblk, 256, 0, st>>>(t_dev, dim, scratch);
  k_gershgorin_final<<<1, 32, 0, st>>>(scratch, nblk, out);
  return cudaGetLastError();
}

cudaError_t launch_imag_check(const double2 *val, int64_t n, int *flag, cudaStream_t st) {
  k_imag_check<<<grid_for(n, 256), 256, 0, st>>>(val, n, flag);
  return cudaGetLastError();
}

cudaError_t launch_pattern_check(const int64_t *rowptr, const double *rv, int rs, int64_t dim, int *flag,
                                 unsigned long long *rowmax, cudaStream_t st) {
  k_pattern_check<<<grid_for(dim, 256), 256, 0, st>>>(rowptr, rv, rs, dim, flag, rowmax);
  return cudaGetLastError();
}

cudaError_t launch_fixed_values(const int64_t *rowptr, const double *rv, int rs, int64_t dim, long long *fval,
                                int16_t *fexp, int *wide, cudaStream_t st) {
  k_fixed_values<<<grid_for(dim, 256), 256, 0, st>>>(rowptr, rv, rs, dim, fval, fexp, wide);
  return cudaGetLastError();
}

cudaError_t launch_real_parts(const double2 *z, int64_t n, double *out, int *flag, cudaStream_t st) {
  k_real_parts<<<grid_for(n, 256), 256, 0, st>>>(z, n, out, flag);
  return cudaGetLastError();
}

cudaError_t launch_exp_setup(int variant, double t0, double h, int64_t nsteps, int nterms, const Coeff *coeffs,
                             const double *term_ab, const double *xi, int m_max, double rho_max, ExpRec *recs,
                             double2 *dd, int64_t nexp, cudaStream_t st) {
  const int warps = 4;
  int64_t blocks = (nexp + warps - 1) / warps;
  k_exp_setup<<<(unsigned)blocks, 32 * warps, 0, st>>>(variant, t0, h, nterms, coeffs, term_ab, xi, m_max, rho_max,
                                                        recs, dd, nexp, exps_per_step(variant));
  return cudaGetLastError();
}

cudaError_t launch_exp_setup_batch(int variant, double t0, double h, int64_t nsteps, int count, const int *nterms_dev,
                                   const Coeff *coeffs, const double *term_ab, const double *xi, int m_max,
                                   double rho_max, ExpRec *recs, double2 *dd, int64_t rec_stride, cudaStream_t st) {
  const int64_t nexp = nsteps * exps_per_step(variant);
  const int warps = 4;
  const int64_t blocks = ((int64_t)count * nexp + warps - 1) / warps;
  if (blocks == 0) return cudaSuccess;
  k_exp_setup_batch<<<(unsigned)blocks, 32 * warps, 0, st>>>(variant, t0, h, count, nterms_dev, coeffs, term_ab, xi,
                                                              m_max, rho_max, recs, dd, nexp, rec_stride,
                                                              exps_per_step(variant));
  return cudaGetLastError();
}

cudaError_t launch_exp_setup_beta(const double *beta_host, int nterms, const double *term_ab, const double *xi,
                                  int m_max, double rho_max, ExpRec *recs, double2 *dd, cudaStream_t st) {
  BetaArg b{};
  for (int k = 0; k < nterms && k < kMaxTerms; k++) b.b[k] = beta_host[k];
  k_exp_setup_beta<<<1, 32, 0, st>>>(b, nterms, term_ab, xi, m_max, rho_max, recs, dd);
  return cudaGetLastError();
}

cudaError_t launch_xxz_diag_tables(const Term *t_dev, int nspins, int lbits, double *dlo, double *dhi,
                                   cudaStream_t st) {
  int64_t n = (int64_t)1 << (lbits + 1 > nspins - lbits ? lbits + 1 : nspins - lbits);
  k_xxz_diag_tables<<<grid_for(n, 256), 256, 0, st>>>(t_dev, nspins, lbits, dlo, dhi);
  return cudaGetLastError();
}

cudaError_t launch_build_xxz_csr(int nspins, const double *J, const double *hz, double delta, int64_t *rowptr,
                                 int32_t *col, double2 *val, cudaStream_t st) {
  BuildParams P{};
  for (int i = 0; i < nspins - 1; i++) P.J[i] = J[i];
  for (int i = 0; i < nspins; i++) P.hz[i] = hz[i];
  int64_t D = (int64_t)1 << nspins;
  k_build_xxz_csr<<<grid_for(D + 1, 256), 256, 0, st>>>(nspins, P, delta, rowptr, col, val);
  return cudaGetLastError();
}

cudaError_t launch_build_field_x_csr(int nspins, int64_t *rowptr, int32_t *col, double2 *val, cudaStream_t st) {
  int64_t D = (int64_t)1 << nspins;
  k_build_field_x_csr<<<grid_for(D + 1, 256), 256, 0, st>>>(nspins, rowptr, col, val);
  return cudaGetLastError();
}

cudaError_t launch_build_longrange_dense(int nspins, double alpha, const double *hz, double delta, double2 *H,
                                         cudaStream_t st) {
  BuildParams P{};
  for (int i = 0; i < nspins; i++) P.hz[i] = hz[i];
  int64_t D = (int64_t)1 << nspins;
  cudaError_t e = cudaMemsetAsync(H, 0, sizeof(double2) * (size_t)D * (size_t)D, st);
  if (e != cudaSuccess) return e;
  k_build_longrange_dense<<<grid_for(D, 128), 128, 0, st>>>(nspins, alpha, P, delta, H);
  return cudaGetLastError();
}

cudaError_t launch_build_field_x_dense(int nspins, double2 *H, cudaStream_t st) {
  int64_t D = (int64_t)1 << nspins;
  cudaError_t e = cudaMemsetAsync(H, 0, sizeof(double2) * (size_t)D * (size_t)D, st);
  if (e != cudaSuccess) return e;
  k_build_field_x_dense<<<grid_for(D, 128), 128, 0, st>>>(nspins, H);
  return cudaGetLastError();
}

}  // namespace mg
