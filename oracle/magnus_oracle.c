/*
 * magnus_oracle.c -- TEST INFRASTRUCTURE, not the product.
 *
 * A plain, slow, obviously-correct FP64 CPU restatement of the method of
 * Auer, Einkemmer, Kandolf, Ostermann, "Magnus integrators on multicore CPUs and
 * GPUs" (arXiv:1709.06483).  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load it; the CUDA library never does, and the
 * two share no code.  Every function cites the passage of the paper it follows.
 *
 * Notation.  The paper writes i psi' = H(t) psi (Sec. 1, Eq. (1)) and
 * Y' = A(t) Y (Sec. 2, Eq. (2)), so A = -iH.  A stored problem is
 * H(t) = sum_k f_k(t) H_k (the split H_1 + h(t) H_2 of Sec. 4).  One exponential
 * is written exp(-iK) with a Hermitian generator K that already contains the
 * step size.
 *
 * Readings of the paper (where it is silent or defers to its ref. [ckor15]):
 *  - Leja points on [-2,2], xi_0 = 2, each next point maximises prod |x - xi_k|;
 *    ties go to the larger x.
 *  - K is shifted and scaled, X = (K - cI)/gamma with [c-2gamma, c+2gamma] the
 *    spectral enclosure, and exp(-iK) = e^{-ic} exp(-i gamma X) is split into
 *    s = ceil(gamma/rho_max) equal substeps.
 *  - Early termination: stop at the first j with
 *    |d_j|*||w_j|| + |d_{j-1}|*||w_{j-1}|| <= tol_abs + tol_rel*||p_j|| (2-norms).
 *  - The spectral enclosure of each stored term is its Gershgorin interval; the
 *    enclosure of a combination sum_k beta_k H_k is the Minkowski sum of the
 *    scaled intervals (Weyl); the M4 commutator adds [-r, r] with
 *    r = kappa * sum_{k<l} |coef_kl| * 2 * hw_k * hw_l (hw = half-width).
 *  - Method M6: the coefficient of B_3 is 1/12 (the printed 1/2 would break
 *    the exactness of the first Magnus term for quadratic A; with 1/12,
 *    B_1 + B_3/12 is the 3-point Gauss rule h(5 A_1 + 8 A_2 + 5 A_3)/18).
 *    Its nested commutators add [-r, r], r a bound of |(i/240)[U, V]| from the
 *    half-widths of the terms' enclosures (see gen_interval).
 *
 * Threads.  Built without OpenMP (the checker) every loop runs in order on one
 * thread.  The `#pragma omp parallel for` lines mark only the row loop of a term
 * product and element-wise vector updates; a separate -fopenmp build, used only
 * to time the CPU baseline on all host cores, spreads those loops over threads.
 * Each entry is still computed by one thread with the same operations in the
 * same order, and every reduction (norms, inner products) stays serial, so both
 * builds give identical bits.
 */
#include "magnus_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAX_TERMS 8

/* ------------------------------------------------------------------------- */
/* Leja points (Sec. 3: interpolation nodes xi_0..xi_m, "Leja points").       */
/* ------------------------------------------------------------------------- */

/* log prod_k |x - xi_k| */
static double leja_logprod(double x, const double *xi, int n) {
  double s = 0.0;
  for (int k = 0; k < n; k++) s += log(fabs(x - xi[k]));
  return s;
}

/* derivative of the log-product: sum_k 1/(x - xi_k) */
static double leja_dlog(double x, const double *xi, int n) {
  double s = 0.0;
  for (int k = 0; k < n; k++) s += 1.0 / (x - xi[k]);
  return s;
}

/*
 * xi_0 = 2 and xi_j = argmax_{x in [-2,2]} prod_{k<j} |x - xi_k|.
 * Once both endpoints are nodes, the maximum lies strictly inside one gap
 * between consecutive nodes; there the log-product is strictly concave, so its
 * unique maximiser is the zero of its derivative, found by bisection to the
 * last bit.  The winning gap is the one with the largest log-product; values
 * within 1e-10 of the best count as a tie, resolved towards the larger x.
 */
int orc_leja_points(int m, double *xi) {
  if (m < 0 || !xi) return ORC_EINVAL;
  xi[0] = 2.0;
  if (m == 0) return ORC_OK;
  xi[1] = -2.0; /* the maximiser of |x - 2| on [-2,2] */
  double *s = (double *)malloc(sizeof(double) * (size_t)(m + 1));
  double *cx = (double *)malloc(sizeof(double) * (size_t)(m + 1));
  double *cl = (double *)malloc(sizeof(double) * (size_t)(m + 1));
  if (!s || !cx || !cl) { free(s); free(cx); free(cl); return ORC_ENOMEM; }
  for (int j = 2; j <= m; j++) {
    /* sorted copy of the current nodes (insertion sort) */
    for (int k = 0; k < j; k++) s[k] = xi[k];
    for (int a = 1; a < j; a++) {
      double v = s[a];
      int b = a - 1;
      while (b >= 0 && s[b] > v) { s[b + 1] = s[b]; b--; }
      s[b + 1] = v;
    }
    double best = -INFINITY;
    for (int g = 0; g + 1 < j; g++) {
      double lo = s[g], hi = s[g + 1];
      double mid = 0.5 * (lo + hi);
      for (;;) {
        mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double slope = leja_dlog(mid, xi, j);
        if (slope == 0.0) break;
        if (slope > 0.0) lo = mid; else hi = mid;
      }
      cx[g] = mid;
      cl[g] = leja_logprod(mid, xi, j);
      if (cl[g] > best) best = cl[g];
    }
    double pick = -INFINITY;
    for (int g = 0; g + 1 < j; g++)
      if (cl[g] >= best - 1e-10 && cx[g] > pick) pick = cx[g];
    xi[j] = pick;
  }
  free(s); free(cx); free(cl);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Divided differences d_i = exp[xi_0,...,xi_i] (Sec. 3).                      */
/* ------------------------------------------------------------------------- */

/* C = A*B for lower-triangular n x n matrices (row-major). */
static void lt_matmul(int n, const double complex *A, const double complex *B, double complex *C) {
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      double complex acc = 0.0;
      if (j <= i)
        for (int k = j; k <= i; k++) acc += A[i * n + k] * B[k * n + j];
      C[i * n + j] = acc;
    }
}

static double mat_norm1(int n, const double complex *A) {
  double best = 0.0;
  for (int j = 0; j < n; j++) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += cabs(A[i * n + j]);
    if (s > best) best = s;
  }
  return best;
}

/*
 * Opitz: for the lower bidiagonal Z with diagonal xi_0..xi_m and ones below it,
 * the first column of g(Z) lists the divided differences g[xi_0..xi_j].  Here
 * g(x) = exp(-i rho x), and g(Z) = exp(-i rho Z) is evaluated by a Taylor series
 * of the scaled matrix (1-norm <= 1/2) followed by repeated squaring.
 */
int orc_divided_differences(int m, const double *xi, double rho, double complex *d) {
  if (m < 0 || !xi || !d) return ORC_EINVAL;
  const int n = m + 1;
  size_t bytes = sizeof(double complex) * (size_t)n * (size_t)n;
  double complex *A = (double complex *)malloc(bytes);
  double complex *T = (double complex *)malloc(bytes);
  double complex *P = (double complex *)malloc(bytes);
  double complex *Q = (double complex *)malloc(bytes);
  if (!A || !T || !P || !Q) { free(A); free(T); free(P); free(Q); return ORC_ENOMEM; }
  memset(A, 0, bytes);
  for (int j = 0; j < n; j++) {
    A[j * n + j] = -I * rho * xi[j];
    if (j > 0) A[j * n + j - 1] = -I * rho;
  }
  int q = 0;
  double nrm = mat_norm1(n, A);
  while (nrm > 0.5) { nrm *= 0.5; q++; }
  double scale = ldexp(1.0, -q);
  for (int e = 0; e < n * n; e++) A[e] *= scale;
  /* T = sum_k A^k / k!, P holds the current term */
  memset(T, 0, bytes);
  memset(P, 0, bytes);
  for (int j = 0; j < n; j++) { T[j * n + j] = 1.0; P[j * n + j] = 1.0; }
  for (int k = 1; k <= 60; k++) {
    lt_matmul(n, P, A, Q);
    for (int e = 0; e < n * n; e++) { P[e] = Q[e] / (double)k; T[e] += P[e]; }
    if (mat_norm1(n, P) <= 1e-20 * mat_norm1(n, T)) break;
  }
  for (int r = 0; r < q; r++) {
    lt_matmul(n, T, T, Q);
    memcpy(T, Q, bytes);
  }
  for (int j = 0; j < n; j++) d[j] = T[j * n + 0];
  free(A); free(T); free(P); free(Q);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Spin-chain Hamiltonians (Sec. 4, Pauli matrices and Kronecker embedding).  */
/* ------------------------------------------------------------------------- */
/*
 * sigma_j^alpha = I x ... x sigma^alpha x ... x I with spin 1 the leftmost
 * factor, so for n spins the basis index is x = sum_j b_j 2^(n-j): spin j sits
 * at bit (n-j).  On a basis state, with z_j = 1 - 2 b_j:
 *   sigma^z_j |x> = z_j |x>,  sigma^x_j |x> = |x ^ bit_j>,
 *   sigma^y_j |x> = i z_j |x ^ bit_j>      (sigma^y = [[0,-i],[i,0]]).
 * Hence sigma^x_i sigma^x_j + sigma^y_i sigma^y_j maps |x> to
 * (1 - z_i z_j) |x ^ bit_i ^ bit_j>: 2 for anti-parallel spins, 0 otherwise,
 * and every such matrix is real symmetric.
 */
static inline int64_t spin_bit(int nspins, int j /* 1-based */) { return (int64_t)1 << (nspins - j); }
static inline double spin_z(int64_t x, int nspins, int j) { return (x & spin_bit(nspins, j)) ? -1.0 : 1.0; }

int64_t orc_xxz_nnz(int nspins, const double *J, double delta) {
  (void)J; (void)delta;
  int64_t D = (int64_t)1 << nspins;
  return D + (int64_t)(nspins - 1) * (D / 2);
}

/*
 * Open XXZ chain: H_s = sum_{i=1}^{n-1} J_i (sx_i sx_{i+1} + sy_i sy_{i+1} + delta sz_i sz_{i+1})
 *                       + sum_{i=1}^{n} h_i sz_i.
 * J[i-1] = J_i, hz[i-1] = h_i.  Row x stores the diagonal (always) and one entry
 * per anti-parallel bond; columns ascending.
 */
int orc_build_xxz_csr(int nspins, const double *J, const double *hz, double delta,
                      int64_t *rowptr, int32_t *col, double complex *val) {
  if (nspins < 2 || nspins > 30) return ORC_EINVAL;
  int64_t D = (int64_t)1 << nspins;
  int64_t pos = 0;
  int64_t ccol[64];
  double complex cval[64];
  for (int64_t x = 0; x < D; x++) {
    rowptr[x] = pos;
    int cnt = 0;
    double diag = 0.0;
    for (int i = 1; i <= nspins - 1; i++) diag += delta * J[i - 1] * spin_z(x, nspins, i) * spin_z(x, nspins, i + 1);
    for (int i = 1; i <= nspins; i++) diag += hz[i - 1] * spin_z(x, nspins, i);
    ccol[cnt] = x; cval[cnt] = diag; cnt++;
    for (int i = 1; i <= nspins - 1; i++) {
      double zz = spin_z(x, nspins, i) * spin_z(x, nspins, i + 1);
      if (zz < 0.0) {
        ccol[cnt] = x ^ spin_bit(nspins, i) ^ spin_bit(nspins, i + 1);
        cval[cnt] = J[i - 1] * (1.0 - zz);
        cnt++;
      }
    }
    for (int a = 1; a < cnt; a++) { /* insertion sort by column */
      int64_t c = ccol[a]; double complex v = cval[a]; int b = a - 1;
      while (b >= 0 && ccol[b] > c) { ccol[b + 1] = ccol[b]; cval[b + 1] = cval[b]; b--; }
      ccol[b + 1] = c; cval[b + 1] = v;
    }
    for (int a = 0; a < cnt; a++) { col[pos] = (int32_t)ccol[a]; val[pos] = cval[a]; pos++; }
  }
  rowptr[D] = pos;
  return ORC_OK;
}

/* Transverse field sum_{i=1}^{n} sx_i: row x has a 1 at every column x ^ bit_i. */
int orc_build_field_x_csr(int nspins, int64_t *rowptr, int32_t *col, double complex *val) {
  if (nspins < 1 || nspins > 30) return ORC_EINVAL;
  int64_t D = (int64_t)1 << nspins;
  int64_t pos = 0;
  int64_t ccol[64];
  for (int64_t x = 0; x < D; x++) {
    rowptr[x] = pos;
    int cnt = 0;
    for (int i = 1; i <= nspins; i++) ccol[cnt++] = x ^ spin_bit(nspins, i);
    for (int a = 1; a < cnt; a++) {
      int64_t c = ccol[a]; int b = a - 1;
      while (b >= 0 && ccol[b] > c) { ccol[b + 1] = ccol[b]; b--; }
      ccol[b + 1] = c;
    }
    for (int a = 0; a < cnt; a++) { col[pos] = (int32_t)ccol[a]; val[pos] = 1.0; pos++; }
  }
  rowptr[D] = pos;
  return ORC_OK;
}

/*
 * Long-range chain, every pair i<j once:
 * H_s = sum_{i<j} J_ij (sx_i sx_j + sy_i sy_j + delta sz_i sz_j) + sum_i h_i sz_i,
 * J_ij = 1/|i-j|^alpha.  Dense, row-major D x D.
 */
int orc_build_longrange_dense(int nspins, double alpha, const double *hz, double delta, double complex *H) {
  if (nspins < 2 || nspins > 15) return ORC_EINVAL;
  int64_t D = (int64_t)1 << nspins;
  memset(H, 0, sizeof(double complex) * (size_t)D * (size_t)D);
  for (int64_t x = 0; x < D; x++) {
    double diag = 0.0;
    for (int i = 1; i <= nspins; i++) diag += hz[i - 1] * spin_z(x, nspins, i);
    for (int i = 1; i <= nspins; i++)
      for (int j = i + 1; j <= nspins; j++) {
        double Jij = 1.0 / pow((double)(j - i), alpha);
        double zz = spin_z(x, nspins, i) * spin_z(x, nspins, j);
        diag += delta * Jij * zz;
        if (zz < 0.0) {
          int64_t y = x ^ spin_bit(nspins, i) ^ spin_bit(nspins, j);
          H[x * D + y] += Jij * (1.0 - zz);
        }
      }
    H[x * D + x] += diag;
  }
  return ORC_OK;
}

int orc_build_field_x_dense(int nspins, double complex *H) {
  if (nspins < 1 || nspins > 15) return ORC_EINVAL;
  int64_t D = (int64_t)1 << nspins;
  memset(H, 0, sizeof(double complex) * (size_t)D * (size_t)D);
  for (int64_t x = 0; x < D; x++)
    for (int i = 1; i <= nspins; i++) H[x * D + (x ^ spin_bit(nspins, i))] = 1.0;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Problem: H(t) = sum_k f_k(t) H_k (Sec. 4, split H = H_1 + h(t) H_2).       */
/* ------------------------------------------------------------------------- */

typedef struct {
  int kind;
  const int64_t *rowptr;
  const int32_t *col;
  const double complex *val;
  double a, b; /* Gershgorin enclosure of the spectrum */
  int set;
} orc_term;

typedef struct {
  double a0;
  int nmodes;
  double *ac, *as, *om;
} orc_coeff;

struct orc_problem {
  int64_t dim;
  int nterms;
  orc_term term[MAX_TERMS];
  orc_coeff coeff[MAX_TERMS];
  double tol_rel, tol_abs, rho_max;
  int m_max;
  double xi[1024];
};

orc_problem *orc_problem_new(int64_t dim, int nterms) {
  if (dim < 1 || nterms < 1 || nterms > MAX_TERMS) return NULL;
  orc_problem *p = (orc_problem *)calloc(1, sizeof(orc_problem));
  if (!p) return NULL;
  p->dim = dim;
  p->nterms = nterms;
  p->tol_rel = 1e-10; /* Sec. 4: relative and absolute tolerance 1e-10 */
  p->tol_abs = 1e-10;
  p->m_max = 100;
  p->rho_max = 4.0;
  orc_leja_points(p->m_max, p->xi);
  return p;
}

void orc_problem_free(orc_problem *p) {
  if (!p) return;
  for (int k = 0; k < MAX_TERMS; k++) { free(p->coeff[k].ac); free(p->coeff[k].as); free(p->coeff[k].om); }
  free(p);
}

/* Gershgorin: spec(H) within [min_i (H_ii - R_i), max_i (H_ii + R_i)], R_i = sum_{j != i} |H_ij|. */
static void gershgorin(orc_term *t, int64_t D) {
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = 0; i < D; i++) {
    double c = 0.0, R = 0.0;
    if (t->kind == ORC_TERM_CSR) {
      for (int64_t e = t->rowptr[i]; e < t->rowptr[i + 1]; e++) {
        if (t->col[e] == i) c += creal(t->val[e]);
        else R += cabs(t->val[e]);
      }
    } else {
      for (int64_t j = 0; j < D; j++) {
        if (j == i) c += creal(t->val[i * D + j]);
        else R += cabs(t->val[i * D + j]);
      }
    }
    if (c - R < lo) lo = c - R;
    if (c + R > hi) hi = c + R;
  }
  t->a = lo;
  t->b = hi;
}

int orc_set_csr(orc_problem *p, int k, const int64_t *rowptr, const int32_t *col, const double complex *val) {
  if (!p || k < 0 || k >= p->nterms || !rowptr || !col || !val) return ORC_EINVAL;
  orc_term *t = &p->term[k];
  t->kind = ORC_TERM_CSR; t->rowptr = rowptr; t->col = col; t->val = val; t->set = 1;
  gershgorin(t, p->dim);
  return ORC_OK;
}

int orc_set_dense(orc_problem *p, int k, const double complex *H) {
  if (!p || k < 0 || k >= p->nterms || !H) return ORC_EINVAL;
  orc_term *t = &p->term[k];
  t->kind = ORC_TERM_DENSE; t->rowptr = NULL; t->col = NULL; t->val = H; t->set = 1;
  gershgorin(t, p->dim);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Lanczos enclosure of a term's spectrum (Sec. 3: the Leja parameters need  */
/* a spectral estimate; this one is tighter than Gershgorin).                 */
/* ------------------------------------------------------------------------- */

/* SplitMix64 (Steele, Lea, Flood 2014) in counter form: output c of the stream that starts at
 * `seed`, i.e. the mix of seed + (c + 1) * 0x9E3779B97F4A7C15. */
static uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double unit_at(uint64_t seed, uint64_t c) { return (double)(splitmix64_at(seed, c) >> 11) * 0x1.0p-53; }

/* number of eigenvalues of the symmetric tridiagonal T (diagonal al[0..m-1], off-diagonal
 * be[1..m-1]) below x, by the signs of the Sturm sequence of the LDL^T pivots */
static int sturm_count(const double *al, const double *be, int m, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < m; i++) {
    double off = (i > 0) ? be[i] * be[i] / q : 0.0;
    q = al[i] - x - off;
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) cnt++;
  }
  return cnt;
}

/* the idx-th smallest eigenvalue of T by bisection (Gershgorin start interval, 200 halvings) */
static double tridiag_eig(const double *al, const double *be, int m, int idx) {
  double lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < m; i++) {
    double r = (i > 0 ? fabs(be[i]) : 0.0) + (i + 1 < m ? fabs(be[i + 1]) : 0.0);
    if (al[i] - r < lo) lo = al[i] - r;
    if (al[i] + r > hi) hi = al[i] + r;
  }
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(al, be, m, mid) > idx) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

/* |last component| of the unit eigenvector of T for the eigenvalue theta: three steps of inverse
 * iteration with the shift theta + shift (outside the spectrum, so T - shift I is definite and the
 * tridiagonal solve needs no pivoting) */
static double tridiag_last_component(const double *al, const double *be, int m, double theta, double shift) {
  double *x = (double *)malloc(sizeof(double) * 3 * (size_t)m);
  if (!x) return 1.0;
  double *c = x + m, *d = x + 2 * m;
  for (int i = 0; i < m; i++) x[i] = 1.0;
  const double sig = theta + shift;
  for (int it = 0; it < 3; it++) {
    /* solve (T - sig I) y = x (Thomas), y into x */
    double piv = al[0] - sig;
    c[0] = (m > 1) ? be[1] / piv : 0.0;
    d[0] = x[0] / piv;
    for (int i = 1; i < m; i++) {
      piv = (al[i] - sig) - be[i] * c[i - 1];
      c[i] = (i + 1 < m) ? be[i + 1] / piv : 0.0;
      d[i] = (x[i] - be[i] * d[i - 1]) / piv;
    }
    x[m - 1] = d[m - 1];
    for (int i = m - 2; i >= 0; i--) x[i] = d[i] - c[i] * x[i + 1];
    double n2 = 0.0;
    for (int i = 0; i < m; i++) n2 += x[i] * x[i];
    const double inv = 1.0 / sqrt(n2);
    for (int i = 0; i < m; i++) x[i] *= inv;
  }
  const double last = fabs(x[m - 1]);
  free(x);
  return last;
}

/*
 * Reading (the Leja parameters need a spectral estimate; Sec. 3 defers to [ckor15]): m steps of the
 * Lanczos recurrence on H_k from the start vector v_i = (2u_{2i} - 1) + i (2u_{2i+1} - 1),
 * u_c = unit_at(1709064830, c), normalised:
 *     w = H v_j;  al_j = Re <v_j, w>;  w -= al_j v_j + be_j v_{j-1};  be_{j+1} = |w|;  v_{j+1} = w / be_{j+1},
 * stopped early when be_{j+1} <= 1e-12 (max |al| + max be) (an invariant subspace).  With
 * theta_min/max the extreme eigenvalues of the tridiagonal T and r = be_m |s_last| the residual
 * norms of their Ritz vectors, the enclosure is
 *     [theta_min - r_min - 0.01 W, theta_max + r_max + 0.01 W] intersected with Gershgorin,
 * W = theta_max - theta_min (Ritz values lie inside the spectrum; the residual and the 1 % margin
 * cover the part of the spectrum the Krylov space has not resolved).
 */
int orc_set_interval_lanczos(orc_problem *p, int k, int m) {
  if (!p || k < 0 || k >= p->nterms || !p->term[k].set || m < 1) return ORC_EINVAL;
  const int64_t D = p->dim;
  if (m > D) m = (int)D;
  double complex *v0 = (double complex *)calloc((size_t)D, sizeof(double complex));
  double complex *v1 = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double complex *w = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double *al = (double *)calloc((size_t)m + 1, sizeof(double));
  double *be = (double *)calloc((size_t)m + 2, sizeof(double));
  if (!v0 || !v1 || !w || !al || !be) { free(v0); free(v1); free(w); free(al); free(be); return ORC_ENOMEM; }
  const uint64_t seed = 1709064830ull;
  double n2 = 0.0;
  for (int64_t i = 0; i < D; i++) {
    v1[i] = (2.0 * unit_at(seed, 2 * (uint64_t)i) - 1.0) + I * (2.0 * unit_at(seed, 2 * (uint64_t)i + 1) - 1.0);
    n2 += creal(v1[i]) * creal(v1[i]) + cimag(v1[i]) * cimag(v1[i]);
  }
  for (int64_t i = 0; i < D; i++) v1[i] /= sqrt(n2);
  int mj = 0;
  double amax = 0.0, bmax = 0.0;
  for (int j = 0; j < m; j++) {
    orc_apply_term(p, k, v1, w);
    double a = 0.0;
    for (int64_t i = 0; i < D; i++) a += creal(conj(v1[i]) * w[i]);
    al[j] = a;
    for (int64_t i = 0; i < D; i++) w[i] -= a * v1[i] + be[j] * v0[i];
    double b2 = 0.0;
    for (int64_t i = 0; i < D; i++) b2 += creal(w[i]) * creal(w[i]) + cimag(w[i]) * cimag(w[i]);
    be[j + 1] = sqrt(b2);
    mj = j + 1;
    if (fabs(a) > amax) amax = fabs(a);
    if (be[j + 1] > bmax) bmax = be[j + 1];
    if (be[j + 1] <= 1e-12 * (amax + bmax)) { be[j + 1] = 0.0; break; }
    for (int64_t i = 0; i < D; i++) { v0[i] = v1[i]; v1[i] = w[i] / be[j + 1]; }
  }
  const double tmin = tridiag_eig(al, be, mj, 0), tmax = tridiag_eig(al, be, mj, mj - 1);
  const double W = tmax - tmin;
  const double eps = 1e-9 * (fabs(tmin) + fabs(tmax) + W + 1e-300);
  const double rmin = (mj > 1 || be[mj] > 0.0) ? be[mj] * tridiag_last_component(al, be, mj, tmin, -eps) : 0.0;
  const double rmax = (mj > 1 || be[mj] > 0.0) ? be[mj] * tridiag_last_component(al, be, mj, tmax, eps) : 0.0;
  double a = tmin - rmin - 0.01 * W, b = tmax + rmax + 0.01 * W;
  orc_term *t = &p->term[k];
  if (a < t->a) a = t->a;
  if (b > t->b) b = t->b;
  t->a = a;
  t->b = b;
  free(v0); free(v1); free(w); free(al); free(be);
  return ORC_OK;
}

int orc_set_coeff(orc_problem *p, int k, double a0, int nmodes, const double *ac, const double *as,
                  const double *om) {
  if (!p || k < 0 || k >= p->nterms || nmodes < 0) return ORC_EINVAL;
  orc_coeff *c = &p->coeff[k];
  free(c->ac); free(c->as); free(c->om);
  c->ac = c->as = c->om = NULL;
  c->a0 = a0;
  c->nmodes = nmodes;
  if (nmodes > 0) {
    c->ac = (double *)malloc(sizeof(double) * (size_t)nmodes);
    c->as = (double *)malloc(sizeof(double) * (size_t)nmodes);
    c->om = (double *)malloc(sizeof(double) * (size_t)nmodes);
    if (!c->ac || !c->as || !c->om) return ORC_ENOMEM;
    for (int m = 0; m < nmodes; m++) {
      c->ac[m] = ac ? ac[m] : 0.0;
      c->as[m] = as ? as[m] : 0.0;
      c->om[m] = om[m];
    }
  }
  return ORC_OK;
}

int orc_set_leja(orc_problem *p, double tol_rel, double tol_abs, int m_max, double rho_max) {
  if (!p || m_max < 1 || m_max > 1000 || !(rho_max > 0.0)) return ORC_EINVAL;
  p->tol_rel = tol_rel; p->tol_abs = tol_abs; p->m_max = m_max; p->rho_max = rho_max;
  return orc_leja_points(m_max, p->xi);
}

int orc_term_interval(const orc_problem *p, int k, double *a, double *b) {
  if (!p || k < 0 || k >= p->nterms || !p->term[k].set) return ORC_EINVAL;
  *a = p->term[k].a; *b = p->term[k].b;
  return ORC_OK;
}

/* f_k(t) = a0 + sum_m (ac_m cos(om_m t) + as_m sin(om_m t)) */
double orc_coeff_eval(const orc_problem *p, int k, double t) {
  const orc_coeff *c = &p->coeff[k];
  double f = c->a0;
  for (int m = 0; m < c->nmodes; m++) f += c->ac[m] * cos(c->om[m] * t) + c->as[m] * sin(c->om[m] * t);
  return f;
}

/* y = H_k x */
int orc_apply_term(const orc_problem *p, int k, const double complex *x, double complex *y) {
  if (!p || k < 0 || k >= p->nterms || !p->term[k].set) return ORC_EINVAL;
  const orc_term *t = &p->term[k];
  const int64_t D = p->dim;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < D; i++) {
    double complex acc = 0.0;
    if (t->kind == ORC_TERM_CSR) {
      for (int64_t e = t->rowptr[i]; e < t->rowptr[i + 1]; e++) acc += t->val[e] * x[t->col[e]];
    } else {
      for (int64_t j = 0; j < D; j++) acc += t->val[i * D + j] * x[j];
    }
    y[i] = acc;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Generators K (one exponential exp(-iK)).                                   */
/* ------------------------------------------------------------------------- */

enum { GEN_LINEAR = 0, GEN_M4 = 1, GEN_M6 = 2 };

typedef struct {
  const orc_problem *p;
  int mode;
  double beta[MAX_TERMS]; /* GEN_LINEAR: K = sum_k beta_k H_k                                */
  double f1[MAX_TERMS];   /* GEN_M4, GEN_M6: f_k(t_n + c_1 h)                                */
  double f2[MAX_TERMS];   /*                 f_k(t_n + c_2 h)                                */
  double f3[MAX_TERMS];   /* GEN_M6:         f_k(t_n + c_3 h)                                */
  double h;               /*         step size                                               */
  double complex *u1, *u2, *t1, *t2; /* scratch of length dim                               */
  double complex *s6[12];            /* GEN_M6 scratch of length dim                        */
  orc_stats *st;
} orc_gen;

/* y = sum_k coef_k H_k x */
static void apply_combo(const orc_gen *g, const double *coef, const double complex *x, double complex *y,
                        double complex *tmp) {
  const int64_t D = g->p->dim;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < D; i++) y[i] = 0.0;
  for (int k = 0; k < g->p->nterms; k++) {
    orc_apply_term(g->p, k, x, tmp);
    if (g->st) g->st->n_termapply++;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < D; i++) y[i] += coef[k] * tmp[i];
  }
}

/*
 * y = K x.
 * GEN_LINEAR: K = sum_k beta_k H_k.
 * GEN_M4 (Sec. 2, Method M4, with A = -iH):
 *   Omega = h/2 (A_1 + A_2) + (sqrt(3) h^2 / 12) [A_2, A_1]
 *         = -i [ h/2 (H_1 + H_2) - i (sqrt(3) h^2/12) [H_2, H_1] ] = -i K,
 * with the commutator applied to a vector as H_2(H_1 x) - H_1(H_2 x).
 */
/*
 * Method M6 (Sec. 2) with A_i = -i H(t_n + c_i h), c = 1/2 -+ sqrt(15)/10, 1/2:
 *   B_1 = h A_2,  B_2 = (sqrt(15)/3) h (A_3 - A_1),  B_3 = (10/3) h (A_3 - 2 A_2 + A_1),
 *   Omega = B_1 + B_3/12 + (1/240) [U, V],
 *   U = -20 B_1 - B_3 + [B_1, B_2],   V = B_2 - (1/60) [B_1, 2 B_3 + [B_1, B_2]],
 * every operator applied to vectors ([F, G] x = F(G x) - G(F x)); K = i Omega.
 */
static void m6_apply_B(orc_gen *g, int j, const double complex *x, double complex *y) {
  const double r15 = sqrt(15.0);
  double coef[MAX_TERMS];
  for (int k = 0; k < g->p->nterms; k++) {
    if (j == 1) coef[k] = g->h * g->f2[k];
    else if (j == 2) coef[k] = r15 / 3.0 * g->h * (g->f3[k] - g->f1[k]);
    else coef[k] = 10.0 / 3.0 * g->h * (g->f3[k] - 2.0 * g->f2[k] + g->f1[k]);
  }
  apply_combo(g, coef, x, y, g->t1); /* y = sum_k coef_k H_k x; B_j x = -i y */
  const int64_t D = g->p->dim;
  for (int64_t i = 0; i < D; i++) y[i] *= -I;
}

/* y = [B_1, B_2] x; uses s6[10], s6[11] */
static void m6_apply_B12(orc_gen *g, const double complex *x, double complex *y) {
  const int64_t D = g->p->dim;
  double complex *a = g->s6[10], *b = g->s6[11];
  m6_apply_B(g, 2, x, a);
  m6_apply_B(g, 1, a, y);  /* B_1 (B_2 x) */
  m6_apply_B(g, 1, x, a);
  m6_apply_B(g, 2, a, b);  /* B_2 (B_1 x) */
  for (int64_t i = 0; i < D; i++) y[i] -= b[i];
}

/* y = U x = -20 B_1 x - B_3 x + [B_1, B_2] x; uses s6[7..11] */
static void m6_apply_U(orc_gen *g, const double complex *x, double complex *y) {
  const int64_t D = g->p->dim;
  double complex *b1 = g->s6[7], *b3 = g->s6[8];
  m6_apply_B(g, 1, x, b1);
  m6_apply_B(g, 3, x, b3);
  m6_apply_B12(g, x, y);
  for (int64_t i = 0; i < D; i++) y[i] += -20.0 * b1[i] - b3[i];
}

/* y = W x = 2 B_3 x + [B_1, B_2] x; uses s6[9..11] */
static void m6_apply_W(orc_gen *g, const double complex *x, double complex *y) {
  const int64_t D = g->p->dim;
  double complex *b3 = g->s6[9];
  m6_apply_B12(g, x, y);
  m6_apply_B(g, 3, x, b3);
  for (int64_t i = 0; i < D; i++) y[i] += 2.0 * b3[i];
}

/* y = V x = B_2 x - (1/60) (B_1 (W x) - W (B_1 x)); uses s6[4..11] */
static void m6_apply_V(orc_gen *g, const double complex *x, double complex *y) {
  const int64_t D = g->p->dim;
  double complex *wx = g->s6[4], *b1wx = g->s6[5], *b1x = g->s6[6], *wb1x = g->s6[7];
  m6_apply_W(g, x, wx);
  m6_apply_B(g, 1, wx, b1wx);
  m6_apply_B(g, 1, x, b1x);
  m6_apply_W(g, b1x, wb1x);
  m6_apply_B(g, 2, x, y);
  for (int64_t i = 0; i < D; i++) y[i] -= (b1wx[i] - wb1x[i]) / 60.0;
}

static void m6_apply_K(orc_gen *g, const double complex *x, double complex *y) {
  const int64_t D = g->p->dim;
  double complex *ux = g->s6[0], *vx = g->s6[1], *uvx = g->s6[2], *vux = g->s6[3];
  m6_apply_U(g, x, ux);
  m6_apply_V(g, x, vx);
  m6_apply_U(g, vx, uvx);
  m6_apply_V(g, ux, vux);
  /* Omega x = B_1 x + B_3 x / 12 + (U V x - V U x) / 240 (B_1 x, B_3 x into ux, vx) */
  m6_apply_B(g, 1, x, ux);
  m6_apply_B(g, 3, x, vx);
  for (int64_t i = 0; i < D; i++) y[i] = I * (ux[i] + vx[i] / 12.0 + (uvx[i] - vux[i]) / 240.0);
}

static void gen_apply(orc_gen *g, const double complex *x, double complex *y) {
  const int64_t D = g->p->dim;
  if (g->mode == GEN_LINEAR) {
    apply_combo(g, g->beta, x, y, g->t1);
    return;
  }
  if (g->mode == GEN_M6) {
    m6_apply_K(g, x, y);
    return;
  }
  const double kappa = sqrt(3.0) * g->h * g->h / 12.0;
  apply_combo(g, g->f1, x, g->u1, g->t1);    /* u1 = H_1 x        */
  apply_combo(g, g->f2, x, g->u2, g->t1);    /* u2 = H_2 x        */
  apply_combo(g, g->f2, g->u1, y, g->t1);    /* y  = H_2 (H_1 x)  */
  apply_combo(g, g->f1, g->u2, g->t2, g->t1);/* t2 = H_1 (H_2 x)  */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < D; i++)
    y[i] = 0.5 * g->h * (g->u1[i] + g->u2[i]) - I * kappa * (y[i] - g->t2[i]);
}

/* Spectral enclosure [a,b] of K (see the readings at the top). */
static void gen_interval(const orc_gen *g, double *a, double *b) {
  const orc_problem *p = g->p;
  double lo = 0.0, hi = 0.0;
  double lin[MAX_TERMS];
  for (int k = 0; k < p->nterms; k++) {
    if (g->mode == GEN_LINEAR) lin[k] = g->beta[k];
    else if (g->mode == GEN_M4) lin[k] = 0.5 * g->h * (g->f1[k] + g->f2[k]);
    else /* GEN_M6: i (B_1 + B_3 / 12) = h (f_2 + (10/36)(f_3 - 2 f_2 + f_1)) */
      lin[k] = g->h * (g->f2[k] + 10.0 / 36.0 * (g->f3[k] - 2.0 * g->f2[k] + g->f1[k]));
  }
  for (int k = 0; k < p->nterms; k++) {
    double x1 = lin[k] * p->term[k].a, x2 = lin[k] * p->term[k].b;
    lo += (x1 < x2) ? x1 : x2;
    hi += (x1 < x2) ? x2 : x1;
  }
  if (g->mode == GEN_M4) {
    const double kappa = sqrt(3.0) * g->h * g->h / 12.0;
    double r = 0.0;
    for (int k = 0; k < p->nterms; k++)
      for (int l = k + 1; l < p->nterms; l++) {
        double coef = g->f2[k] * g->f1[l] - g->f2[l] * g->f1[k];
        double hwk = 0.5 * (p->term[k].b - p->term[k].a);
        double hwl = 0.5 * (p->term[l].b - p->term[l].a);
        r += fabs(coef) * 2.0 * hwk * hwl;
      }
    lo -= kappa * r;
    hi += kappa * r;
  }
  if (g->mode == GEN_M6) {
    /* B_1 = -iP, B_2 = -iQ, B_3 = -iR with P, Q, R = sum_k {p,q,r}_k H_k, S = 20 P + R, C = [P,Q]:
     *   U = iS - C,  V = -iQ + E,  E = [P,R]/30 - (i/60)[P,C],
     *   [U,V] = [S,Q] + i[S,E] - [C,V].
     * Shifting any H_k by a multiple of I changes no commutator, so with the half-widths hw_k:
     *   |[F,G]| <= sum_{k<l} |f_k g_l - f_l g_k| 2 hw_k hw_l  (F, G combinations of the H_k),
     *   |[F,M]| <= 2 |F| |M|,  |F| <= sum_k |f_k| hw_k  (after the shift),
     * so |(i/240)[U,V]| <= r = (|[S,Q]| + 2|S||E| + 2|C||V|) / 240 with
     *   |E| <= |[P,R]|/30 + |P||C|/30,  |V| <= |Q| + |E|. */
    const double r15 = sqrt(15.0);
    double pk[MAX_TERMS], qk[MAX_TERMS], rk[MAX_TERMS], sk[MAX_TERMS], hw[MAX_TERMS];
    for (int k = 0; k < p->nterms; k++) {
      pk[k] = g->h * g->f2[k];
      qk[k] = r15 / 3.0 * g->h * (g->f3[k] - g->f1[k]);
      rk[k] = 10.0 / 3.0 * g->h * (g->f3[k] - 2.0 * g->f2[k] + g->f1[k]);
      sk[k] = 20.0 * pk[k] + rk[k];
      hw[k] = 0.5 * (p->term[k].b - p->term[k].a);
    }
    double pq = 0.0, pr = 0.0, sq = 0.0, pn = 0.0, sn = 0.0, qn = 0.0;
    for (int k = 0; k < p->nterms; k++) {
      pn += fabs(pk[k]) * hw[k];
      sn += fabs(sk[k]) * hw[k];
      qn += fabs(qk[k]) * hw[k];
      for (int l = k + 1; l < p->nterms; l++) {
        pq += fabs(pk[k] * qk[l] - pk[l] * qk[k]) * 2.0 * hw[k] * hw[l];
        pr += fabs(pk[k] * rk[l] - pk[l] * rk[k]) * 2.0 * hw[k] * hw[l];
        sq += fabs(sk[k] * qk[l] - sk[l] * qk[k]) * 2.0 * hw[k] * hw[l];
      }
    }
    const double en = pr / 30.0 + pn * pq / 30.0;
    const double vn = qn + en;
    const double r = (sq + 2.0 * sn * en + 2.0 * pq * vn) / 240.0;
    lo -= r;
    hi += r;
  }
  *a = lo;
  *b = hi;
}

static double vnorm(const double complex *x, int64_t D) {
  double s = 0.0;
  for (int64_t i = 0; i < D; i++) s += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
  return sqrt(s);
}

/*
 * v <- exp(-iK) v by Newton-form Leja interpolation (Sec. 3):
 *   p_m(A) v = sum_i d_i prod_{j<i} (A - xi_j I) v, built by the short recurrence
 *   w = v, p = d_0 v;  for i = 1..m: w = A w - xi_{i-1} w;  p = p + d_i w,
 * applied here to A = X = (K - cI)/gamma and g(x) = exp(-i (gamma/s) x), s times,
 * each substep multiplied by e^{-ic/s}.
 */
static int leja_core(orc_gen *g, double complex *v) {
  const orc_problem *p = g->p;
  const int64_t D = p->dim;
  double a, b;
  gen_interval(g, &a, &b);
  const double c = 0.5 * (a + b);
  const double gamma = 0.25 * (b - a);
  if (g->st) g->st->n_exp++;
  if (!(gamma > 0.0)) { /* K is (enclosed by) a scalar: exp(-iK) v = e^{-ic} v */
    double complex ph = cexp(-I * c);
    for (int64_t i = 0; i < D; i++) v[i] *= ph;
    return ORC_OK;
  }
  int s = (int)ceil(gamma / p->rho_max);
  if (s < 1) s = 1;
  const double rho = gamma / s;
  double complex *d = (double complex *)malloc(sizeof(double complex) * (size_t)(p->m_max + 1));
  double complex *w = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double complex *Kw = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double complex *pp = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  if (!d || !w || !Kw || !pp) { free(d); free(w); free(Kw); free(pp); return ORC_ENOMEM; }
  orc_divided_differences(p->m_max, p->xi, rho, d);
  const double complex phase = cexp(-I * c / s);
  int rc = ORC_OK;
  for (int sub = 0; sub < s && rc == ORC_OK; sub++) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < D; i++) { w[i] = v[i]; pp[i] = d[0] * v[i]; }
    double e_prev = cabs(d[0]) * vnorm(w, D);
    int conv = 0, m = 0;
    for (int j = 1; j <= p->m_max; j++) {
      gen_apply(g, w, Kw);
      if (g->st) g->st->n_matvec++;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < D; i++) w[i] = (Kw[i] - c * w[i]) / gamma - p->xi[j - 1] * w[i];
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < D; i++) pp[i] += d[j] * w[i];
      double e = cabs(d[j]) * vnorm(w, D);
      double pn = vnorm(pp, D);
      if (!isfinite(pn) || !isfinite(e)) { rc = ORC_ENONFINITE; m = j; break; }
      if (e + e_prev <= p->tol_abs + p->tol_rel * pn) { conv = 1; m = j; break; }
      e_prev = e;
    }
    if (rc == ORC_OK && !conv) { rc = ORC_ENOCONV; m = p->m_max; }
    if (g->st) {
      g->st->n_substeps++;
      if (m > g->st->max_m) g->st->max_m = m;
      if (g->st->m_log && g->st->n_substeps <= g->st->m_log_cap) g->st->m_log[g->st->n_substeps - 1] = m;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < D; i++) v[i] = phase * pp[i];
  }
  free(d); free(w); free(Kw); free(pp);
  return rc;
}

static int gen_alloc(orc_gen *g, const orc_problem *p, orc_stats *st) {
  memset(g, 0, sizeof(*g));
  g->p = p;
  g->st = st;
  size_t bytes = sizeof(double complex) * (size_t)p->dim;
  g->u1 = (double complex *)malloc(bytes);
  g->u2 = (double complex *)malloc(bytes);
  g->t1 = (double complex *)malloc(bytes);
  g->t2 = (double complex *)malloc(bytes);
  if (!g->u1 || !g->u2 || !g->t1 || !g->t2) return ORC_ENOMEM;
  return ORC_OK;
}

static int gen_alloc_m6(orc_gen *g) {
  size_t bytes = sizeof(double complex) * (size_t)g->p->dim;
  for (int q = 0; q < 12; q++) {
    if (!g->s6[q]) g->s6[q] = (double complex *)malloc(bytes);
    if (!g->s6[q]) return ORC_ENOMEM;
  }
  return ORC_OK;
}

static void gen_free(orc_gen *g) {
  free(g->u1); free(g->u2); free(g->t1); free(g->t2);
  for (int q = 0; q < 12; q++) free(g->s6[q]);
}

static int check_problem(const orc_problem *p) {
  if (!p) return ORC_EINVAL;
  for (int k = 0; k < p->nterms; k++) if (!p->term[k].set) return ORC_EINVAL;
  return ORC_OK;
}

int orc_expv(const orc_problem *p, const double *beta, double complex *v, orc_stats *st) {
  int rc = check_problem(p);
  if (rc) return rc;
  orc_gen g;
  rc = gen_alloc(&g, p, st);
  if (rc == ORC_OK) {
    g.mode = GEN_LINEAR;
    for (int k = 0; k < p->nterms; k++) g.beta[k] = beta[k];
    rc = leja_core(&g, v);
  }
  gen_free(&g);
  return rc;
}

/* one exponential exp(-i h sum_k (sum_j alpha_j f_k(t_n + c_j h)) H_k) */
static int cf_exponential(orc_gen *g, const double *alpha, const double *c, int J, double tn, double h,
                          double complex *psi) {
  g->mode = GEN_LINEAR;
  for (int k = 0; k < g->p->nterms; k++) {
    double s = 0.0;
    for (int j = 0; j < J; j++) s += alpha[j] * orc_coeff_eval(g->p, k, tn + c[j] * h);
    g->beta[k] = h * s;
  }
  return leja_core(g, psi);
}

/*
 * Time stepping, Y_{n+1} = exp(Omega_n) Y_n (Sec. 2, Eq. (9)) with t_n = t0 + n h:
 *  M2    (Method M2):    Omega = h A(t_n + h/2).
 *  M6    (Method M6):    one exponential with the nested commutators (m6_apply_K).
 *  M4    (Method M4):    one exponential with the commutator (gen_apply).
 *  CF4   (Method Cf4):   exp(h(a1 A_1 + a2 A_2)) exp(h(a2 A_1 + a1 A_2)) Y_n,
 *                        c_{1,2} = 1/2 -+ sqrt(3)/6, a_{1,2} = (3 -+ 2 sqrt(3))/12;
 *                        the right factor acts first.
 *  CF4_3 (Method Cf4:3): three exponentials with the 3x3 alpha table and
 *                        c = 1/2 - sqrt(15)/10, 1/2, 1/2 + sqrt(15)/10; the
 *                        rightmost (third row) acts first.
 */
int orc_propagate(const orc_problem *p, double complex *psi, double t0, double h, int64_t nsteps,
                  int variant, orc_stats *st) {
  int rc = check_problem(p);
  if (rc) return rc;
  if (nsteps < 0) return ORC_EINVAL;
  orc_gen g;
  rc = gen_alloc(&g, p, st);
  const double r3 = sqrt(3.0), r15 = sqrt(15.0);
  const double c4[2] = {0.5 - r3 / 6.0, 0.5 + r3 / 6.0};
  const double a1 = (3.0 - 2.0 * r3) / 12.0, a2 = (3.0 + 2.0 * r3) / 12.0;
  const double c6[3] = {0.5 - r15 / 10.0, 0.5, 0.5 + r15 / 10.0};
  const double al3[3][3] = {
      {37.0 / 240.0 - 10.0 * r15 / 261.0, -1.0 / 30.0, 37.0 / 240.0 + 10.0 * r15 / 261.0},
      {-11.0 / 360.0, 23.0 / 45.0, -11.0 / 360.0},
      {37.0 / 240.0 + 10.0 * r15 / 261.0, -1.0 / 30.0, 37.0 / 240.0 - 10.0 * r15 / 261.0}};
  for (int64_t n = 0; n < nsteps && rc == ORC_OK; n++) {
    const double tn = t0 + (double)n * h;
    if (variant == ORC_CF4) {
      const double right[2] = {a2, a1}, left[2] = {a1, a2};
      rc = cf_exponential(&g, right, c4, 2, tn, h, psi);
      if (rc == ORC_OK) rc = cf_exponential(&g, left, c4, 2, tn, h, psi);
    } else if (variant == ORC_M4) {
      g.mode = GEN_M4;
      g.h = h;
      for (int k = 0; k < p->nterms; k++) {
        g.f1[k] = orc_coeff_eval(p, k, tn + c4[0] * h);
        g.f2[k] = orc_coeff_eval(p, k, tn + c4[1] * h);
      }
      rc = leja_core(&g, psi);
    } else if (variant == ORC_CF4_3) {
      for (int r = 2; r >= 0 && rc == ORC_OK; r--) rc = cf_exponential(&g, al3[r], c6, 3, tn, h, psi);
    } else if (variant == ORC_M2) {
      const double one = 1.0, half = 0.5;
      rc = cf_exponential(&g, &one, &half, 1, tn, h, psi);
    } else if (variant == ORC_M6) {
      rc = gen_alloc_m6(&g);
      g.mode = GEN_M6;
      g.h = h;
      for (int k = 0; k < p->nterms; k++) {
        g.f1[k] = orc_coeff_eval(p, k, tn + c6[0] * h);
        g.f2[k] = orc_coeff_eval(p, k, tn + c6[1] * h);
        g.f3[k] = orc_coeff_eval(p, k, tn + c6[2] * h);
      }
      if (rc == ORC_OK) rc = leja_core(&g, psi);
    } else {
      rc = ORC_EINVAL;
    }
  }
  gen_free(&g);
  return rc;
}

/* The enclosure gen_interval gives the generator of one M4 or M6 step (the nodes of orc_propagate). */
int orc_generator_interval(const orc_problem *p, int variant, double tn, double h, double *a, double *b) {
  int rc = check_problem(p);
  if (rc) return rc;
  if (!a || !b || (variant != ORC_M4 && variant != ORC_M6)) return ORC_EINVAL;
  orc_gen g;
  memset(&g, 0, sizeof(g));
  g.p = p;
  g.h = h;
  const double r3 = sqrt(3.0), r15 = sqrt(15.0);
  for (int k = 0; k < p->nterms; k++) {
    if (variant == ORC_M4) {
      g.mode = GEN_M4;
      g.f1[k] = orc_coeff_eval(p, k, tn + (0.5 - r3 / 6.0) * h);
      g.f2[k] = orc_coeff_eval(p, k, tn + (0.5 + r3 / 6.0) * h);
    } else {
      g.mode = GEN_M6;
      g.f1[k] = orc_coeff_eval(p, k, tn + (0.5 - r15 / 10.0) * h);
      g.f2[k] = orc_coeff_eval(p, k, tn + 0.5 * h);
      g.f3[k] = orc_coeff_eval(p, k, tn + (0.5 + r15 / 10.0) * h);
    }
  }
  gen_interval(&g, a, b);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Adjoint: gradient of a state-transfer fidelity with respect to the drive.  */
/* ------------------------------------------------------------------------- */

/*
 * [a; b] <- exp(Omega_aug) [a; b] for Omega_aug = -i [[K, H_kd], [0, K]], K = sum_k beta_k H_k,
 * by the Newton-form Leja recurrence of Sec. 3 on stacked vectors.  The block matrix has the
 * spectrum of K, so it uses K's enclosure, shift, scale, substeps and divided differences; the
 * early-termination test uses 2-norms of the stacked vectors.
 */
static int frechet_core(const orc_problem *p, const double *beta, int kd, double complex *a, double complex *b,
                        orc_stats *st) {
  const int64_t D = p->dim;
  orc_gen g;
  int rc = gen_alloc(&g, p, st);
  if (rc) { gen_free(&g); return rc; }
  g.mode = GEN_LINEAR;
  for (int k = 0; k < p->nterms; k++) g.beta[k] = beta[k];
  double lo, hi;
  gen_interval(&g, &lo, &hi);
  const double c = 0.5 * (lo + hi), gamma = 0.25 * (hi - lo);
  if (!(gamma > 0.0)) { /* scalar K: exp(-i[[c, H],[0, c]]) = e^{-ic} [[1, -iH],[0, 1]] */
    double complex ph = cexp(-I * c);
    orc_apply_term(p, kd, b, g.u1);
    for (int64_t i = 0; i < D; i++) { a[i] = ph * (a[i] - I * g.u1[i]); b[i] = ph * b[i]; }
    gen_free(&g);
    return ORC_OK;
  }
  int s = (int)ceil(gamma / p->rho_max);
  if (s < 1) s = 1;
  double complex *d = (double complex *)malloc(sizeof(double complex) * (size_t)(p->m_max + 1));
  double complex *wa = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double complex *wb = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double complex *ka = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double complex *kb = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double complex *pa = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double complex *pb = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  if (!d || !wa || !wb || !ka || !kb || !pa || !pb) rc = ORC_ENOMEM;
  if (rc == ORC_OK) orc_divided_differences(p->m_max, p->xi, gamma / s, d);
  const double complex phase = cexp(-I * c / s);
  for (int sub = 0; sub < s && rc == ORC_OK; sub++) {
    for (int64_t i = 0; i < D; i++) { wa[i] = a[i]; wb[i] = b[i]; pa[i] = d[0] * a[i]; pb[i] = d[0] * b[i]; }
    double e_prev = cabs(d[0]) * sqrt(creal(vnorm(wa, D) * vnorm(wa, D) + vnorm(wb, D) * vnorm(wb, D)));
    int conv = 0, m = 0;
    for (int j = 1; j <= p->m_max; j++) {
      /* K_aug [wa; wb] = [K wa + H_kd wb; K wb] */
      gen_apply(&g, wa, ka);
      gen_apply(&g, wb, kb);
      orc_apply_term(p, kd, wb, g.u1);
      if (st) st->n_matvec++;
      for (int64_t i = 0; i < D; i++) {
        double complex na = (ka[i] + g.u1[i] - c * wa[i]) / gamma - p->xi[j - 1] * wa[i];
        double complex nb = (kb[i] - c * wb[i]) / gamma - p->xi[j - 1] * wb[i];
        wa[i] = na;
        wb[i] = nb;
        pa[i] += d[j] * wa[i];
        pb[i] += d[j] * wb[i];
      }
      double nw2 = vnorm(wa, D) * vnorm(wa, D) + vnorm(wb, D) * vnorm(wb, D);
      double np2 = vnorm(pa, D) * vnorm(pa, D) + vnorm(pb, D) * vnorm(pb, D);
      double e = cabs(d[j]) * sqrt(nw2), pn = sqrt(np2);
      if (!isfinite(e) || !isfinite(pn)) { rc = ORC_ENONFINITE; break; }
      if (e + e_prev <= p->tol_abs + p->tol_rel * pn) { conv = 1; m = j; break; }
      e_prev = e;
    }
    if (rc == ORC_OK && !conv) rc = ORC_ENOCONV;
    if (st) {
      st->n_substeps++;
      if (m > st->max_m) st->max_m = m;
    }
    for (int64_t i = 0; i < D; i++) { a[i] = phase * pa[i]; b[i] = phase * pb[i]; }
  }
  if (st) st->n_exp++;
  free(d); free(wa); free(wb); free(ka); free(kb); free(pa); free(pb);
  gen_free(&g);
  return rc;
}

int orc_frechet_expv(const orc_problem *p, const double *beta, int kd, const double complex *v, double complex *a,
                     double complex *b, orc_stats *st) {
  int rc = check_problem(p);
  if (rc) return rc;
  if (kd < 0 || kd >= p->nterms) return ORC_EINVAL;
  for (int64_t i = 0; i < p->dim; i++) { a[i] = 0.0; b[i] = v[i]; }
  return frechet_core(p, beta, kd, a, b, st);
}

/*
 * Commutator-free schedule of the exponentials of one step: for stage q (in application order)
 * the weights w[q][j] of A(t_n + c_j h); J nodes c[j].
 */
static int cf_schedule(int variant, int *nstage, int *J, double w[3][3], double c[3]) {
  const double r3 = sqrt(3.0), r15 = sqrt(15.0);
  if (variant == ORC_CF4) {
    const double a1 = (3.0 - 2.0 * r3) / 12.0, a2 = (3.0 + 2.0 * r3) / 12.0;
    *nstage = 2; *J = 2;
    c[0] = 0.5 - r3 / 6.0; c[1] = 0.5 + r3 / 6.0;
    w[0][0] = a2; w[0][1] = a1;   /* right factor, applied first */
    w[1][0] = a1; w[1][1] = a2;
    return ORC_OK;
  }
  if (variant == ORC_CF4_3) {
    const double al[3][3] = {
        {37.0 / 240.0 - 10.0 * r15 / 261.0, -1.0 / 30.0, 37.0 / 240.0 + 10.0 * r15 / 261.0},
        {-11.0 / 360.0, 23.0 / 45.0, -11.0 / 360.0},
        {37.0 / 240.0 + 10.0 * r15 / 261.0, -1.0 / 30.0, 37.0 / 240.0 - 10.0 * r15 / 261.0}};
    *nstage = 3; *J = 3;
    c[0] = 0.5 - r15 / 10.0; c[1] = 0.5; c[2] = 0.5 + r15 / 10.0;
    for (int q = 0; q < 3; q++)
      for (int j = 0; j < 3; j++) w[q][j] = al[2 - q][j];
    return ORC_OK;
  }
  if (variant == ORC_M2) {
    *nstage = 1; *J = 1;
    c[0] = 0.5;
    w[0][0] = 1.0;
    return ORC_OK;
  }
  return ORC_EINVAL;
}

/*
 * F = |z|^2, z = <phi, psi_T> = phi^H U_M ... U_1 psi0 with U_e = exp(-i K_e) the exponentials in
 * application order.  dz/dc = sum_e (d beta_{kd,e} / dc) <lambda_e, L(Omega_e, -i H_kd) v_e> with
 * v_e the state before exponential e and lambda_e = U_{e+1}^H ... U_M^H phi the costate after it
 * (propagated backward with exp(+i K) = exp(-i (-K))), and dF/dc = 2 Re(conj(z) dz/dc).
 * All forward states are kept (no checkpointing: this is the plain reference).
 */
int orc_adjoint_grad(const orc_problem *p, const double complex *psi0, const double complex *phi, double t0,
                     double h, int64_t nsteps, int variant, int kd, double *F, double *grad) {
  int rc = check_problem(p);
  if (rc) return rc;
  int nstage, J;
  double w[3][3], c[3];
  if (cf_schedule(variant, &nstage, &J, w, c) != ORC_OK || kd < 0 || kd >= p->nterms || nsteps < 0) return ORC_EINVAL;
  const int64_t D = p->dim, nexp = nsteps * nstage;
  const int nm = p->coeff[kd].nmodes, ng = 1 + 2 * nm;
  double complex *states = (double complex *)malloc(sizeof(double complex) * (size_t)(nexp + 1) * (size_t)D);
  double *betas = (double *)malloc(sizeof(double) * (size_t)(nexp > 0 ? nexp : 1) * MAX_TERMS);
  double *dbeta = (double *)malloc(sizeof(double) * (size_t)(nexp > 0 ? nexp : 1) * (size_t)ng);
  double complex *lam = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double complex *fa = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double complex *fb = (double complex *)malloc(sizeof(double complex) * (size_t)D);
  double complex *dz = (double complex *)calloc((size_t)ng, sizeof(double complex));
  if (!states || !betas || !dbeta || !lam || !fa || !fb || !dz) rc = ORC_ENOMEM;
  /* weights of every exponential and their derivatives with respect to the coefficients of term kd */
  for (int64_t n = 0; n < nsteps && rc == ORC_OK; n++) {
    const double tn = t0 + (double)n * h;
    for (int q = 0; q < nstage; q++) {
      const int64_t e = n * nstage + q;
      for (int k = 0; k < p->nterms; k++) {
        double sacc = 0.0;
        for (int j = 0; j < J; j++) sacc += w[q][j] * orc_coeff_eval(p, k, tn + c[j] * h);
        betas[e * MAX_TERMS + k] = h * sacc;
      }
      const orc_coeff *cf = &p->coeff[kd];
      double s0 = 0.0;
      for (int j = 0; j < J; j++) s0 += w[q][j];
      dbeta[e * ng] = h * s0;
      for (int m = 0; m < nm; m++) {
        double sc = 0.0, ss = 0.0;
        for (int j = 0; j < J; j++) {
          sc += w[q][j] * cos(cf->om[m] * (tn + c[j] * h));
          ss += w[q][j] * sin(cf->om[m] * (tn + c[j] * h));
        }
        dbeta[e * ng + 1 + m] = h * sc;
        dbeta[e * ng + 1 + nm + m] = h * ss;
      }
    }
  }
  /* forward, keeping every state */
  if (rc == ORC_OK) memcpy(states, psi0, sizeof(double complex) * (size_t)D);
  for (int64_t e = 0; e < nexp && rc == ORC_OK; e++) {
    memcpy(states + (e + 1) * D, states + e * D, sizeof(double complex) * (size_t)D);
    rc = orc_expv(p, betas + e * MAX_TERMS, states + (e + 1) * D, NULL);
  }
  double complex z = 0.0;
  if (rc == ORC_OK) {
    for (int64_t i = 0; i < D; i++) z += conj(phi[i]) * states[nexp * D + i];
    memcpy(lam, phi, sizeof(double complex) * (size_t)D);
  }
  /* backward */
  double negb[MAX_TERMS];
  for (int64_t e = nexp - 1; e >= 0 && rc == ORC_OK; e--) {
    rc = orc_frechet_expv(p, betas + e * MAX_TERMS, kd, states + e * D, fa, fb, NULL);
    if (rc) break;
    double complex Ge = 0.0;
    for (int64_t i = 0; i < D; i++) Ge += conj(lam[i]) * fa[i];
    for (int q = 0; q < ng; q++) dz[q] += dbeta[e * ng + q] * Ge;
    for (int k = 0; k < p->nterms; k++) negb[k] = -betas[e * MAX_TERMS + k];
    rc = orc_expv(p, negb, lam, NULL);
  }
  if (rc == ORC_OK) {
    *F = creal(z) * creal(z) + cimag(z) * cimag(z);
    for (int q = 0; q < ng; q++) grad[q] = 2.0 * creal(conj(z) * dz[q]);
  }
  free(states); free(betas); free(dbeta); free(lam); free(fa); free(fb); free(dz);
  return rc;
}
