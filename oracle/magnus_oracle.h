/*
 * magnus_oracle.h -- TEST INFRASTRUCTURE, not the product.
 *
 * Plain, slow FP64 CPU restatement of the method of Auer, Einkemmer, Kandolf and
 * Ostermann, "Magnus integrators on multicore CPUs and GPUs" (arXiv:1709.06483):
 * Magnus integrators (Sec. 2: Methods M2, M4, Cf4, Cf4:3) whose exponentials are
 * applied by Newton-form Leja interpolation (Sec. 3).  Only tests/, the smoke
 * check of __graft_entry__ and the CPU-baseline leg of bench.py may load it.  It
 * shares no code, header or table with the CUDA library.
 *
 * Complex numbers are C99 `double complex` (interleaved re,im: the numpy
 * complex128 layout).  All operator matrices are borrowed: the caller keeps them
 * alive while a problem refers to them.
 */
#ifndef MAGNUS_ORACLE_H
#define MAGNUS_ORACLE_H

#include <complex.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENOCONV = 4, ORC_ENONFINITE = 5 };
enum { ORC_TERM_CSR = 0, ORC_TERM_DENSE = 1 };
enum { ORC_M4 = 1, ORC_CF4 = 2, ORC_CF4_3 = 3, ORC_M2 = 4, ORC_M6 = 5 };

typedef struct {
  int64_t n_exp;       /* exponentials applied                                   */
  int64_t n_substeps;  /* Leja substeps (one polynomial each)                    */
  int64_t n_matvec;    /* applications of a generator K (one per Leja iteration) */
  int64_t n_termapply; /* applications of a single stored term H_k               */
  int32_t max_m;       /* largest Leja degree used                               */
  int32_t _pad;
  int32_t *m_log;      /* optional: degree of every substep, in order             */
  int64_t m_log_cap;   /* capacity of m_log                                       */
} orc_stats;

/* Leja points on [-2,2] (xi[0..m]), ties broken towards the larger x. */
int orc_leja_points(int m, double *xi);

/* d[j] = g[xi_0..xi_j] for g(x) = exp(-i*rho*x), j = 0..m (Opitz matrix). */
int orc_divided_differences(int m, const double *xi, double rho, double complex *d);

/* Spin-chain builders (spin 1 = most significant bit of the basis index). */
int64_t orc_xxz_nnz(int nspins, const double *J, double delta);
int orc_build_xxz_csr(int nspins, const double *J, const double *hz, double delta,
                      int64_t *rowptr, int32_t *col, double complex *val);
int orc_build_field_x_csr(int nspins, int64_t *rowptr, int32_t *col, double complex *val);
int orc_build_longrange_dense(int nspins, double alpha, const double *hz, double delta,
                              double complex *H);
int orc_build_field_x_dense(int nspins, double complex *H);

/* Problem: dim, nterms stored terms H_k, each with f_k(t) = a0 + sum_m (ac_m cos(om_m t) + as_m sin(om_m t)). */
typedef struct orc_problem orc_problem;
orc_problem *orc_problem_new(int64_t dim, int nterms);
void orc_problem_free(orc_problem *p);
int orc_set_csr(orc_problem *p, int k, const int64_t *rowptr, const int32_t *col, const double complex *val);
int orc_set_dense(orc_problem *p, int k, const double complex *H);
int orc_set_coeff(orc_problem *p, int k, double a0, int nmodes, const double *ac, const double *as,
                  const double *om);
int orc_set_leja(orc_problem *p, double tol_rel, double tol_abs, int m_max, double rho_max);
int orc_term_interval(const orc_problem *p, int k, double *a, double *b);
/* Replace term k's enclosure by the Lanczos enclosure (m steps) intersected with Gershgorin. */
int orc_set_interval_lanczos(orc_problem *p, int k, int m);
double orc_coeff_eval(const orc_problem *p, int k, double t);

/* y = H_k x */
int orc_apply_term(const orc_problem *p, int k, const double complex *x, double complex *y);

/* v <- exp(-i * sum_k beta_k H_k) v */
int orc_expv(const orc_problem *p, const double *beta, double complex *v, orc_stats *st);

/* psi <- product of nsteps Magnus steps of size h from t0 (variant ORC_M4 / ORC_CF4 / ORC_CF4_3 /
 * ORC_M2 / ORC_M6). */
int orc_propagate(const orc_problem *p, double complex *psi, double t0, double h, int64_t nsteps,
                  int variant, orc_stats *st);

/* [*a, *b]: the spectral enclosure of the generator K of one step of size h from tn of Method M4
 * or M6 (variant ORC_M4 / ORC_M6), the interval whose shift and scale that step's exponential uses. */
int orc_generator_interval(const orc_problem *p, int variant, double tn, double h, double *a, double *b);

/*
 * Frechet derivative of the exponential by the augmented block matrix:
 * [a; b] = exp(Omega_aug) [0; v] with Omega_aug = [[Omega, E], [0, Omega]], Omega = -i sum_k beta_k H_k,
 * E = -i H_kd.  Then a = L(Omega, E) v and b = exp(Omega) v.
 */
int orc_frechet_expv(const orc_problem *p, const double *beta, int kd, const double complex *v, double complex *a,
                     double complex *b, orc_stats *st);

/*
 * Gradient of F = |<phi|psi(T)>|^2, psi(T) = nsteps commutator-free steps (ORC_CF4, ORC_CF4_3 or
 * ORC_M2) from psi0, with respect to the drive coefficients of term kd:
 * grad[0] = dF/da0, grad[1+m] = dF/dac_m, grad[1+nmodes+m] = dF/das_m.  *F receives F.
 */
int orc_adjoint_grad(const orc_problem *p, const double complex *psi0, const double complex *phi, double t0,
                     double h, int64_t nsteps, int variant, int kd, double *F, double *grad);

#ifdef __cplusplus
}
#endif
#endif
