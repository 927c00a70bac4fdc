/*
 * magnus.h -- C ABI of the GB300 (sm_103a) Magnus + Leja library.
 *
 * Computes the solution of the Schroedinger equation i psi' = H(t) psi with a
 * time-dependent Hamiltonian H(t) = sum_k f_k(t) H_k (arXiv:1709.06483, Sec. 1,
 * Eq. (1), and the split H = H_1 + h(t) H_2 of Sec. 4) by fourth-order Magnus
 * integrators (Sec. 2: Method M4 with its commutator applied matrix-free as
 * H_2(H_1 psi) - H_1(H_2 psi), and the commutator-free Method Cf4; also Cf4:3 and
 * the exponential midpoint rule M2), whose exponentials exp(-i K) psi are applied
 * by Newton-form Leja interpolation (Sec. 3) entirely on one GPU.
 *
 * Conventions (all entry points):
 *  - Every function returns a magnus_status; none aborts, none throws.
 *  - "device" pointers are CUDA global-memory pointers on the plan's device;
 *    "host" pointers are ordinary CPU memory.
 *  - Complex numbers are interleaved (re, im) FP64 pairs (CUDA double2 layout,
 *    16-byte aligned), passed as void* so this header needs no CUDA include.
 *  - A state vector psi of a plan with nvec vectors is stored [nvec][dim].
 *  - Work is issued on the plan's stream.  magnus_propagate and leja_expv
 *    synchronise that stream before they return, so that their status is final.
 *  - The plan BORROWS the term matrices (CSR arrays, dense matrices): they must
 *    stay valid and unchanged while the plan exists.  Coefficient arrays and the
 *    spin-chain parameters are copied at creation.  The plan owns its scratch.
 */
#ifndef MAGNUS_H
#define MAGNUS_H

#include <stdint.h>

#if defined(__GNUC__)
#define MAGNUS_API __attribute__((visibility("default")))
#else
#define MAGNUS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MAGNUS_OK = 0,
  MAGNUS_EINVAL = 1,     /* invalid argument; nothing was launched                       */
  MAGNUS_ENOMEM = 2,     /* device allocation failed                                     */
  MAGNUS_ECUDA = 3,      /* a CUDA call failed (see magnus_last_error)                   */
  MAGNUS_ENOCONV = 4,    /* a Leja polynomial reached m_max without meeting the tolerance */
  MAGNUS_ENONFINITE = 5, /* a norm became NaN or Inf                                     */
  MAGNUS_ETIMEOUT = 6,   /* a device-side wait gave up (bounded spin)                     */
  MAGNUS_EDRIFT = 7      /* a substep changed the state's norm by more than options.norm_check
                            allows (exp(-i tau K) of a Hermitian K keeps the norm)         */
} magnus_status;

typedef enum {
  MAGNUS_M4 = 1,   /* Sec. 2, Method M4 (commutator applied matrix-free)        */
  MAGNUS_CF4 = 2,  /* Sec. 2, Method Cf4 (two exponentials)                     */
  MAGNUS_CF4_3 = 3,/* Sec. 2, Method Cf4:3 (three exponentials)                 */
  MAGNUS_M2 = 4,   /* Sec. 2, Method M2 (exponential midpoint rule)             */
  MAGNUS_M6 = 5    /* Sec. 2, Method M6 (order six, nested commutators applied
                      matrix-free; CSR and matrix-free terms, not dense terms or
                      batches).  The weight of B_3 is 1/12: with it B_1 + B_3/12
                      is the 3-point Gauss rule the first Magnus term needs.    */
} magnus_variant;

typedef enum {
  MAGNUS_TERM_CSR = 0,     /* complex128 CSR, row-major, int64 row pointers, int32 columns (Sec. 3, CSR) */
  MAGNUS_TERM_DENSE = 1,   /* complex128 dense dim x dim, row-major                                      */
  MAGNUS_TERM_XXZ = 2,     /* matrix-free open XXZ chain (Sec. 4, Pauli/Kronecker embedding)              */
  MAGNUS_TERM_FIELD_X = 3, /* matrix-free transverse field sum_i sigma^x_i                                */
  MAGNUS_TERM_CSR_REAL = 4,  /* real symmetric CSR: float64 values (12 B per entry instead of 20)           */
  MAGNUS_TERM_DENSE_REAL = 5 /* real symmetric dense dim x dim, float64, row-major (8 B per element)        */
} magnus_term_kind;

typedef enum {
  MAGNUS_FP64 = 0,       /* plain FP64 matvecs                                                     */
  MAGNUS_FP32_SPLIT = 1,   /* dense terms: FP32 (hi, lo) split matvecs, FP64 accumulation          */
  MAGNUS_TENSOR_SLICED = 2 /* dense terms: exact bf16 digit products on the tensor cores           */
} magnus_precision;

/*
 * One stored term H_k.  Spin index convention (MAGNUS_TERM_XXZ / FIELD_X and
 * the builders below): for n spins, spin j (1-based) is bit (n - j) of the basis
 * index, i.e. spin 1 is the leftmost Kronecker factor (Sec. 4).
 *   CSR:     rowptr[dim+1] (device, int64), col[nnz] (device, int32), val[nnz] (device, complex128).
 *            Rows may list their columns in any order, without duplicates.
 *   DENSE:   val[dim*dim] (device, complex128, row-major).
 *   CSR_REAL, DENSE_REAL: as CSR / DENSE with val holding float64 real values (8-byte aligned); the
 *            matrix must be real symmetric.  Every Hamiltonian of the paper's Sec. 4 is real, so this
 *            storage reads 12 B per CSR entry and 8 B per dense element and gives the same results
 *            as the complex storage of the same matrix.
 *   XXZ:     sum_{i=1}^{n-1} J_i (sx_i sx_{i+1} + sy_i sy_{i+1} + delta sz_i sz_{i+1}) + sum_i hz_i sz_i,
 *            J[n-1], hz[n] on the HOST (copied); dim must be 2^nspins.
 *   FIELD_X: sum_{i=1}^{n} sx_i; dim must be 2^nspins.
 * Every term must be Hermitian (the spectral enclosure assumes it).
 */
typedef struct {
  int32_t kind;
  int32_t nspins;
  int64_t nnz;
  const int64_t *rowptr;
  const int32_t *col;
  const void *val;
  const double *J;
  const double *hz;
  double delta;
} magnus_term;

/*
 * out[e] = Re z[e] for e < n (z: device complex128, out: device float64, both caller-owned), on
 * `stream`; synchronises the stream.  Returns MAGNUS_EINVAL (out still written) if some Im z[e] != 0,
 * so a complex-stored real matrix converts to MAGNUS_TERM_CSR_REAL / DENSE_REAL storage exactly
 * (every Hamiltonian of Sec. 4 is real).  Also EINVAL for n < 0 or a null pointer; ENOMEM, ECUDA.
 */
MAGNUS_API magnus_status magnus_real_parts(const void *z, int64_t n, double *out, void *stream);

/* f_k(t) = a0 + sum_{m<nmodes} (ac[m] cos(om[m] t) + as[m] sin(om[m] t)); host arrays, copied. */
typedef struct {
  double a0;
  int32_t nmodes;
  int32_t _pad;
  const double *ac;
  const double *as;
  const double *om;
} magnus_coeff;

typedef enum {
  MAGNUS_INTERVAL_GERSHGORIN = 0, /* Gershgorin enclosure of every term (rigorous)                       */
  MAGNUS_INTERVAL_LANCZOS = 1     /* 48 Lanczos steps per term from a fixed start vector: Ritz extremes
                                     widened by their residual norms and 1 % of the width, intersected
                                     with Gershgorin (tighter, so lower Leja degrees)                     */
} magnus_interval;

/*
 * Options; pass NULL for the defaults in brackets.
 *   tol_rel, tol_abs [1e-10, 1e-10]: Leja early termination (Sec. 4: relative and absolute tolerance 1e-10)
 *   rho_max [4.0]: largest scaled step gamma/s per Leja polynomial (substepping)
 *   m_max [100]:  largest Leja degree per substep (at most 255)
 *   nvec [1]:     number of state vectors propagated together
 *   ctas [0]:     CTAs of the persistent kernel (0 = automatic)
 *   precision [MAGNUS_FP64]: arithmetic of the dense-term matvecs.  MAGNUS_FP32_SPLIT and
 *                     MAGNUS_TENSOR_SLICED need real-valued dense terms (the drive may add
 *                     MAGNUS_TERM_FIELD_X terms); MAGNUS_TENSOR_SLICED also needs dim a multiple of
 *                     128.  MAGNUS_TENSOR_SLICED cuts every dense row (row scale 2^e_r) and every
 *                     state component column (scale 2^e_c) into signed digits and forms their
 *                     products exactly on the bf16 tensor cores, summing them in FP32 (exact within
 *                     a chunk of K) and int64, on tcgen05: values scaled to 31 bits, 4 digits of at
 *                     most 128 in magnitude, the 10 digit pairs of level <= 3, chunks of 512 K;
 *                     neglected part of one output entry below dim * 2^-29 * max_j |H_rj| *
 *                     max_j |w_j|.  Every generator: M2, CF4, CF4:3 one product phase per Leja
 *                     iteration; M4 one for u_k = H_k w and one per commutator pair (H_k u_l and
 *                     H_l u_k from the digits of u_l and u_k).  (Not part of the paper, which
 *                     computes in FP64 only.)
 *   barrier_timeout_s [0 = 4 s]: limit of every device-side wait at a grid barrier; a wait that runs
 *                     out makes the call return MAGNUS_ETIMEOUT and leaves the context usable
 *   test_skip_arrival [0]: testing only -- if nonzero, CTA 0 of the sparse/matrix-free propagation
 *                     kernel leaves before its first grid barrier, so the other CTAs' waits run out
 *   interval [MAGNUS_INTERVAL_GERSHGORIN]: how each term's spectral enclosure is estimated (Sec. 3:
 *                     the Leja parameters need a spectral estimate); plans only, batches
 *                     take Gershgorin
 *   fixed_sums [1]:   fixed-point arithmetic on a copy Z of each Leja vector in int64 pairs, scaled
 *                     from a bound on its largest component (truncation below 2^-55 of that bound
 *                     per component for rows of up to 32 entries): the rows of pattern terms (real
 *                     CSR terms whose stored values are all equal, v sum_e x[col_e], and
 *                     MAGNUS_TERM_FIELD_X next to MAGNUS_TERM_XXZ) are summed exactly in int64;
 *                     the other real CSR terms multiply row-scaled 62-bit mantissas of their values
 *                     by Z (high 64 bits of each product, summed exactly), and the XXZ bond flips
 *                     their weights likewise.  Plans with only CSR terms or the matrix-free chain,
 *                     generators M2, CF4, CF4:3 and M4 (M6 keeps FP64) and magnus_apply; batches:
 *                     M2, CF4, CF4:3.  The scale follows the vector across the whole double range;
 *                     a converted result below 2^-1022 flushes to zero (FP64 would keep a
 *                     subnormal).  0 = FP64 throughout.  Not part of the paper, which computes in
 *                     FP64 only.
 *   row_layout [MAGNUS_ROWS_AUTO]: how the rows of fixed-point CSR plans (every term CSR, fixed_sums)
 *                     read the pattern and product terms; the integer row sums make every layout give
 *                     the same bits.  MAGNUS_ROWS_CSR (the default) -- the CSR arrays as given, a
 *                     row per thread; MAGNUS_ROWS_SLICED -- plan-owned copies cut into 32-row slices:
 *                     the first w entries of every row column-major (w = the slice's shortest row),
 *                     ordered so that rows sharing a column offset read it at the same position, the
 *                     rest row-major (same bytes per entry); MAGNUS_ROWS_STAGED -- those slices
 *                     copied into shared memory two tiles ahead by the TMA bulk engine (two CTAs of 8
 *                     warps per SM; plans of at most two terms; a tile larger than a 6,400-byte slot
 *                     is read from global memory, and a plan stages only if at most 1/64 of its
 *                     tiles are such).
 *   plain_values [0]: 1 = multiply complex-stored CSR and dense values in place as complex128 numbers
 *                     even when every imaginary part is zero (no real-valued specialisation, no
 *                     float64 copy, no pattern or fixed-point rows): the plain FP64 path of the paper,
 *                     kept as the baseline the faster paths are measured against.  Real storage
 *                     (MAGNUS_TERM_*_REAL) is unaffected.  _reserved must be 0.
 *   norm_check [0 = off]: a posteriori check of every substep (plans; batches do not check).  The
 *                     Leja parameters come from a spectral interval; Gershgorin encloses the
 *                     spectrum, the Lanczos interval (MAGNUS_INTERVAL_LANCZOS) does not prove it.
 *                     Every exponential of a Hermitian generator keeps the norm, so a substep whose
 *                     | ||p|| - ||v|| | exceeds norm_check * (tol_abs + tol_rel ||v||) + 1e-13 ||v||
 *                     ends the call with MAGNUS_EDRIFT (p the substep's result, v its input).  The
 *                     largest relative drift is reported in magnus_stats.norm_drift either way.
 */
typedef enum {
  MAGNUS_ROWS_AUTO = 0,   /* the library's choice (MAGNUS_ROWS_CSR) */
  MAGNUS_ROWS_STAGED = 1,
  MAGNUS_ROWS_CSR = 2,
  MAGNUS_ROWS_SLICED = 3
} magnus_row_layout;

typedef struct {
  double tol_rel;
  double tol_abs;
  double rho_max;
  int32_t m_max;
  int32_t nvec;
  int32_t ctas;
  int32_t precision;
  double barrier_timeout_s;
  int32_t test_skip_arrival;
  int32_t interval;
  int32_t fixed_sums;
  int32_t row_layout;
  int32_t plain_values;
  int32_t _reserved;
  double norm_check;
} magnus_options;

typedef struct {
  int64_t n_exp;        /* exponentials applied                               */
  int64_t n_substeps;   /* Leja polynomials evaluated                         */
  int64_t n_matvec;     /* Leja iterations (one application of K each)       */
  int64_t n_termapply;  /* applications of a single stored term H_k          */
  int32_t max_m;        /* largest Leja degree used                           */
  int32_t status;       /* magnus_status of the call                          */
  int32_t *m_log;       /* optional HOST array: degree of every substep       */
  int64_t m_log_cap;    /* its capacity (entries)                             */
  double kernel_ms;     /* device time of the persistent Leja kernel (CUDA events on the plan's stream) */
  int32_t grid;         /* CTAs of that launch                                */
  int32_t block;        /* threads per CTA                                    */
  int32_t fixed_sums;   /* 1 if the call's matvecs ran in fixed point (options.fixed_sums)      */
  int32_t row_layout;   /* the fixed-point CSR rows' layout (magnus_row_layout; 0: not such a call) */
  double norm_drift;    /* largest | ||p|| - ||v|| | / ||v|| over the call's substeps and states (p the
                           substep's result, v its input): 0 up to rounding and the Leja tolerance */
} magnus_stats;

typedef struct magnus_plan_s *magnus_plan_t;

/*
 * Create a plan for dim x dim terms H_0..H_{nterms-1} (nterms <= 4) with
 * coefficient functions coeffs[k], on the current CUDA device and the given
 * stream (a cudaStream_t; NULL = the legacy default stream).  Computes on the
 * device, once: the Leja points on [-2,2] (Sec. 3) and the Gershgorin enclosure
 * [a_k, b_k] of every term's spectrum (Sec. 3, the spectrum estimate the Leja
 * parameters need).  Errors: EINVAL (bad sizes, null pointers, dim not 2^nspins
 * for matrix-free terms), ENOMEM, ECUDA.  *plan is NULL on error.
 */
MAGNUS_API magnus_status magnus_plan_create(magnus_plan_t *plan, int64_t dim, int32_t nterms, const magnus_term *terms,
                                 const magnus_coeff *coeffs, const magnus_options *opt, void *stream);

/* Release the plan and its scratch (after synchronising its stream).  NULL is accepted. */
MAGNUS_API magnus_status magnus_plan_destroy(magnus_plan_t plan);

/* Human-readable description of the last error of this plan ("" if none); plan may be NULL. */
MAGNUS_API const char *magnus_last_error(magnus_plan_t plan);

/* Static name of a status code. */
MAGNUS_API const char *magnus_status_string(magnus_status s);

/*
 * out = exp(-i sum_k beta[k] H_k) v for every one of the plan's nvec vectors
 * (Sec. 3, Newton-form Leja interpolation with early termination).
 * beta: host, nterms reals (the step size is part of beta).
 * v, out: device complex128 [nvec][dim]; may be the same buffer.
 * Errors: EINVAL, ENOCONV, ENONFINITE, ETIMEOUT, ECUDA.
 */
MAGNUS_API magnus_status leja_expv(magnus_plan_t plan, const double *beta, const void *v, void *out, magnus_stats *stats);

/*
 * psi <- Y_{n0+nsteps}: nsteps Magnus steps of size h from t0 (Sec. 2, Eq. (9):
 * Y_{n+1} = exp(Omega_n) Y_n, with t_n = t0 + n h).  psi: device complex128
 * [nvec][dim], in/out.  variant: magnus_variant.  The whole propagation runs in
 * one persistent launch; the only host synchronisation is at the end.
 * Errors: EINVAL, ENOCONV, ENONFINITE, ETIMEOUT, ECUDA.  On error psi holds the
 * state after the last completed exponential.
 */
MAGNUS_API magnus_status magnus_propagate(magnus_plan_t plan, void *psi, double t0, double h, int64_t nsteps,
                               int32_t variant, magnus_stats *stats);

/*
 * Adjoint gradient (no counterpart computed in the paper; built on its Sec. 2 stepping and Sec. 3
 * Leja interpolation).  With psi(T) = nsteps commutator-free steps (MAGNUS_CF4, MAGNUS_CF4_3 or
 * MAGNUS_M2) from psi0 at t0, F = |<phi|psi(T)>|^2 (written to *F) and its gradient with respect to
 * the drive coefficients of term kd: grad[0] = dF/da0, grad[1+m] = dF/dac[m], grad[1+nmodes+m] =
 * dF/das[m] (HOST array of 1 + 2 nmodes doubles).  Each exponential is differentiated through the
 * augmented block matrix [[Omega, -i H_kd], [0, Omega]] with the same Leja kernels, the costate is
 * propagated with exp(+iK), and psi is checkpointed every ckpt_every steps and recomputed segment by
 * segment.  psi0, phi: device complex128 [dim].  Plans with nvec = 1 and CSR / matrix-free terms.
 * Errors: EINVAL, ENOMEM, ENOCONV, ENONFINITE, ETIMEOUT, ECUDA.
 */
MAGNUS_API magnus_status magnus_adjoint_grad(magnus_plan_t plan, const void *psi0, const void *phi, double t0, double h,
                                             int64_t nsteps, int32_t variant, int32_t kd, int32_t ckpt_every, double *F,
                                             double *grad, magnus_stats *stats);

/*
 * Replace the drive coefficient f_k of term k (the time dependence h(t) of the split
 * H = H_1 + h(t) H_2 of Sec. 4; host struct, copied): the next calls on the plan use
 * it (stream-ordered).  The spectral enclosures are those of the terms and do not change.
 * Errors: EINVAL, ECUDA.
 */
MAGNUS_API magnus_status magnus_set_coeff(magnus_plan_t plan, int32_t k, const magnus_coeff *c);

/*
 * y = sum_k beta_k H_k x for every state: the generator matvec of the Leja recurrence (Sec. 3, the
 * operation the method's cost is made of), as a call of its own (expectation values, timing).
 * beta: host, nterms reals.  x, y: device complex128 [nvec][dim], distinct, 16-byte aligned.
 * Plans with fixed_sums (CSR with a pattern or real term, matrix-free chains) take the rows as the
 * Leja iteration does: the plan's fixed-point copy of x (one scale per state, from max |x|), exact
 * integer row sums and value products, one rounding back to FP64 per row and term; a state holding
 * an Inf or NaN takes the FP64 rows.  Three launches then, one otherwise; the plan's copy buffers
 * are in use until they finish (stream-ordered).
 * Asynchronous on the plan's stream (no synchronisation).  Errors: EINVAL, ECUDA.
 */
MAGNUS_API magnus_status magnus_apply(magnus_plan_t plan, const double *beta, const void *x, void *y);

/* Spectral enclosure [*a, *b] of term k (computed at plan creation: Gershgorin, or its
 * intersection with the Lanczos enclosure), the estimate the Leja parameters of Sec. 3 are built
 * on.  a, b: host.  Errors: EINVAL (null plan or pointer, k out of range). */
MAGNUS_API magnus_status magnus_term_interval(magnus_plan_t plan, int32_t k, double *a, double *b);

/* Copy the first count (<= m_max+1) of the plan's Leja points on [-2,2] (Sec. 3, the
 * interpolation nodes; device-computed) to host xi[].  Synchronises the plan's stream.
 * Errors: EINVAL (null plan or pointer, count out of range), ECUDA. */
MAGNUS_API magnus_status magnus_leja_points(magnus_plan_t plan, double *xi, int32_t count);

/*
 * Divided differences d_j = g[xi_0..xi_j], j = 0..count-1, of g(x) = exp(-i rho x)
 * at the plan's Leja points (Sec. 3), computed on the device; d: host complex128[count].
 * Synchronises the plan's stream.  Errors: EINVAL (count out of range, rho < 0 or NaN), ENOMEM, ECUDA.
 */
MAGNUS_API magnus_status magnus_divided_differences(magnus_plan_t plan, double rho, void *d, int32_t count);

/* ---- Hamiltonian builders (device kernels; all pointers device unless noted) ----
 * The spin chains of Sec. 4 from the Pauli matrices in the Kronecker embedding (spin 1 leftmost).
 * Each builder enqueues its kernel on `stream` and returns without synchronising.
 * Errors: EINVAL (nspins out of range, null pointer), ECUDA (launch failure); the text is in
 * magnus_last_error(NULL). */

/* Number of stored entries of the XXZ CSR built below: 2^n + (n-1) 2^(n-1); -1 for nspins outside
 * 2..30. */
MAGNUS_API int64_t magnus_xxz_nnz(int32_t nspins);

/*
 * Open XXZ chain (as MAGNUS_TERM_XXZ) as CSR: per row the diagonal and one entry per
 * anti-parallel bond (value 2 J_i), columns ascending.  J, hz: HOST.  rowptr[2^n+1],
 * col[nnz], val[nnz] device.  stream: cudaStream_t or NULL.
 */
MAGNUS_API magnus_status magnus_build_xxz_csr(int32_t nspins, const double *J, const double *hz, double delta,
                                   int64_t *rowptr, int32_t *col, void *val, void *stream);

/* sum_i sigma^x_i as CSR: N entries of value 1 per row, columns ascending; nnz = n 2^n. */
MAGNUS_API magnus_status magnus_build_field_x_csr(int32_t nspins, int64_t *rowptr, int32_t *col, void *val, void *stream);

/*
 * Long-range chain, dense: sum_{i<j} (sx_i sx_j + sy_i sy_j + delta sz_i sz_j)/|i-j|^alpha + sum_i hz_i sz_i.
 * hz: HOST.  H: device complex128 [2^n][2^n].
 */
MAGNUS_API magnus_status magnus_build_longrange_dense(int32_t nspins, double alpha, const double *hz, double delta, void *H,
                                           void *stream);

/* sum_i sigma^x_i, dense. */
MAGNUS_API magnus_status magnus_build_field_x_dense(int32_t nspins, void *H, void *stream);

/* ---- batches of independent problems ---- */

/* One problem of a batch: a state of dimension dim under terms[nterms] with coeffs[nterms] (as in
 * magnus_plan_create; CSR, XXZ or FIELD_X terms; the CSR arrays are borrowed). */
typedef struct {
  int64_t dim;
  int32_t nterms;
  int32_t _pad;
  const magnus_term *terms;
  const magnus_coeff *coeffs;
} magnus_batch_item;

typedef struct {
  int64_t n_exp, n_substeps, n_matvec, n_termapply; /* summed over all problems                  */
  int32_t max_m;
  int32_t status;
  int32_t *m_log;               /* optional HOST [count][m_log_cap_per_item]: Leja degree per substep */
  int64_t m_log_cap_per_item;
  double graph_ms;              /* device time of the replayed graph (setup + persistent kernel)    */
  int32_t block;                /* CTA size the autotuner chose                                     */
  int32_t cluster;              /* CTAs per thread-block cluster (one problem per cluster)          */
  int32_t fixed_sums;           /* 1 if the matvecs ran in fixed point (options.fixed_sums)         */
  int32_t _pad;
} magnus_batch_stats;

typedef struct magnus_batch_s *magnus_batch_t;

/*
 * A batch of count independent problems (arXiv:1709.06483 Sec. 2 stepping with Sec. 3 Leja
 * interpolation applied to each) that magnus_batch_propagate advances together in ONE persistent
 * launch: every CTA takes whole problems from a work queue, largest first, and synchronises only
 * within itself.  Computes, once, the Gershgorin enclosure of every term and the Leja points.
 * opt: as for plans, with nvec = 1 (one state per problem) and precision MAGNUS_FP64; ctas > 0
 * caps the CTAs; ctas < 0 replaces the autotuner: -ctas = bs + 65536 * cs forces the CTA size bs
 * (128, 256, 512 or 1024) and the cluster size cs (1, 2 or 4; 0 means 1).
 * Each problem runs on one thread-block cluster of cs CTAs that split its rows.
 * The batch uses its own CUDA stream (the stream argument is ignored).  Errors: EINVAL, ENOMEM, ECUDA.
 */
MAGNUS_API magnus_status magnus_batch_create(magnus_batch_t *batch, int32_t count, const magnus_batch_item *items,
                                             const magnus_options *opt, void *stream);

/*
 * psi[i] (device complex128 [dim_i], in/out; psi is a HOST array of count device pointers) <- nsteps
 * Magnus steps of size h from t0 for every problem (Sec. 2, Eq. (9), each exponential by the
 * Leja interpolation of Sec. 3).  The first call times the candidate CTA sizes
 * x cluster sizes on copies of the states (2 steps each) and keeps the fastest; the setup launches and the persistent
 * kernel are captured into a CUDA graph once per (t0, h, nsteps, variant) and replayed.  Synchronous.
 * Errors: EINVAL, ENOCONV, ENONFINITE, ECUDA (the first error of any problem).
 */
MAGNUS_API magnus_status magnus_batch_propagate(magnus_batch_t batch, void *const *psi, double t0, double h,
                                                int64_t nsteps, int32_t variant, magnus_batch_stats *stats);

/* Release the batch, its graph and its scratch.  NULL is accepted.  Returns MAGNUS_OK. */
MAGNUS_API magnus_status magnus_batch_destroy(magnus_batch_t batch);

/* Last error of this batch ("" if none); NULL gives the last error of magnus_batch_create. */
MAGNUS_API const char *magnus_batch_last_error(magnus_batch_t batch);

/* ---- allocation-free entry point ---- */

/*
 * out = exp(-i (beta[0] H_xxz + beta[1] sum_i sigma^x_i)) v for the matrix-free open XXZ chain
 * (H_xxz as MAGNUS_TERM_XXZ: J[nspins-1], hz[nspins] on the HOST, anisotropy delta), Leja
 * tolerance tol (relative and absolute), without a plan and without allocating memory.
 * The paper has no counterpart: this exists for callers that cannot call cudaMalloc -- code whose
 * device memory is entirely owned by another allocator or pool, or latency-sensitive loops that
 * must not pay the implicit synchronisation of cudaMalloc/cudaFree.
 *  - Scratch: one fixed device array of about 3.2 MB inside the library, held by every GPU that
 *    loads the library until the process exits.  Maximum size: nspins <= 16 (dim <= 65536);
 *    larger chains return MAGNUS_EINVAL ("nspins must be 2..16").
 *  - The first call on a device (with that device current) sets the device up: it resolves the
 *    array's device address and computes the Leja points into it, synchronising `stream`.  Make
 *    that first call before any stream capture.
 *  - Every call shares the one array and overwrites it; calls whose GPU work overlaps (other
 *    streams or threads on the same device) race and give wrong results.  Serialise them.
 *  - v, out: device complex128 [2^nspins], 16-byte aligned, may alias.  stream: cudaStream_t or
 *    NULL.  The call synchronises the stream before it returns.
 *  - Calls no cudaMalloc, cudaFree or other allocating routine.  Error text: magnus_last_error(NULL).
 *  - Arithmetic: FP64 sums and products throughout (the generic rows of the persistent kernel), where
 *    a plan defaults to fixed-point sums; results agree with leja_expv to the Leja tolerance.
 */
MAGNUS_API magnus_status magnus_expv_xxz_static(int32_t nspins, const double *J, const double *hz, double delta,
                                                const double *beta, const void *v, void *out, double tol,
                                                void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MAGNUS_H */
