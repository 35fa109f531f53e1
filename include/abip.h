/*
 * abip.h -- C ABI of libabip, a GB300 (sm_103a) implementation of ABIP, the
 * ADMM-based interior-point method for linear programming of Lin, Ma, Ye and
 * Zhang (arXiv 1805.12344).
 *
 * Problem (Sec. 2, the primal-dual pair (P)/(D)):
 *     minimise c^T x  subject to  A x = b,  x >= 0,      A is m x n, m <= n,
 * with A of full row rank.  ABIP solves the homogeneous self-dual embedding of
 * this pair (Sec. 3.1, matrix Q) by path following on the log-barrier
 * subproblem, each barrier subproblem being solved inexactly by ADMM
 * (Algorithm 2, with the over-relaxation of Sec. 4.2).  Every step of the
 * solve runs in the library's own CUDA kernels on the current device.
 *
 * Conventions for every entry point:
 *   - Return value: ABIP_OK (0) or a negative ABIP_E_* code.  A handle keeps a
 *     message for the last failure (abip_last_error).
 *   - Pointers marked "host or device" may point to host memory or to memory of
 *     the current CUDA device; the library detects which.
 *   - The library copies every input it needs at setup; the caller keeps
 *     ownership of its arrays and may free them after the call returns.
 *   - Outputs are caller-allocated.
 *   - A handle must not be used by two host threads at once; distinct handles
 *     are independent.
 *   - Dense matrices are row-major with leading dimension ld >= n.  CSR uses
 *     int64 row pointers (m+1 entries, row_ptr[0] = 0) and int32 column indices
 *     that are in range; column order within a row is free.
 */
#ifndef ABIP_H
#define ABIP_H

#include <stdint.h>

#if defined(__GNUC__)
#define ABIP_API __attribute__((visibility("default")))
#else
#define ABIP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------------- */
#define ABIP_OK              0
#define ABIP_E_INVALID_ARG  -1   /* null pointer, bad enum, non-finite input, bad params */
#define ABIP_E_DIM          -2   /* m < 1, n < m, ld < n, malformed CSR */
#define ABIP_E_CUDA         -3   /* a CUDA runtime call failed (message kept) */
#define ABIP_E_OOM          -4   /* device allocation failed */
#define ABIP_E_NOT_SOLVED   -5   /* state requested before any solve */
#define ABIP_E_NUMERICAL    -6   /* Cholesky breakdown, non-finite value mid-solve, PCG failure */
#define ABIP_E_UNSUPPORTED  -7   /* a parameter combination this build does not provide */
#define ABIP_E_TIMEOUT      -8   /* a device-side wait ran past its limit (the kernel returned) */

/* ---- enums ---------------------------------------------------------------- */
#define ABIP_DENSE_ROWMAJOR  0
#define ABIP_CSR             1

#define ABIP_F32             0
#define ABIP_F64             1

/* solve status (Sec. 4.1; Thm 2.2 / Cor. 2.3 for the certificates) */
#define ABIP_UNSOLVED              0
#define ABIP_OPTIMAL               1
#define ABIP_PRIMAL_INFEASIBLE     2
#define ABIP_DUAL_INFEASIBLE       3
#define ABIP_MAX_ITER              4   /* ADMM cap reached (Sec. 5: the "---" entries) */

/* arithmetic of the iteration */
#define ABIP_PREC_F64        0   /* every vector and product in FP64 */
#define ABIP_PREC_MIXED      1   /* FP64 iterate and products, updated by FP32 products of the iterate's
                                    changes (sparse path: FP32 PCG for the correction of each projection
                                    solve, with an FP64 right-hand side); FP64 tests.  A CSR A's values
                                    are used rounded to FP32 */
#define ABIP_PREC_MIXED_BF16 2   /* as MIXED; the shared-A batch runs its products with A on the tensor
                                    cores (tcgen05, bfloat16 operands, FP32 accumulation): A as one
                                    bfloat16 plane when exact in bfloat16, else as three (any A within
                                    the FP32 range); other paths treat it as MIXED */

/* linear system for the projection (Sec. 4.4) */
#define ABIP_LINSYS_DENSE_CHOL  0   /* G = I + A A^T formed once, Cholesky G = L L^T, triangular solves */
#define ABIP_LINSYS_PCG         1   /* Jacobi-preconditioned CG on G, warm-started */
#define ABIP_LINSYS_SPARSE_LDL  2   /* direct projection through the quasi-definite system
                                       K = [I A^T; A -I] (Sec. 4.4): minimum-degree order and
                                       symbolic factor on the host (abip_ldl_analyze), numeric
                                       LDL^T once per setup and two triangular sweeps per update
                                       on the GPU.  CSR or dense input, precision F64 only */

/* ---- data ----------------------------------------------------------------- */
typedef struct {
    int32_t m, n;
    int32_t fmt;            /* ABIP_DENSE_ROWMAJOR or ABIP_CSR */
    int32_t dtype;          /* element type of val: ABIP_F32 or ABIP_F64 */
    int32_t on_device;      /* 1: val, row_ptr, col_idx are device pointers; 0: host */
    const void* val;        /* dense: m rows of ld elements; CSR: nnz values */
    int64_t ld;             /* dense leading dimension (>= n); ignored for CSR */
    const int64_t* row_ptr; /* CSR: m+1 entries */
    const int32_t* col_idx; /* CSR: nnz entries in [0, n) */
    int64_t nnz;            /* CSR: number of stored entries */
} abip_matrix;

typedef struct {
    double beta;            /* barrier weight; mu0 = beta (Algorithm 2); default 1 */
    double gamma;           /* mu <- gamma mu between inner loops; default 0.1 */
    double alpha;           /* over-relaxation in [0, 2) (Sec. 4.2); default 1.8 (Sec. 5) */
    double eps;             /* tolerance of every Sec. 4.1 test; default 1e-6 */
    int64_t max_admm_iters; /* cap on ADMM updates; default 1e6 (Sec. 5) */
    int32_t linsys;         /* ABIP_LINSYS_*; default: dense Cholesky for dense A, PCG for CSR */
    double cg_tol;          /* PCG stop: ||r|| <= cg_tol * max(1, ||rhs||); default 1e-10 */
    int32_t cg_max_iter;    /* PCG iteration cap per solve (exceeding it -> ABIP_E_NUMERICAL); default 1000 */
    double cg_rel;          /* > 0: PCG tolerance max(cg_tol, cg_rel * relative KKT residual of the
                               current iterate) instead of cg_tol alone; default 0 (fixed) */
    int32_t cg_warm;        /* PCG start: 0 previous solution, 1 linear extrapolation 2 z_k - z_{k-1},
                               2 quadratic extrapolation 3 z_k - 3 z_{k-1} + z_{k-2}; default 2 */
    int32_t precision;      /* ABIP_PREC_*; default ABIP_PREC_F64 */
    int32_t warmstart;      /* 0: keep-larger rescale of (x,s), (tau,kappa) and sqrt(gamma) on y, theta
                               (Sec. 5); 1: sqrt(gamma) on every component (Eq. update-next-iterate) */
    int32_t stop_rule;      /* 0: Sec. 4.1 tests; 1: stop once mu < eps (outer-count mode) */
    int32_t check_every;    /* mixed precision: minimum number of ADMM updates between two exact FP64
                               confirmations of the Sec. 4.1 tests (each screen pass that comes
                               sooner waits); 1 = confirm whenever the screen passes */
    int32_t grid_ctas;      /* 0: automatic; else the persistent grid size (tests) */
    int64_t barrier_limit_ns; /* sparse paths: wall-clock limit of one grid-barrier wait in the
                                 persistent kernel, and of one wait of the direct projection's
                                 factorisation and sweeps on an entry another warp computes; a
                                 wait past it ends the call with ABIP_E_TIMEOUT (the kernel
                                 returns).  0: 4 s (default) */
    int32_t bb_beta;        /* 1: choose beta at the start of every outer iteration by the
                               Barzilai-Borwein spectral rule with safeguarding and the heuristic
                               selection of Sec. 4.3 (two trial ADMM updates per estimate, a redo
                               from the same start when the estimate moves by more than
                               eps_penalty, at most bb_max_redo redos, never past max_admm_iters;
                               the trial updates count as ADMM updates).  Dense Cholesky path in
                               FP64 only (ABIP_E_UNSUPPORTED elsewhere).  Default 0 */
    int32_t bb_max_redo;    /* redos of one selection; default 5 */
    double eps_cor;         /* curvature-quality threshold of the safeguard; default 0.2 (Sec. 5) */
    double eps_penalty;     /* threshold of the heuristic selection; default 0.1 (Sec. 5) */
    int32_t autotune;       /* abip_solve_batch: 1 = time the occupancy variants of the solve kernel
                               on a 30-update run of this batch and use the fastest; the choice is
                               cached per (GPU, precision, batch shape) for the process and, when the
                               environment names a file in ABIP_TUNE_CACHE, in that JSON file.
                               Results do not depend on the choice.  Default 0 */
    int32_t batch_order;    /* abip_solve_batch: 1 = hand the instances to the CTAs largest first
                               (m n + m^2 descending), 0 = in the given order; default 1 */
    double gamma_max;       /* adaptive decrease ratio (Sec. 5 raises gamma near the optimum without a
                               rule): 0 = gamma at every mu <- gamma mu (default); else in [gamma, 1):
                               each decrease takes gamma + (gamma_max - gamma) t, t the position of
                               log10 rho between log10 0.1 (t = 0) and log10 eps (t = 1), clamped to
                               [0, 1], rho = max(pres, dres, dgap) of the iterate at the decrease.
                               Every path; the warm start of Eq. update-next-iterate takes the same
                               ratio */
    int32_t reserved[4];
} abip_params;

typedef struct {
    int32_t status;         /* ABIP_OPTIMAL, ... */
    int32_t outer_iters;    /* number of mu decreases */
    int64_t admm_iters;     /* ADMM updates executed */
    int64_t cg_iters;       /* total PCG iterations (PCG path) */
    double tau, kappa, theta, mu;
    double obj;             /* c^T x / tau */
    double pres, dres, dgap;/* relative residuals of Sec. 4.1 at the returned iterate */
    double setup_s, solve_s;/* wall-clock seconds of abip_setup and of the last solve */
    double kernel_s;        /* device time of the solve kernel, from CUDA events on the solve stream */
    int64_t launches;       /* kernels the solve call launched */
    int64_t fp32_iters;     /* ADMM updates whose products were FP32 (mixed precision: every path
                               keeps the iterate and its products in FP64 and updates them with
                               FP32 products of the changes) */
    double beta;            /* beta of the last outer iteration (params.beta unless bb_beta) */
    int32_t ctas_per_sm;    /* resident CTAs per SM of the dense solve launch (dense paths) */
    int32_t tuned;          /* abip_solve_batch with autotune: 1 chosen by timing in this call,
                               2 taken from the cache; 0 otherwise */
} abip_info;

typedef struct abip_handle abip_handle;

/* Fill p with the defaults listed above.  Returns ABIP_E_INVALID_ARG if p is NULL. */
ABIP_API int abip_default_params(abip_params* p);

/*
 * Build the embedding and the projection data for one LP (Sec. 3.1 and 4.4):
 * bbar = b - A e, cbar = c - e, zbar = c^T e + 1 (Eq. bar-b-c-z-re); for dense
 * Cholesky, G = I + A A^T and its factor L (Sec. 4.4, last paragraph); for PCG,
 * the Jacobi diagonal of G; then M^{-1} H and the 2 x 2 Schur complement K used
 * by every projection (the Remark of Sec. 4.4 on caching M^{-1} h).
 * A, b (m doubles), c (n doubles): host or device (b and c follow A->on_device).
 * Non-finite entries -> ABIP_E_INVALID_ARG.  p may be NULL (defaults).
 * On success *out owns device memory until abip_free.
 */
ABIP_API int abip_setup(const abip_matrix* A, const double* b, const double* c,
               const abip_params* p, abip_handle** out);

/*
 * Run Algorithm 2 from its start (y = 0, x = s = e, tau = kappa = theta = 1,
 * mu0 = beta) until a Sec. 4.1 test passes or max_admm_iters is reached.
 * x (n), y (m), s (n): caller-allocated, host or device, may be NULL.  They
 * receive (Sec. 4.1):
 *   OPTIMAL / MAX_ITER:     x/tau, y/tau, s/tau
 *   PRIMAL_INFEASIBLE:      x, y/(b^T y), s/(b^T y)   (y is the certificate)
 *   DUAL_INFEASIBLE:        -x/(c^T x), y, s          (x is the certificate)
 * info may be NULL.  stream: a cudaStream_t (NULL = default stream).  The call
 * returns when the solve has finished.
 */
ABIP_API int abip_solve(abip_handle* h, double* x, double* y, double* s,
               abip_info* info, void* stream);

/*
 * Solve `count` independent dense LPs in one persistent launch (one CTA per
 * instance at a time, pulled from a device work queue, each with its own
 * convergence state).  A[i] (dense row-major), b[i], c[i]: host pointers
 * (on_device = 0) or device pointers (on_device = 1) per instance.  x, y, s:
 * arrays of `count` caller-allocated output pointers (same memory kind as the
 * inputs), entries may be NULL.  infos: `count` entries, may be NULL.
 * Each instance needs 40m + 24n bytes (FP64) or 48m + 40n bytes (mixed) of shared
 * memory, at most 200 KB (ABIP_E_UNSUPPORTED otherwise); larger LPs go through
 * abip_setup with linsys = PCG.
 */
ABIP_API int abip_solve_batch(int32_t count, const abip_matrix* A, const double* const* b,
                     const double* const* c, const abip_params* p,
                     double* const* x, double* const* y, double* const* s,
                     abip_info* infos, void* stream);

/*
 * Solve `count` LPs  min c_k^T x  s.t.  A x = b_k,  x >= 0  that share one dense A
 * (e.g. basis pursuit with one dictionary and many measurements).  Algorithm 2 runs
 * for all instances in lockstep with per-instance convergence control; each update's
 * products are GEMMs over the instances (A [X S], A^T Y, G^{-1} Q, A^T Z_y with
 * G = I + A A^T of Sec. 4.4 inverted once from its FP64 Cholesky factor).
 *   A: one dense row-major matrix (host or device, F32 or F64), 1 <= m <= n.
 *   b[k] (m), c[k] (n): host or device.  x, y, s: arrays of `count` caller-allocated
 *   output pointers (host or device; entries may be NULL), scaled as abip_solve's.
 *   infos: `count` entries or NULL.  p->precision: ABIP_PREC_F64 (FP64 throughout),
 *   ABIP_PREC_MIXED (FP64 state; the products are updated by FP32 GEMMs of the state's
 *   changes and recomputed in FP64 every 200 cycles and before every termination
 *   decision) or ABIP_PREC_MIXED_BF16 (as MIXED with the products with A on the tensor
 *   cores: the changes are split into three bfloat16 terms, so the products keep FP32
 *   accuracy; A must be exactly representable in bfloat16, else ABIP_E_INVALID_ARG;
 *   shapes other than m, n multiples of 128 and count a multiple of 16 per chunk of 64
 *   use the FP32 GEMMs).
 * Instances are processed in chunks of 64.  Needs m <= 25600.  Errors: as
 * abip_solve_batch; ABIP_E_UNSUPPORTED for a CSR A.
 */
ABIP_API int abip_solve_batch_shared(int32_t count, const abip_matrix* A, const double* const* b,
                                     const double* const* c, const abip_params* p,
                                     double* const* x, double* const* y, double* const* s,
                                     abip_info* infos, void* stream);

/*
 * Gradient of a loss L(x*) of the returned primal solution x* = x / tau with respect
 * to (c, b, A), by implicit differentiation of the central point of the HSD
 * embedding at the final mu of the last abip_solve (the fixed point of the ADMM
 * inner loop at that mu, system HSD-log-kkt of Sec. 3.2: Q u = v with r = 0 and
 * xi = -n-1, x o s = tau kappa = mu / beta).  The final ADMM iterate is first
 * polished onto that point by damped Newton steps; then J^T lam = dL/dz is solved by
 * eliminating ds and dkappa, which leaves the reduced Jacobian
 * K = Q + diag(0, S X^-1, kappa / tau, 0) of order m + n + 2, factored by LU with
 * partial pivoting in FP64 (one step of iterative refinement), and
 * dL/dp = -lam^T dF/dp, counting the dependence of bbar, cbar, zbar on (A, b, c)
 * (Eq. bar-b-c-z-re).  The handle's state is left unchanged.
 *   dl_dx: n entries, dL/dx* (host or device).
 *   dl_dc (n), dl_db (m), dl_dA (m*n dense row-major, every entry, also for CSR
 *   input): caller-allocated outputs, host or device, each may be NULL.
 * Needs a dense handle (linsys = dense, or the automatic choice for dense input):
 * ABIP_E_UNSUPPORTED otherwise.  ABIP_E_NOT_SOLVED before the first solve;
 * ABIP_E_INVALID_ARG for an infeasibility result (no tau > 0) or non-finite dl_dx;
 * ABIP_E_NUMERICAL if K has an exactly zero pivot (singular at the central point).
 */
ABIP_API int abip_backward(abip_handle* h, const double* dl_dx,
                           double* dl_dc, double* dl_db, double* dl_dA);

/*
 * abip_backward for the instances of one abip_solve_batch call, one CTA per
 * instance in one launch.  A, b, c, p: as given to abip_solve_batch.  x, y, s,
 * infos: what that call returned (the outputs are x/tau, y/tau, s/tau; the raw
 * iterate is rebuilt from them and infos[k].tau, theta, kappa, mu, beta; beta = 0 reads
 * as p->beta).  dl_dx[k]
 * (n_k), outputs dl_dc[k] (n_k), dl_db[k] (m_k), dl_dA[k] (m_k*n_k): per-instance
 * pointers, host or device; the output arrays and their entries may be NULL.
 * Every instance needs status OPTIMAL or MAX_ITER.  Errors as abip_backward.
 */
ABIP_API int abip_backward_batch(int32_t count, const abip_matrix* A, const double* const* b,
                                 const double* const* c, const abip_params* p,
                                 const double* const* x, const double* const* y,
                                 const double* const* s, const abip_info* infos,
                                 const double* const* dl_dx, double* const* dl_dc,
                                 double* const* dl_db, double* const* dl_dA, void* stream);

/*
 * Copy the raw iterate after the last solve into buf (host or device, m + 2n + 4
 * doubles): (y[m], x[n], tau, theta, s[n], kappa, mu).  ABIP_E_NOT_SOLVED before
 * the first solve.
 */
ABIP_API int abip_get_state(const abip_handle* h, double* buf);

/*
 * Load a raw iterate (same layout as abip_get_state: y[m], x[n], tau, theta, s[n],
 * kappa, mu; host or device) into h.  The next abip_solve starts from it instead
 * of Algorithm 2's start (resume or warm start); the solve after that starts
 * from Algorithm 2's start again.  x, s, tau, kappa and mu must be > 0 and all
 * entries finite, else ABIP_E_INVALID_ARG.
 */
ABIP_API int abip_set_state(abip_handle* h, const double* buf);

/* Number of doubles abip_get_state writes (m + 2n + 4). */
ABIP_API int64_t abip_state_size(const abip_handle* h);

/*
 * Solve one small dense LP without allocating any memory.  For callers that
 * cannot call cudaMalloc (their device memory is owned by a framework's pool,
 * they run under a fixed memory budget, or they must not grow the process's
 * footprint): every scratch byte comes from one fixed array of 167,680 bytes that
 * the library holds on each device that loads it, until the process exits.  The
 * paper has no counterpart; this is the dense Cholesky path of abip_setup +
 * abip_solve for one instance, same kernels and same arithmetic.
 *   m, n, A (m x ld row-major FP64), b (m), c (n): inputs, device pointers.
 *   x (n), y (m), s (n): outputs, device pointers (same meaning as abip_solve).
 *   p: NULL for defaults; FP64 only.  info: host, may be NULL.  stream: cudaStream_t.
 * Limits: m <= 128, n <= 512 (larger -> ABIP_E_UNSUPPORTED).  Inputs are not
 * checked for non-finite values.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and should come before any stream
 * capture.  Every call uses the same array and leaves its contents behind:
 * calls whose work overlaps on the GPU (other host threads, other streams) race
 * and must be serialised by the caller.  Returns when the solve has finished.
 */
ABIP_API int abip_solve_dense_noalloc(int32_t m, int32_t n, const double* A, int64_t ld,
                                      const double* b, const double* c, const abip_params* p,
                                      double* x, double* y, double* s, abip_info* info, void* stream);

/* ---- presolve (Sec. 4.5) --------------------------------------------------- */
/*
 * Host presolve of the general LP
 *     min c^T x  s.t.  A x = b,  l <= x <= w        (l_j may be -inf, w_j +inf)
 * into the standard form the solver takes (min chat^T xhat, Ahat xhat = bhat, xhat >= 0):
 * the reductions P1-P7 of Sec. 4.5 (empty rows and columns, infeasible, fixed and free
 * variables, singleton rows, and the rows the Dulmage-Mendelsohn decomposition shows
 * dependent), the rewriting of the bounds (x = l + xbar with xbar + t = w - l when both are
 * finite, x = w - xbar when only w is, x = x+ - x- when free), then `ruiz` passes of Ruiz
 * equilibration (Ahat = D A E, bhat = D b, chat = E c; the Remark closing Sec. 4.5).
 * The objective of the original LP is chat^T xhat + info->obj_offset.
 *   A: host matrix (dense or CSR, F32 or F64; m >= 0, n >= 1, no n >= m requirement).
 *   b (m), c (n), l (n), w (n): host; non-finite b, c or NaN bounds -> ABIP_E_INVALID_ARG.
 *   tol in (0, 1): the tolerance of the zero tests (1e-9 is a good default).
 *   *out: receives the presolved problem (free with abip_presolve_free), also when the
 *   reductions alone decide the LP: info->status is then ABIP_PRIMAL_INFEASIBLE or
 *   ABIP_DUAL_INFEASIBLE (the reason in abip_last_error(NULL)), or ABIP_OPTIMAL when they
 *   removed every row (m = n = 0: abip_postsolve with empty x, y gives the solution);
 *   else 0.
 * Host code only; no GPU is needed.
 */
typedef struct abip_presolved abip_presolved;

typedef struct {
    int32_t status;          /* 0: the standard-form LP below is to be solved; else the status */
    int32_t m, n;            /* standard form */
    int64_t nnz;
    double obj_offset;
    int32_t empty_rows;      /* P1 */
    int32_t singleton_rows;  /* P6 (each fixes one column) */
    int32_t dependent_rows;  /* P7 */
    int32_t fixed_cols;      /* P4 */
    int32_t empty_cols;      /* P2 */
    int32_t free_split;      /* P5: free columns written as x+ - x- */
    int32_t upper_rows;      /* rows xbar + t = w - l added for finite upper bounds */
    int32_t reserved[5];
} abip_presolve_info;

ABIP_API int abip_presolve(const abip_matrix* A, const double* b, const double* c, const double* l,
                           const double* w, double tol, int32_t ruiz, abip_presolved** out,
                           abip_presolve_info* info);

/* Copy the standard-form LP out (host arrays sized from the info: row_ptr m+1, col_idx
   and val nnz, b m, c n; any may be NULL).  ABIP_E_INVALID_ARG when status != 0. */
ABIP_API int abip_presolved_lp(const abip_presolved* P, int64_t* row_ptr, int32_t* col_idx, double* val,
                               double* b, double* c);

/* Map a solution (x n, y m; s unused, may be NULL) of the standard-form LP back to the
   original LP (host): x_out (n0), y_out (m0, may be NULL), z_out = c - A^T y_out (n0, may
   be NULL), obj = c^T x_out (may be NULL).  Dropped rows get y = 0; a singleton row gets
   the y that makes the reduced cost of the column it fixed zero. */
ABIP_API int abip_postsolve(const abip_presolved* P, const double* x, const double* y, const double* s,
                            double* x_out, double* y_out, double* z_out, double* obj);

ABIP_API void abip_presolve_free(abip_presolved* P);

/*
 * Symbolic analysis of the sparse direct projection (linsys = ABIP_LINSYS_SPARSE_LDL,
 * Sec. 4.4).  With yhat = -y the projection's system M [y; x] = r becomes
 * K [x; yhat] = [r_x; r_y] with the quasi-definite K = [I_n A^T; A -I_m] of order n + m,
 * node j < n standing for x_j and node n + i for row i of A.  Every symmetric permutation
 * of K has an LDL^T factor (pivots > 0 on x nodes, < 0 on row nodes); this call orders K
 * by minimum degree (ties by node number; once the remaining graph is complete, the rest
 * in node order) and counts the factor's nonzeros.  Host only: no GPU is touched.
 *   A           the constraint matrix (host pointers, on_device = 0), CSR or dense
 *   perm        n + m int32 or NULL: perm[p] = node of the p-th pivot
 *   col_counts  n + m int64 or NULL: strictly-lower nonzeros of column p of L
 *   nnz_l       NULL or receives their sum
 * ABIP_E_INVALID_ARG / ABIP_E_DIM for a bad matrix (on_device = 1 included);
 * ABIP_E_UNSUPPORTED when the factor would hold more than 4e8 nonzeros or the ordering
 * passes its work limit (the message in abip_last_error(NULL)).
 */
ABIP_API int abip_ldl_analyze(const abip_matrix* A, int32_t* perm, int64_t* col_counts, int64_t* nnz_l);

/* Release every resource of h (NULL is accepted). */
ABIP_API void abip_free(abip_handle* h);

/* Name of a status code ("optimal", ...). */
ABIP_API const char* abip_status_str(int32_t status);

/* Message of the last failure on h, or of the last failed abip_setup/abip_solve_batch
   when h is NULL.  Never NULL. */
ABIP_API const char* abip_last_error(const abip_handle* h);

/* Library version string. */
ABIP_API const char* abip_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ABIP_H */
