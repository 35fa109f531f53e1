// Host-side internals of libabip: the handle, the device control block and the
// kernel entry points shared between translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/abip.h"

namespace abip {

constexpr int kGridThreads = 768;   // threads per CTA of the persistent grid kernel (one CTA per SM)
constexpr int kNumSlots = 24;       // reduction slots of the grid kernel

enum GridMode : int { MODE_SETUP = 0, MODE_SOLVE = 1 };

// Control block of one single-instance solve, resident in device memory.  The
// host writes the inputs, the kernel writes the outputs.
struct SolveCtl {
  // inputs
  double beta, gamma, alpha, eps, cg_tol, cg_rel;
  double gamma_max;               // > 0: adaptive decrease ratio (adaptive_gamma)
  double zbar, xi, nb, nc;
  double Kinv[4];                 // inverse of the 2x2 Schur complement, row-major
  int64_t max_admm;
  int32_t cg_max, warmstart, stop_rule, mode;
  int32_t cg_warm, pad2;
  int32_t check_every, pad0;
  // state carried across calls (in/out)
  double tau, kappa, theta, mu;
  int64_t admm_iters, cg_iters;
  int32_t outer_iters, status;
  // outputs
  double pres, dres, dgap, ctx, bty, inner2;
  double K[4];                    // MODE_SETUP: the Schur complement K = I + S + H^T M^{-1} H
  double sum_c, sum_b2, sum_c2;   // MODE_SETUP: c^T e, ||b||^2, ||c||^2
  int32_t err;                    // DevErr
  int32_t pad1;
  unsigned long long* prof;       // optional phase timers (kProfBuckets ns counters), null = off
  unsigned long long bar_limit_ns;// wall-clock limit of one grid-barrier wait (0: kBarrierLimitNs)
  int64_t refreshes;              // mixed path: exact FP64 recomputations of the maintained products
  int32_t setup_rounds;           // mixed path: refinement rounds of the setup solves
  int32_t pad4;
  unsigned long long ldl_epoch;   // sparse direct projection: solves done so far (flag epochs)
};

// phase timer buckets of the solve kernel (CTA 0's view, nanoseconds)
enum ProfBucket : int {
  P_PCG_INIT = 0, P_CG_AT, P_CG_A, P_CG_UPD, P_ZX, P_UPD, P_RES, P_WARM, P_BARRIER, P_TOTALS, P_SETUP,
  kProfBuckets
};

// A sparse matrix in SELL form with L lanes per row: rows sorted by length
// (longest first), cut into slices of C = 32/L consecutive sorted rows (one warp
// per slice).  Row r of a slice is handled by lanes r*L .. r*L+L-1; entry k of the
// row belongs to lane r*L + k%L at chunk k/L, stored at sp[s] + 32 (k/L) + r*L + k%L.
// Every lane of a slice is padded with zeros to the slice's longest lane (padding
// points at a column the row uses).  perm maps sorted position to row (-1 = none).
struct SellMat {
  int rows = 0, nslices = 0;
  int lanes = 1;                  // L: lanes per row (1, 2, 4, 8, 16 or 32)
  const int64_t* sp = nullptr;    // nslices + 1 offsets (multiples of 32)
  const int32_t* ci = nullptr;    // column indices, padded
  const void* val = nullptr;      // values (float or double), padded
  const int32_t* perm = nullptr;  // nslices * C
  const int32_t* wsl = nullptr;   // per global warp w: slices [wsl[w], wsl[w+1]), balanced by nonzeros
};

// two interleaved vectors, gathered together with one load
template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Device error code of the sparse direct projection, beside the DevErr codes: a pivot of
// the wrong sign or not finite, or a row missing from the symbolic pattern.
constexpr int DEV_ERR_LDL = 5;

// Sparse direct projection (Sec. 4.4): the LDL^T factor of P K P^T with the
// quasi-definite K = [[I_n, A^T], [A, -I_m]] (pattern and order from ldl_host.h), and
// the arrays of its sync-free factorisation and triangular solves.  N = 0: not used.
struct LdlDev {
  int N = 0;
  const int32_t* perm = nullptr;  // N: node of pivot p (x_j: j, yhat_i: n + i)
  const int64_t* Lp = nullptr;    // N + 1: column p of L (strictly lower) is Li / Lx[Lp[p] .. Lp[p+1])
  const int32_t* Li = nullptr;    // nnz(L) row indices, increasing within a column
  double* Lx = nullptr;           // nnz(L): K's entries when uploaded, L after the factorisation
  const int64_t* Rp = nullptr;    // N + 1: row p of L is Rk / Rpos[Rp[p] .. Rp[p+1])
  const int32_t* Rk = nullptr;    // nnz(L): column k < p of each entry of row p, increasing
  const int32_t* Rpos = nullptr;  // nnz(L): position of L(p, k) in Li / Lx
  double* Dd = nullptr;           // N: pivots D_p
  double* zf = nullptr;           // 2N: forward sweep L z = P r, one buffer of N per solve parity
  double* wb = nullptr;           // 2N: backward sweep L^T w = D^{-1} z, likewise
                                  // (an entry not yet computed holds kLdlEmpty)
  unsigned long long* flag = nullptr;  // N, zeroed at setup: 1 once column p is factored
};

// Bit pattern of a sweep entry not yet computed: a signalling NaN, which no arithmetic
// result can be (operations return quiet NaNs), so a reader can wait on the value itself.
constexpr unsigned long long kLdlEmpty = 0x7FF4A5A5A5A5A5A5ull;

// Everything the direct projection's device routines touch, kept in device memory so
// that they take one plain pointer (the grid kernel's GridData is a kernel parameter).
struct LdlView {
  LdlDev F;
  int m = 0, n = 0;
  const double* b = nullptr; const double* c = nullptr;
  const double* bbar = nullptr; const double* cbar = nullptr;
  const double* y = nullptr; const double* x = nullptr; const double* s = nullptr;   // iterate
  double* zy = nullptr; double* zx = nullptr;                                        // M^{-1} w
  double* g1y = nullptr; double* g1x = nullptr; double* g2y = nullptr; double* g2x = nullptr;
  double* partials = nullptr;
  SolveCtl* ctl = nullptr;
};

// Device pointers of the sparse single-instance path.
template <typename T>
struct GridData {
  int m, n;
  SellMat A;                                                  // rows of A
  SellMat AT;                                                 // rows of A^T
  const T* b; const T* c;                                     // problem data in T
  T* bbar; T* cbar; T* dinv;                                  // embedding constants, Jacobi diagonal
  T* g1y; T* g1x; T* g2y; T* g2x;                            // M^{-1} h1, M^{-1} h2
  T* y; T* x; T* s;                                           // iterate (r = 0, xi = -n-1 implicit)
  T* Ax; T* As; T* ATy;                                       // products for the residuals
  T* zy; T* zx;                                               // M^{-1} w (zy warm-starts PCG)
  T* zp2; T* zp3;                                             // the two zy before the last (extrapolated start)
  T* r; T* p; T* Gp;                                          // PCG work vectors
  typename Vec2<T>::type* ut;                                 // (u, t) per column: A^T zr and A^T p
  typename Vec2<T>::type* zd;                                 // (zr, D^{-1} Gp) per row, double-buffered
  typename Vec2<T>::type* zd2;
  double* partials;                                           // kNumSlots * gridDim doubles
  unsigned long long* bar;                                    // barrier arrival counter
  SolveCtl* ctl;
  int ldl_N;                                                  // > 0: direct projection instead of PCG
  const LdlView* ldlv;                                        // its arrays (device memory)
};

// Per column of the mixed sparse path: the FP32 change (dx, ds) of the iterate and
// W = A^T (z_y + delta_0) in FP64, gathered together (16 bytes) by the products with A.
struct XSW {
  float dx, ds;
  double w;
};

// Device pointers of the sparse mixed-precision path (grid_delta.cu): the iterate, the
// products the update needs and the embedding data in FP64; the matrix values, the
// changes of the iterate and the PCG work vectors of the correction solve in FP32.
struct GridDelta {
  int m, n;
  SellMat A;                                   // rows of A (float values)
  SellMat AT;                                  // rows of A^T (float values)
  const double* b; const double* c;
  double* bbar; double* cbar;                  // embedding constants
  double* g1y; double* g1x; double* g2y; double* g2x;   // M^{-1} h1, M^{-1} h2
  double* y; double* x; double* s;             // iterate (r = 0, xi = -n-1 implicit)
  double* Ax; double* As; double* ATy;         // maintained products for the residuals
  double* zy; double* ATz;                     // z_y = G^{-1} q and A^T z_y
  float* dinv;                                 // Jacobi diagonal 1 / (1 + sum_j A_ij^2)
  float* dz;                                   // correction of z_y: the start of the next solve, then its
                                               // PCG iterate
  float* d1; float* d2;                        // the last two corrections (extrapolated start)
  float* r; float* p; float* Gp;               // PCG work vectors
  float2* ut; float2* zd; float2* zd2;         // (A^T zr, A^T p); (zr, D^{-1} Gp), double-buffered
  float* wdel;                                 // n: sum over PCG iterations of alpha A^T p
  XSW* xsw;                                    // per column: (dx, ds, W), W = A^T (z_y + start)
  float* dy;                                   // change of y
  double* partials;                            // kNumSlots * gridDim doubles
  unsigned long long* bar;                     // barrier arrival counter
  SolveCtl* ctl;
};

// Launch the persistent grid kernel (cooperative).  val_f64: whether A's values are double.
cudaError_t launch_grid_solver_f64(const GridData<double>& d, bool val_f64, int grid, cudaStream_t st);
int grid_solver_max_ctas(bool val_f64, int device);
cudaError_t launch_grid_delta(const GridDelta& d, int grid, cudaStream_t st);
int grid_delta_max_ctas(int device);

// ---------------------------------------------------------------------------
// dense CTA-per-instance path
// ---------------------------------------------------------------------------

// Per-instance descriptor of the batched dense solver (device array).
struct DenseInst {
  int32_t m, n;
  int64_t ld;                  // leading dimension of A (row-major)
  const double* A;             // m x ld, FP64
  const double* b; const double* c;
  double* L;                   // m x m Cholesky factor of G (row-major, lower)
  double* bbar; double* cbar;  // embedding constants
  double* g1; double* g2;      // M^{-1} h1, M^{-1} h2, (m + n) each: [y part, x part]
  double* y; double* x; double* s;   // iterate
  double* work;                // bb_work_doubles(m, n) when the Barzilai-Borwein rule is on, else null
  double* out_x; double* out_y; double* out_s;   // device outputs (may be null)
  // mixed precision (null on the FP64 path): FP32 A (rows padded to ldf), FP32 A^T
  // (rows padded to ldtf) and the FP32 explicit inverse of G = I + A A^T (m x ldtf)
  const float* Af; const float* ATf; float* Ginvf;
  double zbar, nb, nc;
  double Kinv[4];
  // results
  double tau, kappa, theta, mu;
  double pres, dres, dgap, obj, ctx, bty;
  int64_t admm_iters;
  int32_t outer_iters, status;
  int32_t err;
  int32_t resume;              // 1: start from y, x, s and the scalars below instead of Algorithm 2's start
  double r_tau, r_kappa, r_theta, r_mu;
  int64_t r_iters;             // counters carried into a resumed solve
  int32_t r_outer;
  int32_t fp32_iters_hi;       // mixed path: ADMM updates done in FP32 (low and high 31 bits)
  int32_t fp32_iters_lo;
  int32_t ldf, ldtf;           // padded row lengths of Af (n) and of ATf / Ginvf (m), multiples of 4
  int32_t pad3;
  double beta_last;            // beta of the last outer iteration
};

// One instance of the central-point differentiation (dense A, FP64, device pointers).
struct BackwardInst {
  int32_t m, n;
  int64_t ld;
  const double* A; const double* b; const double* c;
  double* y; double* x; double* s;  // in: final ADMM iterate (raw); out: Newton-polished point
  double tau, theta, kappa;         // in/out like y, x, s
  double cmu;                       // mu / beta of the central point
  const double* dl_dx;              // dL/dx*, x* = x / tau (n)
  double* dA; double* db; double* dc;   // outputs (each may be null); dA m x n row-major
  double* K;                        // (m + n + 2)^2 scratch: the reduced Jacobian and its LU
  double* work;                     // backward_work_doubles(m, n) doubles scratch
  int32_t newton_max;
  int32_t pad;
  double newton_tol;
  double fnorm;                     // out: ||F|| at the point differentiated
  int32_t steps, err;               // out: Newton steps taken; 1 if a factorisation broke down
};

struct DenseParams {
  double beta, gamma, alpha, eps;
  int64_t max_admm;
  int32_t warmstart, stop_rule;
  int32_t mixed;          // 1: FP32 iterates with FP64 termination decisions
  int32_t check_every;    // mixed: minimum spacing of FP64 confirmations (updates)
  int32_t bb;             // 1: Barzilai-Borwein beta at each outer iteration (FP64 path)
  int32_t bb_max_redo;
  double eps_cor, eps_penalty;
  double gamma_max;       // > 0: adaptive decrease ratio (adaptive_gamma)
};

// global scratch of the Barzilai-Borwein selection per instance (DenseInst::work)
inline size_t bb_work_doubles(int m, int n) { return 4 * (size_t)m + 6 * (size_t)n; }

cudaError_t launch_dense_setup(DenseInst* inst, int count, int* queue, int grid, size_t smem, cudaStream_t st);
// Occupancy variants of the dense solve kernel (the batch autotuner's choice)
constexpr int kDenseVariants = 3;
cudaError_t launch_dense_solve(DenseInst* inst, int count, DenseParams prm, int* queue, const int* order,
                               int grid, size_t smem, int variant, cudaStream_t st);
int dense_solve_ctas_per_sm(bool mixed, size_t smem, int variant);
int dense_max_ctas(int device);
cudaError_t launch_dense_backward(BackwardInst* insts, int count, int grid, cudaStream_t st);
inline size_t backward_work_doubles(int m, int n) { return 2 * (size_t)m + 4 * (size_t)n + 5 * ((size_t)m + n + 2); }

// shared by the allocation-free entry point (defined in abip_api.cu)
int check_params_internal(const abip_params& p, std::string& why);
int noalloc_fail(int code, const std::string& msg);


// ---------------------------------------------------------------------------
// Batch of LPs sharing one dense A (shared_solver.cu)
// ---------------------------------------------------------------------------
enum ShAction : int32_t { SH_INIT = 0, SH_STEP = 1, SH_WARM = 2, SH_DONE = 4 };

// Per-instance scalars of the shared-A batch.
struct ShInst {
  double tau, kappa, theta, mu, cmu;
  double zbar, nb, nc, Kinv[4];
  double inner2, pres, dres, dgap, ctx, bty;
  double t1, t2;
  int64_t total, level_start, next_confirm;
  int32_t outer, status, action, last, err;
  int32_t pending;                 // mixed: the FP32-maintained screen passed; decide at the next refresh
  double gam;                      // the decrease ratio of the last mu <- gam mu (the warm start's)
};

struct ShParams {
  double beta, gamma, alpha, eps;
  int64_t max_admm;
  int32_t warmstart, stop_rule, mixed, n;
  int64_t confirm_gap;
  int32_t refresh;                 // mixed: FP64 recomputation of the maintained products every `refresh` cycles
  int32_t tc;                      // mixed: products with A on the tensor cores: 0 off, else the number
                                   // of bfloat16 terms of A (1: A exact in bfloat16, 3: A in FP32)
  double gamma_max;                // > 0: adaptive decrease ratio (adaptive_gamma)
};

// Device arrays of one iteration type; every vector is [length x B], instance fastest.
// XS = [X | S] (n x 2B), AXS = [AX | AS] (m x 2B), G1 / G2 = M^{-1} h1 / h2 ((m+n) x B).
template <typename T>
struct ShView {
  int m, n, B;
  const T* A; const T* Ginv;
  T* b; T* bbar; T* c; T* cbar; T* G1; T* G2;
  T* Y; T* XS; T* AXS; T* ATY; T* Q; T* ZY; T* ZX;
};

struct SharedBatchArgs {
  int m, n, count;                 // count <= 64
  const double* A;                 // host, m x n row-major FP64
  const double* const* b;          // host, count vectors of m
  const double* const* c;          // host, count vectors of n
  ShParams prm;
  cudaStream_t stream;
};

struct SharedBatchResult {
  ShInst inst;
  std::vector<double> x, y, s;     // scaled outputs (Sec. 4.1)
  double setup_s;                  // device time of the setup (Gram, Cholesky, inverse, M^{-1} H)
  double kernel_s;                 // device time of the iterations
  int64_t launches;
  bool tensor_cores;               // the products with A ran on tcgen05
};

int shared_batch_run(const SharedBatchArgs& a, std::vector<SharedBatchResult>& out, std::string& err);

}  // namespace abip

// The opaque handle of the C ABI.
struct abip_handle {
  int device = 0;
  int m = 0, n = 0;
  int path = 0;                 // 0 = CSR grid path, 1 = dense CTA path
  int mixed = 0;
  int val_f64 = 0;
  abip_params prm{};
  double setup_s = 0, solve_s = 0;
  bool solved = false;
  std::string err;
  // device arena
  void* arena = nullptr;
  size_t arena_bytes = 0;
  abip::SolveCtl* ctl = nullptr;
  abip::GridData<double> gd64{};
  abip::GridDelta gdd{};
  double* stage = nullptr;            // m + 2n doubles for scaled outputs
  int grid = 0;
  // dense path
  abip::DenseInst* dinst = nullptr;   // device, one entry
  int* queue = nullptr;
  abip::DenseInst hinst{};            // host mirror of the descriptor
  double nb = 0, nc = 0;
  int64_t padded_nnz_a = 0, padded_nnz_at = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double kernel_s = 0;
  int64_t launches = 0;
  bool resume = false;                // next solve starts from a state set by abip_set_state
  std::vector<double> resume_state;   // y, x, tau, theta, s, kappa, mu
};
