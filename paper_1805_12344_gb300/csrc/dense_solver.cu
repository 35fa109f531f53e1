// Dense ABIP, one CTA per LP instance (persistent: CTAs pull instance ids from a
// device work queue, so a batch of uneven LPs runs in one launch and every
// instance keeps its own convergence state).
//
// Setup (per instance): G = I + A A^T (Sec. 4.4, dense A), its Cholesky factor
// G = L L^T in FP64, the embedding constants of Eq. bar-b-c-z-re, M^{-1} h1,
// M^{-1} h2 and the inverse of the 2x2 Schur complement (Sec. 4.4 generalised to
// the 4-block Q).  Solve: Algorithm 2 with over-relaxation (Sec. 4.2), the
// projection through two blocked triangular solves with L, and the Sec. 4.1 tests
// after every update.  All vectors of the iteration live in shared memory.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "abip_device.cuh"
#include "abip_internal.h"

namespace abip {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// next instance id from the work queue (thread 0), broadcast to the CTA; `order` (may be
// null) lists the instances in the order they are handed out
__device__ __forceinline__ int next_instance(int* queue, int count, const int* order = nullptr) {
  __shared__ int s_id;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int q = atomicAdd(queue, 1);
    s_id = q < count ? (order ? order[q] : q) : -1;
  }
  __syncthreads();
  return s_id;
}

// w <- L^{-1} w, L lower triangular (row-major, leading dimension m), w in shared memory.
template <typename T>
__device__ void trsv_lower(const T* __restrict__ L, int m, T* w) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int kb = 0; kb < m; kb += 32) {
    const int nb = min(32, m - kb);
    if (wid == 0) {
      T wl = lane < nb ? w[kb + lane] : T(0);
      for (int j = 0; j < nb; ++j) {
        if (lane == j) wl = wl / L[(size_t)(kb + j) * m + kb + j];
        const T wj = __shfl_sync(0xffffffffu, wl, j);
        if (lane > j && lane < nb) wl -= L[(size_t)(kb + lane) * m + kb + j] * wj;
      }
      if (lane < nb) w[kb + lane] = wl;
    }
    __syncthreads();
    const T wb = lane < nb ? w[kb + lane] : T(0);
    for (int i = kb + nb + wid; i < m; i += kWarps) {
      T a = lane < nb ? L[(size_t)i * m + kb + lane] * wb : T(0);
      a = warp_sum(a);
      if (lane == 0) w[i] -= a;
    }
    __syncthreads();
  }
}

// w <- L^{-T} w.
template <typename T>
__device__ void trsv_lower_t(const T* __restrict__ L, int m, T* w) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nblk = (m + 31) / 32;
  for (int bk = nblk - 1; bk >= 0; --bk) {
    const int kb = bk * 32;
    const int nb = min(32, m - kb);
    if (wid == 0) {
      T wl = lane < nb ? w[kb + lane] : T(0);
      for (int j = nb - 1; j >= 0; --j) {
        if (lane == j) wl = wl / L[(size_t)(kb + j) * m + kb + j];
        const T zj = __shfl_sync(0xffffffffu, wl, j);
        if (lane < j) wl -= L[(size_t)(kb + j) * m + kb + lane] * zj;
      }
      if (lane < nb) w[kb + lane] = wl;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kb; i += kThreads) {
      T a = T(0);
      for (int j = 0; j < nb; ++j) a += L[(size_t)(kb + j) * m + i] * w[kb + j];
      w[i] -= a;
    }
    __syncthreads();
  }
}

// out[i] = sum_j A_ij v_j (warp per row, accumulated in Acc); optional second vector.
template <bool TWO, typename Acc, typename TA, typename TV, typename TO>
__device__ void gemv_rows(const TA* __restrict__ A, int64_t ld, int m, int n, const TV* v0,
                          const TV* v1, TO* o0, TO* o1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < m; i += kWarps) {
    const TA* row = A + (size_t)i * ld;
    Acc a0 = Acc(0), a1 = Acc(0);
    for (int j = lane; j < n; j += 32) {
      const Acc a = (Acc)row[j];
      a0 += a * (Acc)v0[j];
      if (TWO) a1 += a * (Acc)v1[j];
    }
    a0 = warp_sum(a0);
    if (TWO) a1 = warp_sum(a1);
    if (lane == 0) {
      o0[i] = (TO)a0;
      if (TWO) o1[i] = (TO)a1;
    }
  }
}

// out[j] = sum_i A_ij v_i (thread per column, rows unrolled by 4).
__device__ void gemv_cols(const double* __restrict__ A, int64_t ld, int m, int n, const double* v,
                          double* o) {
  for (int j = threadIdx.x; j < n; j += kThreads) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int i = 0;
    for (; i + 4 <= m; i += 4) {
      a0 += A[(size_t)i * ld + j] * v[i];
      a1 += A[(size_t)(i + 1) * ld + j] * v[i + 1];
      a2 += A[(size_t)(i + 2) * ld + j] * v[i + 2];
      a3 += A[(size_t)(i + 3) * ld + j] * v[i + 3];
    }
    for (; i < m; ++i) a0 += A[(size_t)i * ld + j] * v[i];
    o[j] = (a0 + a1) + (a2 + a3);
  }
}

// Cholesky of G (lower triangle stored in L, row-major), in place, one CTA.
__device__ bool cholesky(double* L, int m) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_ok = 1;
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      const double d = L[(size_t)k * m + k];
      if (!(d > 0.0) || !isfinite(d)) s_ok = 0;
      L[(size_t)k * m + k] = sqrt(d);
    }
    __syncthreads();
    if (!s_ok) return false;
    const double dk = L[(size_t)k * m + k];
    for (int i = k + 1 + threadIdx.x; i < m; i += kThreads) L[(size_t)i * m + k] /= dk;
    __syncthreads();
    const int rem = m - k - 1;
    // trailing update of the lower triangle: rows i > k, columns k < j <= i
    for (int idx = threadIdx.x; idx < rem * rem; idx += kThreads) {
      const int ii = idx / rem, jj = idx % rem;
      if (jj <= ii) {
        const int i = k + 1 + ii, j = k + 1 + jj;
        L[(size_t)i * m + j] -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      }
    }
    __syncthreads();
  }
  // zero the strict upper triangle (kept clean for readers)
  for (int idx = threadIdx.x; idx < m * m; idx += kThreads) {
    const int i = idx / m, j = idx % m;
    if (j > i) L[idx] = 0.0;
  }
  __syncthreads();
  return true;
}

// G = I + A A^T into the lower triangle of L (32x32 output tiles through shared memory).
__device__ void gram(const double* __restrict__ A, int64_t ld, int m, int n, double* L, double* sm) {
  double* Ti = sm;            // 32 x 33
  double* Tk = sm + 32 * 33;  // 32 x 33
  const int nt = (m + 31) / 32;
  const int tr = threadIdx.x / 32, tc = threadIdx.x % 32;   // 8 x 32 threads, 4 rows each
  for (int bi = 0; bi < nt; ++bi) {
    for (int bk = 0; bk <= bi; ++bk) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int j0 = 0; j0 < n; j0 += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += kThreads) {
          const int r = e / 32, c = e % 32;
          const int gi = bi * 32 + r, gk = bk * 32 + r, gj = j0 + c;
          Ti[r * 33 + c] = (gi < m && gj < n) ? A[(size_t)gi * ld + gj] : 0.0;
          Tk[r * 33 + c] = (gk < m && gj < n) ? A[(size_t)gk * ld + gj] : 0.0;
        }
        __syncthreads();
        for (int c = 0; c < 32; ++c) {
          const double kv = Tk[tc * 33 + c];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] += Ti[(tr * 4 + q) * 33 + c] * kv;
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int gi = bi * 32 + tr * 4 + q, gk = bk * 32 + tc;
        if (gi < m && gk <= gi) L[(size_t)gi * m + gk] = acc[q] + (gi == gk ? 1.0 : 0.0);
      }
    }
  }
  __syncthreads();
}

// M [zy; zx] = [a; d]  ->  zy = G^{-1}(a - A d), zx = d + A^T zy (Sec. 4.4).
// a (m), d (n) in shared memory; results in zy (m), zx (n); tmp (m) scratch.
__device__ void solve_M(const DenseInst& I, const double* a, const double* d, double* zy, double* zx,
                        double* tmp) {
  gemv_rows<false, double>(I.A, I.ld, I.m, I.n, d, d, tmp, tmp);
  __syncthreads();
  for (int i = threadIdx.x; i < I.m; i += kThreads) zy[i] = a[i] - tmp[i];
  __syncthreads();
  trsv_lower<double>(I.L, I.m, zy);
  trsv_lower_t<double>(I.L, I.m, zy);
  gemv_cols(I.A, I.ld, I.m, I.n, zy, zx);
  for (int j = threadIdx.x; j < I.n; j += kThreads) zx[j] += d[j];
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) dense_setup_kernel(DenseInst* insts, int count, int* queue) {
  extern __shared__ double sm[];
  __shared__ double red[32 * 8];
  for (;;) {
    const int id = next_instance(queue, count);
    if (id < 0) return;
    DenseInst& I = insts[id];
    const int m = I.m, n = I.n;
    // embedding constants
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < m; i += kThreads) {
      double rs = 0.0;
      for (int j = 0; j < n; ++j) rs += I.A[(size_t)i * I.ld + j];
      I.bbar[i] = I.b[i] - rs;
      acc[1] += I.b[i] * I.b[i];
    }
    for (int j = threadIdx.x; j < n; j += kThreads) {
      I.cbar[j] = I.c[j] - 1.0;
      acc[0] += I.c[j];
      acc[2] += I.c[j] * I.c[j];
    }
    block_allsum<3>(acc, red);
    const double zbar = acc[0] + 1.0;
    gram(I.A, I.ld, m, n, I.L, sm);
    if (!cholesky(I.L, m)) {
      if (threadIdx.x == 0) { I.err = DEV_ERR_CHOLESKY; I.status = 0; }
      continue;
    }
    // M^{-1} h1, M^{-1} h2 with h1 = [-b; c], h2 = [bbar; -cbar]
    double* a = sm;            // m
    double* d = sm + m;        // n
    double* tmp = sm + m + n;  // m
    for (int col = 0; col < 2; ++col) {
      double* g = col == 0 ? I.g1 : I.g2;
      for (int i = threadIdx.x; i < m; i += kThreads) a[i] = col == 0 ? -I.b[i] : I.bbar[i];
      for (int j = threadIdx.x; j < n; j += kThreads) d[j] = col == 0 ? I.c[j] : -I.cbar[j];
      __syncthreads();
      solve_M(I, a, d, g, g + m, tmp);
    }
    // K = I + S + H^T M^{-1} H, S = [[0, zbar], [-zbar, 0]]
    double k4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < m; i += kThreads) {
      k4[0] += -I.b[i] * I.g1[i]; k4[1] += -I.b[i] * I.g2[i];
      k4[2] += I.bbar[i] * I.g1[i]; k4[3] += I.bbar[i] * I.g2[i];
    }
    for (int j = threadIdx.x; j < n; j += kThreads) {
      k4[0] += I.c[j] * I.g1[m + j]; k4[1] += I.c[j] * I.g2[m + j];
      k4[2] += -I.cbar[j] * I.g1[m + j]; k4[3] += -I.cbar[j] * I.g2[m + j];
    }
    block_allsum<4>(k4, red);
    if (threadIdx.x == 0) {
      const double K0 = 1.0 + k4[0], K1 = zbar + k4[1], K2 = -zbar + k4[2], K3 = 1.0 + k4[3];
      const double det = K0 * K3 - K1 * K2;
      I.Kinv[0] = K3 / det; I.Kinv[1] = -K1 / det; I.Kinv[2] = -K2 / det; I.Kinv[3] = K0 / det;
      I.zbar = zbar;
      I.nb = sqrt(acc[1]);
      I.nc = sqrt(acc[2]);
      I.err = isfinite(det) && det != 0.0 ? 0 : DEV_ERR_NONFINITE;
    }
    __syncthreads();
    if (I.Ginvf) {   // mixed precision: the FP32 explicit inverse of G, column by column
      double* w = sm;   // m
      for (int col = 0; col < m; ++col) {
        for (int i = threadIdx.x; i < m; i += kThreads) w[i] = i == col ? 1.0 : 0.0;
        __syncthreads();
        trsv_lower<double>(I.L, m, w);
        trsv_lower_t<double>(I.L, m, w);
        for (int i = threadIdx.x; i < m; i += kThreads) I.Ginvf[(size_t)col * I.ldtf + i] = (float)w[i];
        __syncthreads();
      }
    }
  }
}

// The instance data a solve of iteration type T reads.
template <typename T>
struct DView {
  const T* A; const T* L; const T* g1; const T* g2; const T* b; const T* c; const T* bbar; const T* cbar;
};
__device__ __forceinline__ DView<double> view(const DenseInst& I, double) {
  return {I.A, I.L, I.g1, I.g2, I.b, I.c, I.bbar, I.cbar};
}

// Residual products Ax, As, A^T y and the nine sums of the Sec. 4.1 tests and
// Eq. inner-stop, with products accumulated in Acc:
//   0 ||Qu-v||^2 (vector blocks), 1 ||Ax/tau - b||^2, 2 ||(A^T y + s)/tau - c||^2,
//   3 ||Ax||^2, 4 ||A^T y + s||^2, 5 b^T y, 6 bbar^T y, 7 c^T x, 8 cbar^T x.
template <typename Acc, typename T>
__device__ void residual_sums(const DView<T>& V, int m, int n, int64_t ld, const T* x, const T* s, const T* y,
                              double tau, double theta, T* Ax, T* As, double (&out)[9], double* red) {
  gemv_rows<true, Acc>(V.A, ld, m, n, x, s, Ax, As);
  __syncthreads();
  Acc acc[9] = {Acc(0), Acc(0), Acc(0), Acc(0), Acc(0), Acc(0), Acc(0), Acc(0), Acc(0)};
  const Acc ta = (Acc)tau, th = (Acc)theta;
  for (int i = threadIdx.x; i < m; i += kThreads) {
    const Acc ax = (Acc)Ax[i], bi = (Acc)V.b[i], yi = (Acc)y[i], bb = (Acc)V.bbar[i];
    const Acc ry = ax - bi * ta + bb * th;
    const Acc pr = ax / ta - bi;
    acc[0] += ry * ry; acc[1] += pr * pr; acc[3] += ax * ax;
    acc[5] += bi * yi; acc[6] += bb * yi;
  }
  for (int j = threadIdx.x; j < n; j += kThreads) {
    Acc a0 = Acc(0), a1 = Acc(0), a2 = Acc(0), a3 = Acc(0);
    int i = 0;
    for (; i + 4 <= m; i += 4) {
      a0 += (Acc)V.A[(size_t)i * ld + j] * (Acc)y[i];
      a1 += (Acc)V.A[(size_t)(i + 1) * ld + j] * (Acc)y[i + 1];
      a2 += (Acc)V.A[(size_t)(i + 2) * ld + j] * (Acc)y[i + 2];
      a3 += (Acc)V.A[(size_t)(i + 3) * ld + j] * (Acc)y[i + 3];
    }
    for (; i < m; ++i) a0 += (Acc)V.A[(size_t)i * ld + j] * (Acc)y[i];
    const Acc aty = (a0 + a1) + (a2 + a3);
    const Acc sj = (Acc)s[j], cj = (Acc)V.c[j], cb = (Acc)V.cbar[j], xj = (Acc)x[j];
    const Acc rx = -aty + cj * ta - cb * th - sj;
    const Acc dr = (aty + sj) / ta - cj;
    acc[0] += rx * rx; acc[2] += dr * dr; acc[4] += (aty + sj) * (aty + sj);
    acc[7] += cj * xj; acc[8] += cb * xj;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) out[k] = (double)acc[k];
  block_allsum<9>(out, red);
}

// Sec. 4.3 spectral estimate from the dot products d = (<dv,dv>, <dv,du~>, <du~,du~>,
// <dv,du>, <du,du>) of the curvature pairs: for each pair the steepest-descent and
// minimum-gradient steps SD = <dv,dv>/<dv,d>, MG = <dv,d>/<d,d>, their hybrid (MG when
// 2 MG > SD, else SD - MG/2) and the correlation <dv,d>/(|dv||d|); the safeguard keeps the
// estimates whose correlation exceeds eps_cor (both: their geometric mean) and returns
// beta when neither does.
__device__ double bb_estimate(const double* d, double beta, double eps_cor) {
  const double vv = d[0], nv = sqrt(vv);
  auto pair = [&](double vd, double dd, double& step) -> double {
    if (vd == 0.0 || dd == 0.0 || nv == 0.0) { step = 0.0; return -1.0; }
    const double sd = vv / vd, mg = vd / dd;
    step = 2.0 * mg > sd ? mg : sd - mg / 2.0;
    return vd / (nv * sqrt(dd));
  };
  double phi, psi;
  const double phi_cor = pair(d[1], d[2], phi);
  const double psi_cor = pair(d[3], d[4], psi);
  if (phi_cor > eps_cor && psi_cor > eps_cor) return sqrt(phi * psi);
  if (phi_cor > eps_cor) return phi;
  if (psi_cor > eps_cor) return psi;
  return beta;
}

// Algorithm 2 for one instance with the CTA, FP64 iterates (T = double).  Shared
// layout: y, zy, w, Ax, As (m each), x, s, zx (n each).
template <typename T>
__device__ void dense_solve_one(DenseInst& I, const DenseParams& P, T* sm, double* red) {
  const DView<T> V = view(I, T(0));
  const int m = I.m, n = I.n;
  T* y = sm;
  T* zy = y + m;
  T* w = zy + m;
  T* Ax = w + m;
  T* As = Ax + m;
  T* x = As + m;
  T* s = x + n;
  T* zx = s + n;
  const double alpha = P.alpha, beta = P.beta, gamma = P.gamma, eps = P.eps;
  const double zbar = I.zbar, xi = -(double)n - 1.0, nb = I.nb, nc = I.nc;
  const double Ki0 = I.Kinv[0], Ki1 = I.Kinv[1], Ki2 = I.Kinv[2], Ki3 = I.Kinv[3];
  // start of Algorithm 2, or a state loaded by abip_set_state
  double tau = 1.0, kappa = 1.0, theta = 1.0, mu = beta;
  int64_t total = 0;
  int outer = 0, status = 0;
  if (I.resume) {
    for (int i = threadIdx.x; i < m; i += kThreads) y[i] = (T)I.y[i];
    for (int j = threadIdx.x; j < n; j += kThreads) { x[j] = (T)I.x[j]; s[j] = (T)I.s[j]; }
    tau = I.r_tau; kappa = I.r_kappa; theta = I.r_theta; mu = I.r_mu;
    total = I.r_iters;
    outer = I.r_outer;
  } else {
    for (int i = threadIdx.x; i < m; i += kThreads) y[i] = T(0);
    for (int j = threadIdx.x; j < n; j += kThreads) { x[j] = T(1); s[j] = T(1); }
  }
  __syncthreads();
  double inner2 = 0, pres = 0, dres = 0, dgap = 0, ctx = 0, bty = 0;

  // Sec. 4.1 tests on the sums; returns the status they give (0 = continue)
  auto tests = [&](const double (&a)[9], double margin) -> int {
    const double ps = sqrt(a[1]) / (1.0 + nb), ds = sqrt(a[2]) / (1.0 + nc);
    const double gp = fabs(a[7] / tau - a[5] / tau) / (1.0 + fabs(a[7] / tau) + fabs(a[5] / tau));
    if (ps <= margin * eps && ds <= margin * eps && gp <= margin * eps) return ABIP_OPTIMAL;
    if (a[5] > 0 && sqrt(a[4]) <= margin * eps * a[5] / nb) return ABIP_PRIMAL_INFEASIBLE;
    if (a[7] < 0 && sqrt(a[3]) <= margin * eps * (-a[7]) / nc) return ABIP_DUAL_INFEASIBLE;
    return 0;
  };
  auto absorb = [&](const double (&a)[9]) {
    bty = a[5];
    ctx = a[7];
    const double rt = a[5] - a[7] + zbar * theta - kappa;
    const double rth = -a[6] + a[8] - zbar * tau - xi;
    inner2 = a[0] + rt * rt + rth * rth;
    pres = sqrt(a[1]) / (1.0 + nb);
    dres = sqrt(a[2]) / (1.0 + nc);
    dgap = fabs(ctx / tau - bty / tau) / (1.0 + fabs(ctx / tau) + fabs(bty / tau));
  };
  auto evaluate = [&](bool final_test) -> bool {
    double a[9];
    residual_sums<T>(V, m, n, I.ld, x, s, y, tau, theta, Ax, As, a, red);
    absorb(a);
    if (!isfinite(inner2)) return false;
    if (!final_test || P.stop_rule != 0) return true;
    status = tests(a, 1.0);
    return true;
  };

  // One ADMM update with barrier weight bk (Algorithm 2 with the relaxation of Sec. 4.2),
  // from the state and its products Ax, As.  ut (global, m + n, may be null) receives the
  // projection u~ = (u~_y, u~_x); (t1, t2) = (u~_tau, u~_theta).
  double t1 = 0.0, t2 = 0.0;
  auto admm_update = [&](double bk, double* ut) {
    // projection: w_y = y, w_x = x + s; zy = G^{-1}(y - A(x + s)) = G^{-1}(y - Ax - As)
    for (int i = threadIdx.x; i < m; i += kThreads) zy[i] = y[i] - (Ax[i] + As[i]);
    for (int j = threadIdx.x; j < n; j += kThreads) zx[j] = x[j] + s[j];
    __syncthreads();
    trsv_lower<T>(V.L, m, zy);
    trsv_lower_t<T>(V.L, m, zy);
    // zx = w_x + A^T zy, and H^T z
    T hz0 = T(0), hz1 = T(0);
    for (int j = threadIdx.x; j < n; j += kThreads) {
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      int i = 0;
      for (; i + 4 <= m; i += 4) {
        a0 += V.A[(size_t)i * I.ld + j] * zy[i];
        a1 += V.A[(size_t)(i + 1) * I.ld + j] * zy[i + 1];
        a2 += V.A[(size_t)(i + 2) * I.ld + j] * zy[i + 2];
        a3 += V.A[(size_t)(i + 3) * I.ld + j] * zy[i + 3];
      }
      for (; i < m; ++i) a0 += V.A[(size_t)i * I.ld + j] * zy[i];
      const T z = zx[j] + ((a0 + a1) + (a2 + a3));
      zx[j] = z;
      hz0 += V.c[j] * z;
      hz1 -= V.cbar[j] * z;
    }
    for (int i = threadIdx.x; i < m; i += kThreads) {
      hz0 -= V.b[i] * zy[i];
      hz1 += V.bbar[i] * zy[i];
    }
    double hz[2] = {(double)hz0, (double)hz1};
    block_allsum<2>(hz, red);
    const double v1 = tau + kappa + hz[0], v2 = theta + xi + hz[1];
    t1 = Ki0 * v1 + Ki1 * v2;
    t2 = Ki2 * v1 + Ki3 * v2;
    const T a = (T)alpha, a1 = (T)(1.0 - alpha), t1T = (T)t1, t2T = (T)t2, cmu = (T)(mu / bk);
    for (int i = threadIdx.x; i < m; i += kThreads) {
      const T uy = zy[i] - V.g1[i] * t1T - V.g2[i] * t2T;
      if (ut) ut[i] = (double)uy;
      y[i] = a * uy + a1 * y[i];
    }
    for (int j = threadIdx.x; j < n; j += kThreads) {
      const T ux = zx[j] - V.g1[m + j] * t1T - V.g2[m + j] * t2T;
      if (ut) ut[m + j] = (double)ux;
      const T xh = a * ux + a1 * x[j];
      T xn, sn;
      barrier_step<T>(xh - s[j], cmu, xn, sn);
      x[j] = xn;
      s[j] = sn;
    }
    {
      const double th_ = alpha * t1 + (1.0 - alpha) * tau;
      double tn, kn;
      barrier_step<double>(th_ - kappa, mu / bk, tn, kn);
      tau = tn;
      kappa = kn;
      theta = alpha * t2 + (1.0 - alpha) * theta;
    }
    __syncthreads();
  };

  // Sec. 4.3 at the start of an outer iteration k >= 1 (readings B5, B7): from the start point S0, two
  // trial updates with beta_k give the curvature pairs
  //   dv = v^_2 - v^_1, v^_i = v_{i-1} - alpha u~_i - (1 - alpha) u_{i-1} + alpha u_i,
  //   du~ = alpha (u~_2 - u~_1) + (1 - alpha) (u_1 - u_0),  du = -(u_2 - u_1)
  // (u = (y, x, tau, theta), v = (r, s, kappa, xi), r = 0 and xi fixed); the safeguarded
  // spectral estimate beta^ (bb_estimate) keeps beta_k (no reliable curvature), averages
  // it with beta^ (|beta^ - beta_k| <= eps_penalty), or becomes the new beta_k for a redo
  // from S0.  At most bb_max_redo redos, and no round that would pass `budget` updates;
  // the iteration continues from the last trial state.  Returns the updates spent.
  double beta_k = beta;
  auto bb_select = [&](int64_t budget) -> int64_t {
    double* S0 = I.work;            // y0, x0, s0
    double* S1 = S0 + m + 2 * n;    // y1, x1, s1
    double* U1 = S1 + m + 2 * n;    // u~_1 (y, x parts)
    double* U2 = U1 + m + n;        // u~_2
    for (int i = threadIdx.x; i < m; i += kThreads) S0[i] = (double)y[i];
    for (int j = threadIdx.x; j < n; j += kThreads) { S0[m + j] = (double)x[j]; S0[m + n + j] = (double)s[j]; }
    const double tau0 = tau, kappa0 = kappa, theta0 = theta;
    double b = beta_k, used = beta_k;
    int64_t spent = 0;
    for (int round = 0; round <= P.bb_max_redo; ++round) {
      if (spent + 2 > budget) break;
      if (round > 0) {
        for (int i = threadIdx.x; i < m; i += kThreads) y[i] = (T)S0[i];
        for (int j = threadIdx.x; j < n; j += kThreads) { x[j] = (T)S0[m + j]; s[j] = (T)S0[m + n + j]; }
        tau = tau0; kappa = kappa0; theta = theta0;
      }
      __syncthreads();
      gemv_rows<true, T>(V.A, I.ld, m, n, x, s, Ax, As);
      __syncthreads();
      admm_update(b, U1);
      const double ut1 = t1, uth1 = t2, tau1 = tau, kappa1 = kappa, theta1 = theta;
      for (int i = threadIdx.x; i < m; i += kThreads) S1[i] = (double)y[i];
      for (int j = threadIdx.x; j < n; j += kThreads) { S1[m + j] = (double)x[j]; S1[m + n + j] = (double)s[j]; }
      gemv_rows<true, T>(V.A, I.ld, m, n, x, s, Ax, As);
      __syncthreads();
      admm_update(b, U2);
      spent += 2;
      used = b;
      // <dv,dv>, <dv,du~>, <du~,du~>, <dv,du>, <du,du>
      double d[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      auto add = [&](double u0, double u1, double u2, double w1, double w2, double v0, double v1) {
        const double vh1 = v0 - alpha * w1 - (1.0 - alpha) * u0 + alpha * u1;
        const double vh2 = v1 - alpha * w2 - (1.0 - alpha) * u1 + alpha * u2;
        const double dv = vh2 - vh1;
        const double dt = alpha * (w2 - w1) + (1.0 - alpha) * (u1 - u0);
        const double du = -(u2 - u1);
        d[0] += dv * dv; d[1] += dv * dt; d[2] += dt * dt; d[3] += dv * du; d[4] += du * du;
      };
      for (int i = threadIdx.x; i < m; i += kThreads) add(S0[i], S1[i], (double)y[i], U1[i], U2[i], 0.0, 0.0);
      for (int j = threadIdx.x; j < n; j += kThreads)
        add(S0[m + j], S1[m + j], (double)x[j], U1[m + j], U2[m + j], S0[m + n + j], S1[m + n + j]);
      if (threadIdx.x == 0) {
        add(tau0, tau1, tau, ut1, t1, kappa0, kappa1);     // tau position: v = kappa
        add(theta0, theta1, theta, uth1, t2, xi, xi);      // theta position: v = xi
      }
      block_allsum<5>(d, red);
      const double bh = bb_estimate(d, b, P.eps_cor);
      if (bh == b) { beta_k = b; return spent; }   // no reliable curvature: keep this round's beta
      if (fabs(bh - b) <= P.eps_penalty) { beta_k = 0.5 * (b + bh); return spent; }
      b = bh;
    }
    beta_k = used;
    return spent;
  };
  // the start of an outer iteration: the selection of beta (when on), then the sums of the
  // state; false stops the solve (non-finite sums, or the selection reached the cap)
  auto outer_start = [&]() -> bool {
    // reading B7: from the second outer iteration on (the first starts at the exact central
    // point of mu0 = beta, a fixed point of the ADMM map: its curvature pairs are rounding noise)
    if (P.bb && outer >= 1 && total + 2 <= P.max_admm) {
      total += bb_select(P.max_admm - total);
      if (total >= P.max_admm) {
        status = ABIP_MAX_ITER;
        double a[9];
        residual_sums<T>(V, m, n, I.ld, x, s, y, tau, theta, Ax, As, a, red);
        absorb(a);
        return false;
      }
    }
    return evaluate(false);
  };

  bool ok = outer_start();
  while (ok) {
    if (inner2 <= mu) {
      const double gk = adaptive_gamma(gamma, P.gamma_max, eps, fmax(pres, fmax(dres, dgap)));
      mu *= gk;
      ++outer;
      if (P.stop_rule == 1 && mu < eps) { status = ABIP_OPTIMAL; break; }
      if (outer >= kMaxOuter) { status = ABIP_MAX_ITER; break; }   // mu has underflowed
      const T g = (T)gk, sg = (T)sqrt(gk);
      if (P.warmstart == 1) {
        for (int j = threadIdx.x; j < n; j += kThreads) { x[j] *= sg; s[j] *= sg; }
        tau *= sqrt(gk); kappa *= sqrt(gk);
      } else {
        for (int j = threadIdx.x; j < n; j += kThreads) {
          if (x[j] >= s[j]) s[j] *= g; else x[j] *= g;
        }
        if (tau >= kappa) kappa *= gk; else tau *= gk;
      }
      for (int i = threadIdx.x; i < m; i += kThreads) y[i] *= sg;
      theta *= sqrt(gk);
      __syncthreads();
      ok = outer_start();
      continue;
    }
    admm_update(beta_k, nullptr);
    ++total;
    ok = evaluate(true);
    if (status != 0) break;
    if (total >= P.max_admm) { status = ABIP_MAX_ITER; break; }
  }
  // outputs: raw state and the scaled candidate or certificate (Sec. 4.1)
  double sx = 1.0 / tau, sy = 1.0 / tau;
  if (status == ABIP_PRIMAL_INFEASIBLE) { sx = 1.0; sy = 1.0 / bty; }
  if (status == ABIP_DUAL_INFEASIBLE) { sx = -1.0 / ctx; sy = 1.0; }
  for (int i = threadIdx.x; i < m; i += kThreads) {
    I.y[i] = (double)y[i];
    if (I.out_y) I.out_y[i] = (double)y[i] * sy;
  }
  for (int j = threadIdx.x; j < n; j += kThreads) {
    I.x[j] = (double)x[j];
    I.s[j] = (double)s[j];
    if (I.out_x) I.out_x[j] = (double)x[j] * sx;
    if (I.out_s) I.out_s[j] = (double)s[j] * sy;
  }
  if (threadIdx.x == 0) {
    I.tau = tau; I.kappa = kappa; I.theta = theta; I.mu = mu;
    I.resume = 0;
    I.pres = pres; I.dres = dres; I.dgap = dgap; I.ctx = ctx; I.bty = bty; I.obj = ctx / tau;
    I.admm_iters = total; I.outer_iters = outer; I.status = status;
    I.beta_last = beta_k;
    // ok is also false when the trial updates of the selection reached the cap (finite sums)
    if (!ok && !(status == ABIP_MAX_ITER && isfinite(inner2))) I.err = DEV_ERR_NONFINITE;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Mixed precision: FP64 state, FP32 products of changes
// ---------------------------------------------------------------------------
// The iterate (y, x, s, tau, kappa, theta) and the products the update needs
// (Ax, As, A^T y, z_y = G^{-1} q with q = y - Ax - As, A^T z_y) are kept in FP64.  Each
// update changes them by FP32 products of the change of the iterate:
//   z_y += G^{-1} (q - q_prev)            (FP32, with the explicit inverse formed at setup)
//   A^T z_y += A^T (G^{-1} (q - q_prev))   (FP32)
//   Ax += A dx, As += A ds, A^T y += A^T dy (FP32, after the update)
// so FP32 rounding scales with the step, not with the iterate, and there is no FP32
// accuracy floor.  Every kDeltaRefresh updates, and whenever the Sec. 4.1 tests pass on
// the maintained sums with a factor-4 margin, the products are recomputed exactly in
// FP64; the tests are decided on the exact sums.
constexpr int kDeltaRefresh = 100;

// o0[i] += sum_j M[i][j] v0[j] (and o1 with v1) for rows i < rows: each warp takes four
// rows at a time (rows w, w + 8, w + 16, w + 24 of a group of 32), float4 loads, FP32
// accumulation, so that four rows' loads are in flight per warp.  M rows are ldm floats
// (a multiple of 4, zero padded); v0, v1 hold ldm floats, 16-byte aligned.  f0
// (optional) receives the FP32 row sums.
template <bool TWO>
__device__ void rows_f32(const float* __restrict__ M, int ldm, int rows, const float* v0, const float* v1,
                         double* o0, double* o1, float* f0) {
  constexpr int R = 4;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nq = ldm / 4;
  const float4* p0 = reinterpret_cast<const float4*>(v0);
  const float4* p1 = reinterpret_cast<const float4*>(v1);
  for (int g = 0; g < rows; g += R * kWarps) {
    float a0[R], a1[R];
    const float4* r[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      a0[q] = 0.f;
      a1[q] = 0.f;
      const int i = g + wid + q * kWarps;
      r[q] = reinterpret_cast<const float4*>(M + (size_t)min(i, rows - 1) * ldm);
    }
    for (int t = lane; t < nq; t += 32) {
      const float4 x = p0[t];
      float4 z = x;
      if (TWO) z = p1[t];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const float4 a = r[q][t];
        a0[q] += a.x * x.x + a.y * x.y + a.z * x.z + a.w * x.w;
        if (TWO) a1[q] += a.x * z.x + a.y * z.y + a.z * z.z + a.w * z.w;
      }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = g + wid + q * kWarps;
      const float s0 = warp_sum(a0[q]);
      const float s1 = TWO ? warp_sum(a1[q]) : 0.f;
      if (lane == 0 && i < rows) {
        o0[i] += (double)s0;
        if (TWO) o1[i] += (double)s1;
        if (f0) f0[i] = s0;
      }
    }
  }
}

__device__ void dense_solve_delta(DenseInst& I, const DenseParams& P, unsigned char* smraw, double* red) {
  const int m = I.m, n = I.n;
  const int64_t ld = I.ld;
  double* y = reinterpret_cast<double*>(smraw);
  double* Ax = y + m;
  double* As = Ax + m;
  double* zy = As + m;
  double* qp = zy + m;
  double* x = qp + m;
  double* s = x + n;
  double* ATy = s + n;
  double* ATz = ATy + n;
  const int mp = I.ldtf, np = I.ldf;
  float* dy = reinterpret_cast<float*>(smraw + (((size_t)(5 * m + 4 * n) * 8 + 15) / 16) * 16);
  float* dq = dy + mp;
  float* dz = dq + mp;
  float* dx = dz + mp;
  float* ds = dx + np;
  const double alpha = P.alpha, beta = P.beta, gamma = P.gamma, eps = P.eps;
  const double zbar = I.zbar, xi = -(double)n - 1.0, nb = I.nb, nc = I.nc;
  const double Ki0 = I.Kinv[0], Ki1 = I.Kinv[1], Ki2 = I.Kinv[2], Ki3 = I.Kinv[3];
  double tau = 1.0, kappa = 1.0, theta = 1.0, mu = beta;
  int64_t total = 0;
  int outer = 0, status = 0;
  if (I.resume) {
    for (int i = threadIdx.x; i < m; i += kThreads) y[i] = I.y[i];
    for (int j = threadIdx.x; j < n; j += kThreads) { x[j] = I.x[j]; s[j] = I.s[j]; }
    tau = I.r_tau; kappa = I.r_kappa; theta = I.r_theta; mu = I.r_mu;
    total = I.r_iters;
    outer = I.r_outer;
  } else {
    for (int i = threadIdx.x; i < m; i += kThreads) y[i] = 0.0;
    for (int j = threadIdx.x; j < n; j += kThreads) { x[j] = 1.0; s[j] = 1.0; }
  }
  // the padding of the FP32 vectors meets zero padding of the FP32 matrices
  for (int i = threadIdx.x; i < 3 * mp + 2 * np; i += kThreads) dy[i] = 0.f;
  __syncthreads();
  int64_t since_refresh = 0, next_confirm = 0;
  double inner2 = 0, pres = 0, dres = 0, dgap = 0, ctx = 0, bty = 0;

  // exact FP64 products of the current state
  auto refresh = [&]() {
    gemv_rows<true, double>(I.A, ld, m, n, x, s, Ax, As);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += kThreads) {
      const double q = y[i] - (Ax[i] + As[i]);
      qp[i] = q;
      zy[i] = q;
    }
    __syncthreads();
    trsv_lower<double>(I.L, m, zy);
    trsv_lower_t<double>(I.L, m, zy);
    for (int j = threadIdx.x; j < n; j += kThreads) {
      double a0 = 0.0, a1 = 0.0;
      for (int i = 0; i < m; ++i) {
        const double aij = I.A[(size_t)i * ld + j];
        a0 += aij * y[i];
        a1 += aij * zy[i];
      }
      ATy[j] = a0;
      ATz[j] = a1;
    }
    __syncthreads();
    since_refresh = 0;
  };
  // the nine sums from the maintained products (as residual_sums)
  auto sums = [&](double (&out)[9]) {
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double itau = 1.0 / tau;
    for (int i = threadIdx.x; i < m; i += kThreads) {
      const double ax = Ax[i], bi = I.b[i], yi = y[i], bb = I.bbar[i];
      const double ry = ax - bi * tau + bb * theta;
      const double pr = ax * itau - bi;
      acc[0] += ry * ry; acc[1] += pr * pr; acc[3] += ax * ax;
      acc[5] += bi * yi; acc[6] += bb * yi;
    }
    for (int j = threadIdx.x; j < n; j += kThreads) {
      const double aty = ATy[j], sj = s[j], cj = I.c[j], cb = I.cbar[j], xj = x[j];
      const double rx = -aty + cj * tau - cb * theta - sj;
      const double dr = (aty + sj) * itau - cj;
      acc[0] += rx * rx; acc[2] += dr * dr; acc[4] += (aty + sj) * (aty + sj);
      acc[7] += cj * xj; acc[8] += cb * xj;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = acc[k];
    block_allsum<9>(out, red);
  };
  auto tests = [&](const double (&a)[9], double margin) -> int {
    const double ps = sqrt(a[1]) / (1.0 + nb), dsn = sqrt(a[2]) / (1.0 + nc);
    const double gp = fabs(a[7] / tau - a[5] / tau) / (1.0 + fabs(a[7] / tau) + fabs(a[5] / tau));
    if (ps <= margin * eps && dsn <= margin * eps && gp <= margin * eps) return ABIP_OPTIMAL;
    if (a[5] > 0 && sqrt(a[4]) <= margin * eps * a[5] / nb) return ABIP_PRIMAL_INFEASIBLE;
    if (a[7] < 0 && sqrt(a[3]) <= margin * eps * (-a[7]) / nc) return ABIP_DUAL_INFEASIBLE;
    return 0;
  };
  auto absorb = [&](const double (&a)[9]) {
    bty = a[5];
    ctx = a[7];
    const double rt = a[5] - a[7] + zbar * theta - kappa;
    const double rth = -a[6] + a[8] - zbar * tau - xi;
    inner2 = a[0] + rt * rt + rth * rth;
    pres = sqrt(a[1]) / (1.0 + nb);
    dres = sqrt(a[2]) / (1.0 + nc);
    dgap = fabs(ctx / tau - bty / tau) / (1.0 + fabs(ctx / tau) + fabs(bty / tau));
  };
  auto evaluate = [&](bool final_test) -> bool {
    double a[9];
    sums(a);
    absorb(a);
    if (!isfinite(inner2)) return false;
    if (!final_test || P.stop_rule != 0) return true;
    if (total >= next_confirm && tests(a, 4.0) != 0) {
      refresh();
      sums(a);
      absorb(a);
      status = tests(a, 1.0);
      next_confirm = total + P.check_every;
    }
    return true;
  };
  // maintained products after a change (dy, dx, ds) of the iterate
  auto maintain = [&]() {
    rows_f32<true>(I.Af, np, m, dx, ds, Ax, As, nullptr);
    rows_f32<false>(I.ATf, mp, n, dy, dy, ATy, ATy, nullptr);
    __syncthreads();
  };

  refresh();
  bool ok = evaluate(false);
  while (ok) {
    if (inner2 <= mu) {
      const double gk = adaptive_gamma(gamma, P.gamma_max, eps, fmax(pres, fmax(dres, dgap)));
      mu *= gk;
      ++outer;
      if (P.stop_rule == 1 && mu < eps) { status = ABIP_OPTIMAL; break; }
      if (outer >= kMaxOuter) { status = ABIP_MAX_ITER; break; }
      const double sg = sqrt(gk);
      for (int j = threadIdx.x; j < n; j += kThreads) {
        const double x0 = x[j], s0 = s[j];
        if (P.warmstart == 1) { x[j] = x0 * sg; s[j] = s0 * sg; }
        else if (x0 >= s0) s[j] = s0 * gk;
        else x[j] = x0 * gk;
        dx[j] = (float)(x[j] - x0);
        ds[j] = (float)(s[j] - s0);
      }
      if (P.warmstart == 1) { tau *= sg; kappa *= sg; }
      else if (tau >= kappa) kappa *= gk;
      else tau *= gk;
      for (int i = threadIdx.x; i < m; i += kThreads) {
        const double y0 = y[i];
        y[i] = y0 * sg;
        dy[i] = (float)(y[i] - y0);
      }
      theta *= sg;
      __syncthreads();
      maintain();
      ok = evaluate(false);
      continue;
    }
    // projection on the change of q = y - A(x + s)
    for (int i = threadIdx.x; i < m; i += kThreads) {
      const double q = y[i] - (Ax[i] + As[i]);
      dq[i] = (float)(q - qp[i]);
      qp[i] = q;
    }
    __syncthreads();
    // zy += G^{-1} dq (dz keeps the FP32 change), A^T zy += A^T dz
    rows_f32<false>(I.Ginvf, mp, m, dq, dq, zy, zy, dz);
    __syncthreads();
    rows_f32<false>(I.ATf, mp, n, dz, dz, ATz, ATz, nullptr);
    __syncthreads();
    double hz[2] = {0.0, 0.0};
    for (int j = threadIdx.x; j < n; j += kThreads) {
      const double z = x[j] + s[j] + ATz[j];
      hz[0] += I.c[j] * z;
      hz[1] -= I.cbar[j] * z;
    }
    for (int i = threadIdx.x; i < m; i += kThreads) {
      hz[0] -= I.b[i] * zy[i];
      hz[1] += I.bbar[i] * zy[i];
    }
    block_allsum<2>(hz, red);
    const double v1 = tau + kappa + hz[0], v2 = theta + xi + hz[1];
    const double t1 = Ki0 * v1 + Ki1 * v2, t2 = Ki2 * v1 + Ki3 * v2;
    const double cmu = mu / beta;
    for (int i = threadIdx.x; i < m; i += kThreads) {
      const double uy = zy[i] - I.g1[i] * t1 - I.g2[i] * t2;
      const double y0 = y[i];
      y[i] = alpha * uy + (1.0 - alpha) * y0;
      dy[i] = (float)(y[i] - y0);
    }
    for (int j = threadIdx.x; j < n; j += kThreads) {
      const double z = x[j] + s[j] + ATz[j];
      const double ux = z - I.g1[m + j] * t1 - I.g2[m + j] * t2;
      const double x0 = x[j], s0 = s[j];
      const double xh = alpha * ux + (1.0 - alpha) * x0;
      double xn, sn;
      barrier_step_newton(xh - s0, cmu, xn, sn);   // few FP64 operations (the FP64 pipe binds here)
      x[j] = xn;
      s[j] = sn;
      dx[j] = (float)(xn - x0);
      ds[j] = (float)(sn - s0);
    }
    {
      const double th_ = alpha * t1 + (1.0 - alpha) * tau;
      double tn, kn;
      barrier_step<double>(th_ - kappa, mu / beta, tn, kn);
      tau = tn;
      kappa = kn;
      theta = alpha * t2 + (1.0 - alpha) * theta;
    }
    __syncthreads();
    maintain();
    ++total;
    if (++since_refresh >= kDeltaRefresh) refresh();
    ok = evaluate(true);
    if (status != 0) break;
    if (total >= P.max_admm) { status = ABIP_MAX_ITER; break; }
  }
  // outputs: raw state and the scaled candidate or certificate (Sec. 4.1)
  double sx = 1.0 / tau, sy = 1.0 / tau;
  if (status == ABIP_PRIMAL_INFEASIBLE) { sx = 1.0; sy = 1.0 / bty; }
  if (status == ABIP_DUAL_INFEASIBLE) { sx = -1.0 / ctx; sy = 1.0; }
  for (int i = threadIdx.x; i < m; i += kThreads) {
    I.y[i] = y[i];
    if (I.out_y) I.out_y[i] = y[i] * sy;
  }
  for (int j = threadIdx.x; j < n; j += kThreads) {
    I.x[j] = x[j];
    I.s[j] = s[j];
    if (I.out_x) I.out_x[j] = x[j] * sx;
    if (I.out_s) I.out_s[j] = s[j] * sy;
  }
  if (threadIdx.x == 0) {
    I.tau = tau; I.kappa = kappa; I.theta = theta; I.mu = mu;
    I.resume = 0;
    I.pres = pres; I.dres = dres; I.dgap = dgap; I.ctx = ctx; I.bty = bty; I.obj = ctx / tau;
    I.admm_iters = total; I.outer_iters = outer; I.status = status;
    I.fp32_iters_lo = (int32_t)(total & 0x7fffffff);
    I.fp32_iters_hi = (int32_t)(total >> 31);
    if (!ok) I.err = DEV_ERR_NONFINITE;
  }
  __syncthreads();
}

// Solve kernels, one CTA per instance at a time.  MINB (resident CTAs per SM the
// compiler plans registers for) is the knob of the batch autotuner: the variants run the
// same arithmetic and differ only in occupancy.
template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB) dense_solve_mixed_kernel(DenseInst* insts, int count,
                                                                           DenseParams P, int* queue,
                                                                           const int* order) {
  extern __shared__ double sm_raw[];
  __shared__ double red[32 * 9];
  for (;;) {
    const int id = next_instance(queue, count, order);
    if (id < 0) return;
    DenseInst& I = insts[id];
    if (I.err != 0) continue;
    dense_solve_delta(I, P, reinterpret_cast<unsigned char*>(sm_raw), red);
  }
}

template <typename T, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) dense_solve_kernel(DenseInst* insts, int count, DenseParams P,
                                                                     int* queue, const int* order) {
  extern __shared__ double sm_raw[];
  __shared__ double red[32 * 9];
  T* sm = reinterpret_cast<T*>(sm_raw);
  for (;;) {
    const int id = next_instance(queue, count, order);
    if (id < 0) return;
    DenseInst& I = insts[id];
    if (I.err != 0) continue;
    dense_solve_one<T>(I, P, sm, red);
  }
}

// ---------------------------------------------------------------------------
// Differentiation at the central point (system HSD-log-kkt), one CTA per instance
// ---------------------------------------------------------------------------
// Unknowns z = (y, x, tau, theta, s, kappa); F(z) = (Q u - v with r = 0 and xi = -n-1;
// x o s - cm e; tau kappa - cm), cm = mu / beta.  Eliminating ds = (r5 - S dx) / X and
// dkappa = (r6 - kappa dtau) / tau from J dz = r leaves K (dy, dx, dtau, dtheta) =
// (r1, r2 + r5 / x, r3 + r6 / tau, r4) with
//   K = Q + diag(0, S X^{-1}, kappa / tau, 0)      (order m + n + 2),
// and the adjoint J^T lam = g reduces to K^T (lam1, lam2, lam3, lam4) =
// (g1, g2 - S X^{-1} g5, g3 - kappa g6 / tau, g4).  K is factored by LU with partial
// pivoting in FP64: unlike the normal equations A X S^{-1} A^T, whose condition number
// grows like 1/mu^2 on degenerate LPs, K's grows like that of J itself.

// Block argmax of |v| over this thread's candidates (ties: smaller index); broadcast.
__device__ int block_argmax(double v, int idx, double* red, int* redi) {
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = v; redi[threadIdx.x >> 5] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = red[0];
    int bi = redi[0];
    for (int k = 1; k < kWarps; ++k)
      if (red[k] > bv || (red[k] == bv && redi[k] < bi)) { bv = red[k]; bi = redi[k]; }
    red[32] = bv;
    redi[32] = bi;
  }
  __syncthreads();
  const int r = redi[32];
  __syncthreads();
  return r;
}

// In-place LU with partial pivoting of the N x N row-major K (P K = L U, L unit lower),
// right-looking with 32-column panels; the trailing update runs as 64 x 64 tiles through
// shared memory (16 x 16 threads, 4 x 4 outputs each).  ipiv[k] = row swapped with k.
// Returns false on an exactly zero pivot.
__device__ bool lu_factor(double* K, int N, int* ipiv, double* sm, double* red, int* redi) {
  const int tid = threadIdx.x;
  for (int j0 = 0; j0 < N; j0 += 32) {
    const int jb = min(32, N - j0);
    for (int k = j0; k < j0 + jb; ++k) {
      double best = -1.0;
      int bi = N;
      for (int i = k + tid; i < N; i += kThreads) {
        const double v = fabs(K[(size_t)i * N + k]);
        if (v > best) { best = v; bi = i; }
      }
      const int piv = block_argmax(best, bi, red, redi);
      if (tid == 0) ipiv[k] = piv;
      if (piv != k)
        for (int j = tid; j < N; j += kThreads) {
          const double t = K[(size_t)k * N + j];
          K[(size_t)k * N + j] = K[(size_t)piv * N + j];
          K[(size_t)piv * N + j] = t;
        }
      __syncthreads();
      const double p = K[(size_t)k * N + k];
      if (p == 0.0 || !isfinite(p)) return false;
      for (int i = k + 1 + tid; i < N; i += kThreads) K[(size_t)i * N + k] /= p;
      __syncthreads();
      const int nc = j0 + jb - (k + 1);
      if (nc > 0) {
        const int rows = N - k - 1;
        for (int e = tid; e < rows * nc; e += kThreads) {
          const int i = k + 1 + e / nc, j = k + 1 + e % nc;
          K[(size_t)i * N + j] -= K[(size_t)i * N + k] * K[(size_t)k * N + j];
        }
      }
      __syncthreads();
    }
    const int c0 = j0 + jb;
    if (c0 >= N) break;
    // U12 = L11^{-1} K12: one thread per column, L11 from shared memory
    double* L11 = sm;   // 32 x 33
    for (int e = tid; e < jb * jb; e += kThreads) {
      const int r = e / jb, q = e % jb;
      L11[r * 33 + q] = K[(size_t)(j0 + r) * N + j0 + q];
    }
    __syncthreads();
    for (int j = c0 + tid; j < N; j += kThreads) {
      double col[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) col[r] = r < jb ? K[(size_t)(j0 + r) * N + j] : 0.0;
#pragma unroll
      for (int r = 1; r < 32; ++r) {
        double acc = col[r];
#pragma unroll
        for (int q = 0; q < r; ++q) acc -= L11[r * 33 + q] * col[q];
        col[r] = acc;
      }
      for (int r = 1; r < jb; ++r) K[(size_t)(j0 + r) * N + j] = col[r];
    }
    __syncthreads();
    // trailing update K22 -= L21 U12
    double* Lt = sm;             // 64 x 33
    double* Ut = sm + 64 * 33;   // 32 x 65
    const int tr = tid / 16, tc = tid % 16;
    for (int i0 = c0; i0 < N; i0 += 64) {
      for (int k0 = c0; k0 < N; k0 += 64) {
        for (int e = tid; e < 64 * 32; e += kThreads) {
          const int r = e / 32, q = e % 32;
          const int gi = i0 + r;
          Lt[r * 33 + q] = (gi < N && q < jb) ? K[(size_t)gi * N + j0 + q] : 0.0;
        }
        for (int e = tid; e < 32 * 64; e += kThreads) {
          const int q = e / 64, cc = e % 64;
          const int gk = k0 + cc;
          Ut[q * 65 + cc] = (gk < N && q < jb) ? K[(size_t)(j0 + q) * N + gk] : 0.0;
        }
        __syncthreads();
        double acc[4][4] = {};
        for (int q = 0; q < 32; ++q) {
          double lv[4], uv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) lv[a] = Lt[(tr * 4 + a) * 33 + q];
#pragma unroll
          for (int bq = 0; bq < 4; ++bq) uv[bq] = Ut[q * 65 + tc * 4 + bq];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int bq = 0; bq < 4; ++bq) acc[a][bq] += lv[a] * uv[bq];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int gi = i0 + tr * 4 + a;
          if (gi >= N) continue;
#pragma unroll
          for (int bq = 0; bq < 4; ++bq) {
            const int gk = k0 + tc * 4 + bq;
            if (gk < N) K[(size_t)gi * N + gk] -= acc[a][bq];
          }
        }
        __syncthreads();
      }
    }
  }
  return true;
}

// w <- K^{-1} w from the factors of lu_factor.
__device__ void lu_solve(const double* K, int N, const int* ipiv, double* w) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0)
    for (int k = 0; k < N; ++k) {
      const int p = ipiv[k];
      if (p != k) { const double t = w[k]; w[k] = w[p]; w[p] = t; }
    }
  __syncthreads();
  for (int kb = 0; kb < N; kb += 32) {   // L (unit diagonal)
    const int nb = min(32, N - kb);
    if (wid == 0) {
      double wl = lane < nb ? w[kb + lane] : 0.0;
      for (int j = 0; j < nb; ++j) {
        const double wj = __shfl_sync(0xffffffffu, wl, j);
        if (lane > j && lane < nb) wl -= K[(size_t)(kb + lane) * N + kb + j] * wj;
      }
      if (lane < nb) w[kb + lane] = wl;
    }
    __syncthreads();
    const double wb = lane < nb ? w[kb + lane] : 0.0;
    for (int i = kb + nb + wid; i < N; i += kWarps) {
      double a = lane < nb ? K[(size_t)i * N + kb + lane] * wb : 0.0;
      a = warp_sum(a);
      if (lane == 0) w[i] -= a;
    }
    __syncthreads();
  }
  const int nblk = (N + 31) / 32;
  for (int bk = nblk - 1; bk >= 0; --bk) {   // U
    const int kb = bk * 32, nb = min(32, N - kb);
    if (wid == 0) {
      double wl = lane < nb ? w[kb + lane] : 0.0;
      for (int j = nb - 1; j >= 0; --j) {
        if (lane == j) wl = wl / K[(size_t)(kb + j) * N + kb + j];
        const double zj = __shfl_sync(0xffffffffu, wl, j);
        if (lane < j) wl -= K[(size_t)(kb + lane) * N + kb + j] * zj;
      }
      if (lane < nb) w[kb + lane] = wl;
    }
    __syncthreads();
    const double wb = lane < nb ? w[kb + lane] : 0.0;
    for (int i = wid; i < kb; i += kWarps) {
      double a = lane < nb ? K[(size_t)i * N + kb + lane] * wb : 0.0;
      a = warp_sum(a);
      if (lane == 0) w[i] -= a;
    }
    __syncthreads();
  }
}

// w <- K^{-T} w from the same factors (K^T = U^T L^T P).
__device__ void lu_solve_t(const double* K, int N, const int* ipiv, double* w) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int kb = 0; kb < N; kb += 32) {   // U^T (lower, diagonal of U)
    const int nb = min(32, N - kb);
    if (wid == 0) {
      double wl = lane < nb ? w[kb + lane] : 0.0;
      for (int j = 0; j < nb; ++j) {
        if (lane == j) wl = wl / K[(size_t)(kb + j) * N + kb + j];
        const double zj = __shfl_sync(0xffffffffu, wl, j);
        if (lane > j && lane < nb) wl -= K[(size_t)(kb + j) * N + kb + lane] * zj;
      }
      if (lane < nb) w[kb + lane] = wl;
    }
    __syncthreads();
    for (int k = kb + nb + threadIdx.x; k < N; k += kThreads) {
      double a = 0.0;
      for (int j = 0; j < nb; ++j) a += K[(size_t)(kb + j) * N + k] * w[kb + j];
      w[k] -= a;
    }
    __syncthreads();
  }
  const int nblk = (N + 31) / 32;
  for (int bk = nblk - 1; bk >= 0; --bk) {   // L^T (upper, unit diagonal)
    const int kb = bk * 32, nb = min(32, N - kb);
    if (wid == 0) {
      double wl = lane < nb ? w[kb + lane] : 0.0;
      for (int j = nb - 1; j >= 0; --j) {
        const double zj = __shfl_sync(0xffffffffu, wl, j);
        if (lane < j) wl -= K[(size_t)(kb + j) * N + kb + lane] * zj;
      }
      if (lane < nb) w[kb + lane] = wl;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kb; k += kThreads) {
      double a = 0.0;
      for (int j = 0; j < nb; ++j) a += K[(size_t)(kb + j) * N + k] * w[kb + j];
      w[k] -= a;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = N - 1; k >= 0; --k) {
      const int p = ipiv[k];
      if (p != k) { const double t = w[k]; w[k] = w[p]; w[p] = t; }
    }
  __syncthreads();
}

__device__ double block_dot(const double* a, const double* b, int len, double* red) {
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < len; i += kThreads) v[0] += a[i] * b[i];
  block_allsum<1>(v, red);
  return v[0];
}

// Block minimum of one value per thread (result broadcast).
__device__ double block_min(double a, double* red) {
  for (int o = 16; o > 0; o >>= 1) a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = red[0];
    for (int k = 1; k < kWarps; ++k) r = fmin(r, red[k]);
    red[32] = r;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

__device__ void backward_one(BackwardInst& P, double* sm, double* red, int* redi) {
  const int m = P.m, n = P.n, N = m + n + 2;
  const int64_t ld = P.ld;
  const double* A = P.A;
  const double* b = P.b;
  const double* c = P.c;
  const double cm = P.cmu, xi = -(double)n - 1.0;
  double* y = P.y;
  double* x = P.x;
  double* s = P.s;
  double* K = P.K;
  double* bbar = P.work;         // m
  double* F1 = bbar + m;         // m
  double* cbar = F1 + m;         // n
  double* F2 = cbar + n;         // n
  double* F5 = F2 + n;           // n
  double* sig = F5 + n;          // n: S X^{-1}
  double* rhs = sig + n;         // N
  double* sol = rhs + N;         // N
  double* res = sol + N;         // N
  double* tmp = res + N;         // N
  int* ipiv = reinterpret_cast<int*>(tmp + N);   // N
  double tau = P.tau, kappa = P.kappa, theta = P.theta;

  // embedding constants of Eq. bar-b-c-z-re: bbar = b - A e, cbar = c - e, zbar = c^T e + 1
  for (int j = threadIdx.x; j < n; j += kThreads) cbar[j] = c[j] - 1.0;
  for (int j = threadIdx.x; j < n; j += kThreads) tmp[j] = 1.0;
  __syncthreads();
  gemv_rows<false, double>(A, ld, m, n, tmp, tmp, bbar, bbar);
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += kThreads) bbar[i] = b[i] - bbar[i];
  double zs[1] = {0.0};
  for (int j = threadIdx.x; j < n; j += kThreads) zs[0] += c[j];
  block_allsum<1>(zs, red);
  const double zbar = zs[0] + 1.0;

  // F at the current point: F1, F2, F5 kept; the tau, theta and tau-kappa rows in Fs;
  // returns ||F||^2
  auto residual = [&](double (&Fs)[3]) -> double {
    gemv_rows<false, double>(A, ld, m, n, x, x, F1, F1);
    __syncthreads();
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < m; i += kThreads) {
      F1[i] = F1[i] - b[i] * tau + bbar[i] * theta;
      acc[0] += F1[i] * F1[i];
      acc[1] += b[i] * y[i];
      acc[2] += bbar[i] * y[i];
    }
    for (int j = threadIdx.x; j < n; j += kThreads) {
      double aty = 0.0;
      for (int i = 0; i < m; ++i) aty += A[(size_t)i * ld + j] * y[i];
      F2[j] = -aty + c[j] * tau - cbar[j] * theta - s[j];
      F5[j] = x[j] * s[j] - cm;
      acc[0] += F2[j] * F2[j] + F5[j] * F5[j];
      acc[3] += c[j] * x[j];
      acc[4] += cbar[j] * x[j];
    }
    block_allsum<5>(acc, red);
    Fs[0] = acc[1] - acc[3] + zbar * theta - kappa;
    Fs[1] = -acc[2] + acc[4] - zbar * tau - xi;
    Fs[2] = tau * kappa - cm;
    return acc[0] + Fs[0] * Fs[0] + Fs[1] * Fs[1] + Fs[2] * Fs[2];
  };
  // K at the current point, then its LU factors
  auto factor = [&]() -> bool {
    for (int j = threadIdx.x; j < n; j += kThreads) sig[j] = s[j] / x[j];
    const double kt = kappa / tau;
    for (size_t e = threadIdx.x; e < (size_t)N * N; e += kThreads) {
      const int r = (int)(e / N), q = (int)(e % N);
      double v = 0.0;
      if (r < m) {                      // y rows: [0, A, -b, bbar]
        if (q >= m && q < m + n) v = A[(size_t)r * ld + (q - m)];
        else if (q == m + n) v = -b[r];
        else if (q == m + n + 1) v = bbar[r];
      } else if (r < m + n) {           // x rows: [-A^T, S X^{-1}, c, -cbar]
        const int j = r - m;
        if (q < m) v = -A[(size_t)q * ld + j];
        else if (q == r) v = s[j] / x[j];
        else if (q == m + n) v = c[j];
        else if (q == m + n + 1) v = -cbar[j];
      } else if (r == m + n) {          // tau row: [b^T, -c^T, kappa/tau, zbar]
        if (q < m) v = b[q];
        else if (q < m + n) v = -c[q - m];
        else if (q == m + n) v = kt;
        else v = zbar;
      } else {                          // theta row: [-bbar^T, cbar^T, -zbar, 0]
        if (q < m) v = -bbar[q];
        else if (q < m + n) v = cbar[q - m];
        else if (q == m + n) v = -zbar;
      }
      K[e] = v;
    }
    __syncthreads();
    return lu_factor(K, N, ipiv, sm, red, redi);
  };
  // out = K v (sgn = 1) or K^T v (sgn = -1): the skew part Q flips sign, the diagonal stays
  auto kmul = [&](const double* v, double* out, double sgn) {
    const double vt = v[m + n], vth = v[m + n + 1];
    gemv_rows<false, double>(A, ld, m, n, v + m, v + m, out, out);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += kThreads) out[i] = sgn * (out[i] - b[i] * vt + bbar[i] * vth);
    double dd[4] = {0, 0, 0, 0};
    for (int i = threadIdx.x; i < m; i += kThreads) { dd[0] += b[i] * v[i]; dd[1] += bbar[i] * v[i]; }
    for (int j = threadIdx.x; j < n; j += kThreads) {
      double aty = 0.0;
      for (int i = 0; i < m; ++i) aty += A[(size_t)i * ld + j] * v[i];
      out[m + j] = sgn * (-aty + c[j] * vt - cbar[j] * vth) + sig[j] * v[m + j];
      dd[2] += c[j] * v[m + j];
      dd[3] += cbar[j] * v[m + j];
    }
    block_allsum<4>(dd, red);
    if (threadIdx.x == 0) {
      out[m + n] = sgn * (dd[0] - dd[2] + zbar * vth) + (kappa / tau) * vt;
      out[m + n + 1] = sgn * (-dd[1] + dd[3] - zbar * vt);
    }
    __syncthreads();
  };
  // sol = K^{-1} rhs (or K^{-T}) with one step of iterative refinement
  auto refined = [&](double sgn) {
    for (int e = threadIdx.x; e < N; e += kThreads) sol[e] = rhs[e];
    __syncthreads();
    if (sgn > 0) lu_solve(K, N, ipiv, sol);
    else lu_solve_t(K, N, ipiv, sol);
    kmul(sol, tmp, sgn);
    for (int e = threadIdx.x; e < N; e += kThreads) res[e] = rhs[e] - tmp[e];
    __syncthreads();
    if (sgn > 0) lu_solve(K, N, ipiv, res);
    else lu_solve_t(K, N, ipiv, res);
    for (int e = threadIdx.x; e < N; e += kThreads) sol[e] += res[e];
    __syncthreads();
  };

  bool ok = true;
  int steps = 0;
  double Fs[3];
  double fn2 = residual(Fs);
  // Newton to the rounding floor: stop once ||F|| is small and no longer halves
  const double scale2 = (1.0 + tau + kappa) * (1.0 + tau + kappa);
  double prev = INFINITY;
  for (; steps < P.newton_max; ++steps) {
    if (fn2 <= P.newton_tol * P.newton_tol * scale2) break;
    if (fn2 > 0.25 * prev && fn2 <= 1e-20 * scale2) break;
    prev = fn2;
    if (!factor()) { ok = false; break; }
    for (int i = threadIdx.x; i < m; i += kThreads) rhs[i] = -F1[i];
    for (int j = threadIdx.x; j < n; j += kThreads) rhs[m + j] = -F2[j] - F5[j] / x[j];
    if (threadIdx.x == 0) {
      rhs[m + n] = -Fs[0] - Fs[2] / tau;
      rhs[m + n + 1] = -Fs[1];
    }
    __syncthreads();
    refined(1.0);
    const double dtau = sol[m + n], dth = sol[m + n + 1];
    if (!isfinite(dtau) || !isfinite(dth)) { ok = false; break; }
    const double dkap = (-Fs[2] - kappa * dtau) / tau;
    // largest step in (0, 1] keeping x, s, tau, kappa at least 1 % inside the orthant
    double amax = 1.0;
    for (int j = threadIdx.x; j < n; j += kThreads) {
      const double dx = sol[m + j];
      const double ds = (-F5[j] - s[j] * dx) / x[j];
      if (dx < 0) amax = fmin(amax, -0.99 * x[j] / dx);
      if (ds < 0) amax = fmin(amax, -0.99 * s[j] / ds);
    }
    if (threadIdx.x == 0) {
      if (dtau < 0) amax = fmin(amax, -0.99 * tau / dtau);
      if (dkap < 0) amax = fmin(amax, -0.99 * kappa / dkap);
    }
    const double step = block_min(amax, red);
    for (int j = threadIdx.x; j < n; j += kThreads) {
      const double dx = sol[m + j];
      const double ds = (-F5[j] - s[j] * dx) / x[j];
      x[j] += step * dx;
      s[j] += step * ds;
    }
    for (int i = threadIdx.x; i < m; i += kThreads) y[i] += step * sol[i];
    tau += step * dtau;
    theta += step * dth;
    kappa += step * dkap;
    __syncthreads();
    fn2 = residual(Fs);
  }
  if (ok && !factor()) ok = false;
  if (ok) {
    // Adjoint: g = (0, g_x, g_tau, 0, 0, 0) with g_x = dL/dx* / tau and
    // g_tau = -(dL/dx*)^T x / tau^2, so K^T (lam1, lam2, lam3, lam4) = (0, g_x, g_tau, 0)
    for (int i = threadIdx.x; i < m; i += kThreads) rhs[i] = 0.0;
    for (int j = threadIdx.x; j < n; j += kThreads) rhs[m + j] = P.dl_dx[j] / tau;
    const double gtau = -block_dot(P.dl_dx, x, n, red) / (tau * tau);
    if (threadIdx.x == 0) {
      rhs[m + n] = gtau;
      rhs[m + n + 1] = 0.0;
    }
    __syncthreads();
    refined(-1.0);
    const double* l1 = sol;
    const double* l2 = sol + m;
    const double lam3 = sol[m + n], lam4 = sol[m + n + 1];
    if (!isfinite(lam3) || !isfinite(lam4)) ok = false;
    // dL/dp = -lam^T dF/dp (F is affine in A, b, c through bbar, cbar, zbar too)
    if (ok && P.db)
      for (int i = threadIdx.x; i < m; i += kThreads) P.db[i] = -(l1[i] * (theta - tau) + (lam3 - lam4) * y[i]);
    if (ok && P.dc)
      for (int j = threadIdx.x; j < n; j += kThreads)
        P.dc[j] = -(l2[j] * (tau - theta) + lam3 * (theta - x[j]) + lam4 * (x[j] - tau));
    if (ok && P.dA)
      for (int i = 0; i < m; ++i) {
        const double li = l1[i], yi = y[i];
        for (int j = threadIdx.x; j < n; j += kThreads)
          P.dA[(size_t)i * n + j] = -(li * (x[j] - theta) - l2[j] * yi + lam4 * yi);
      }
  }
  if (threadIdx.x == 0) {
    P.fnorm = sqrt(fn2);
    P.steps = steps;
    P.err = ok ? 0 : 1;
    P.tau = tau;
    P.theta = theta;
    P.kappa = kappa;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) dense_backward_kernel(BackwardInst* insts, int count) {
  __shared__ double sm[64 * 33 + 32 * 65];
  __shared__ double red[32 * 5];   // block_allsum<K> needs 32 K doubles; K <= 5 here
  __shared__ int redi[40];
  for (int k = blockIdx.x; k < count; k += gridDim.x) backward_one(insts[k], sm, red, redi);
}

}  // namespace

// dynamic shared memory of the solve kernel: 5m + 3n doubles, at most this many bytes
constexpr size_t kDenseSmemMax = 200 * 1024;

cudaError_t launch_dense_setup(DenseInst* inst, int count, int* queue, int grid, size_t smem, cudaStream_t st) {
  // the caller sizes smem for the largest instance: max(2m + n, 2 * 32 * 33) doubles
  cudaError_t e = cudaFuncSetAttribute(dense_setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmemMax);
  if (e != cudaSuccess) return e;
  dense_setup_kernel<<<grid, kThreads, smem, st>>>(inst, count, queue);
  return cudaGetLastError();
}

// the solve kernel of a precision and an occupancy variant (0, 1, 2: MINB 1, 2, 3 for FP64
// and 2, 3, 4 for mixed precision), with its dynamic shared memory limit raised
using DenseSolveFn = void (*)(DenseInst*, int, DenseParams, int*, const int*);
DenseSolveFn dense_solve_fn(bool mixed, int variant) {
  DenseSolveFn f;
  if (mixed) f = variant == 2 ? dense_solve_mixed_kernel<4> : variant == 1 ? dense_solve_mixed_kernel<3>
                                                                             : dense_solve_mixed_kernel<2>;
  else f = variant == 2 ? dense_solve_kernel<double, 3> : variant == 1 ? dense_solve_kernel<double, 2>
                                                                         : dense_solve_kernel<double, 1>;
  cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmemMax);
  return f;
}

cudaError_t launch_dense_solve(DenseInst* inst, int count, DenseParams prm, int* queue, const int* order,
                               int grid, size_t smem, int variant, cudaStream_t st) {
  // the caller sizes smem for the largest instance: (5m + 3n) doubles (FP64), 48m + 40n bytes (mixed)
  DenseSolveFn f = dense_solve_fn(prm.mixed != 0, variant);
  cudaGetLastError();
  f<<<grid, kThreads, smem, st>>>(inst, count, prm, queue, order);
  return cudaGetLastError();
}

int dense_solve_ctas_per_sm(bool mixed, size_t smem, int variant) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, dense_solve_fn(mixed, variant), kThreads, smem);
  return per;
}

cudaError_t launch_dense_backward(BackwardInst* insts, int count, int grid, cudaStream_t st) {
  dense_backward_kernel<<<grid, kThreads, 0, st>>>(insts, count);
  return cudaGetLastError();
}

int dense_max_ctas(int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return sms;
}

}  // namespace abip

// ===========================================================================
// Allocation-free entry point (abip_solve_dense_noalloc)
// ===========================================================================
// Some callers cannot allocate device memory: code running where cudaMalloc is
// forbidden or unsafe (inside a framework that owns every device allocation
// through its own pool, a real-time loop with a fixed memory budget, a plugin
// that may not grow the process's footprint).  For them this entry point solves
// one small dense LP with every byte of scratch taken from the fixed array
// below; the caller passes its inputs and outputs as device pointers.

namespace {

constexpr int kNoAllocMaxM = 128;    // largest m the fixed scratch holds
constexpr int kNoAllocMaxN = 512;    // largest n
constexpr size_t kBlk = 256;
constexpr size_t rup(size_t b) { return (b + kBlk - 1) / kBlk * kBlk; }
// layout: descriptor | work queue | L (m*m) | seven vector blocks of m + n doubles:
// bbar, cbar, g1, g2, y, x, s
constexpr size_t kOffQueue = rup(sizeof(abip::DenseInst));
constexpr size_t kOffL = kOffQueue + kBlk;
constexpr size_t kOffVec = kOffL + rup((size_t)kNoAllocMaxM * kNoAllocMaxM * sizeof(double));
constexpr size_t kVecBlk = rup((size_t)(kNoAllocMaxM + kNoAllocMaxN) * sizeof(double));
constexpr size_t kNoAllocBytes = kOffVec + 7 * kVecBlk;

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[64] = {};       // device address of the scratch array, per device

}  // namespace

// The scratch of abip_solve_dense_noalloc: 167,680 bytes on every device that loads
// the library, held until the process exits.  Every call uses all of it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

extern "C" ABIP_API int abip_solve_dense_noalloc(int32_t m, int32_t n, const double* A, int64_t ld,
                                                 const double* b, const double* c, const abip_params* p,
                                                 double* x, double* y, double* s, abip_info* info,
                                                 void* stream) {
  using abip::DenseInst;
  if (!A || !b || !c || !x || !y || !s) return abip::noalloc_fail(ABIP_E_INVALID_ARG, "NULL pointer argument");
  if (m < 1 || n < m || ld < n) return abip::noalloc_fail(ABIP_E_DIM, "need 1 <= m <= n and ld >= n");
  if (m > kNoAllocMaxM || n > kNoAllocMaxN)
    return abip::noalloc_fail(ABIP_E_UNSUPPORTED, "abip_solve_dense_noalloc holds at most m = 128, n = 512");
  abip_params prm;
  if (p) prm = *p;
  else abip_default_params(&prm);
  std::string why;
  if (!abip::check_params_internal(prm, why)) return abip::noalloc_fail(ABIP_E_INVALID_ARG, why);
  if (prm.precision != ABIP_PREC_F64) return abip::noalloc_fail(ABIP_E_UNSUPPORTED, "abip_solve_dense_noalloc is FP64 only");
  if (prm.bb_beta) return abip::noalloc_fail(ABIP_E_UNSUPPORTED, "abip_solve_dense_noalloc has no scratch for bb_beta");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return abip::noalloc_fail(ABIP_E_CUDA, "cudaGetDevice failed");
  const void* ptrs[6] = {A, b, c, x, y, s};
  for (const void* q : ptrs) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) ||
        (at.type == cudaMemoryTypeDevice && at.device != dev)) {
      cudaGetLastError();
      return abip::noalloc_fail(ABIP_E_INVALID_ARG, "every array must be device memory of the current device");
    }
  }
  // set-up, once per device, with that device current: the device address of the array
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return abip::noalloc_fail(ABIP_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      g_noalloc_ptr[dev] = ptr;
    }
    base = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DenseInst* dinst = reinterpret_cast<DenseInst*>(base);
  int* queue = reinterpret_cast<int*>(base + kOffQueue);
  double* vec = reinterpret_cast<double*>(base + kOffVec);
  const size_t vstride = kVecBlk / sizeof(double);
  DenseInst I{};
  I.m = m; I.n = n; I.ld = ld;
  I.A = A; I.b = b; I.c = c;
  I.L = reinterpret_cast<double*>(base + kOffL);
  I.bbar = vec; I.cbar = vec + vstride;
  I.g1 = vec + 2 * vstride; I.g2 = vec + 3 * vstride;
  I.y = vec + 4 * vstride; I.x = vec + 5 * vstride; I.s = vec + 6 * vstride;
  I.out_x = x; I.out_y = y; I.out_s = s;
  // I.err, I.status, I.resume start at zero in the copied descriptor
  cudaMemcpyAsync(dinst, &I, sizeof(I), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(queue, 0, 2 * sizeof(int), st);
  const size_t smem_setup = std::max((size_t)(2 * 32 * 33), (size_t)(2 * m + n)) * sizeof(double);
  abip::dense_setup_kernel<<<1, abip::kThreads, smem_setup, st>>>(dinst, 1, queue);
  cudaMemsetAsync(queue, 0, 2 * sizeof(int), st);
  abip::DenseParams dp{prm.beta, prm.gamma, prm.alpha, prm.eps, prm.max_admm_iters, prm.warmstart,
                       prm.stop_rule, 0, 1, 0, 0, 0.0, 0.0, prm.gamma_max};
  const size_t smem_solve = (size_t)(5 * m + 3 * n) * sizeof(double);
  abip::dense_solve_kernel<double, 1><<<1, abip::kThreads, smem_solve, st>>>(dinst, 1, dp, queue, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&I, dinst, sizeof(I), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return abip::noalloc_fail(ABIP_E_CUDA, std::string("abip_solve_dense_noalloc: ") + cudaGetErrorString(e));
  if (I.err != 0) return abip::noalloc_fail(ABIP_E_NUMERICAL, "Cholesky breakdown or non-finite value");
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = I.status; info->outer_iters = I.outer_iters; info->admm_iters = I.admm_iters;
    info->tau = I.tau; info->kappa = I.kappa; info->theta = I.theta; info->mu = I.mu;
    info->obj = I.obj; info->pres = I.pres; info->dres = I.dres; info->dgap = I.dgap;
    info->launches = 2;
  }
  return ABIP_OK;
}
