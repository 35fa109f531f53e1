// Persistent cooperative kernel running ABIP (Algorithm 2 with the over-relaxation
// of Sec. 4.2) on one sparse LP in mixed precision: the iterate and every product
// the update and the Sec. 4.1 tests need are kept in FP64, and each ADMM update
// changes them by FP32 products of the change of the iterate.
//
//   * Residual products: after an update, Ax += A dx, As += A ds, A^T y += A^T dy
//     (FP32 products of the FP32-rounded changes, added to FP64), recomputed exactly
//     (FP64 products of the FP64 state) every kDeltaRefresh updates, after each mu
//     decrease and before any termination decision.
//   * Projection (Sec. 4.4): G z_y = q with G = I + A A^T and q = y - Ax - As.  z_y and
//     A^T z_y are kept in FP64; each update solves G delta = e for the correction by
//     Jacobi-PCG in FP32, where the right-hand side e = q - z_y - A (A^T z_y) is formed
//     in FP64 (one step of iterative refinement per update), then z_y += delta and
//     A^T z_y += A^T delta.  The start of the correction solve extrapolates the last two
//     corrections, the same start point as extrapolating the last three solutions
//     (reading A10).
//   * The prox and dual update of x, s, tau, kappa (Eqs. Simple-Update:Barrier-X and
//     Simple-Update:Dual, two-root form, reading A9) run in FP64 on the FP64 state.
//
// FP32 rounding thus scales with the size of each change, not with the iterate, so the
// Sec. 4.1 tolerances below FP32's unit roundoff times ||A|| ||y|| are reachable.  The
// setup computes M^{-1} H in FP64 by refining FP32 PCG solves with FP64 residuals.
#include <cmath>

#include "abip_device.cuh"
#include "abip_internal.h"
#include "sell.cuh"

namespace abip {

namespace {

using namespace sell;

// reduction slots (a slot is never rewritten before a barrier separates its previous read);
// S_RES and S_PCG0 are adjacent so that one read gives the tests and the next PCG start
enum Slot : int {
  S_RES = 0,     // 9: residual sums
  S_PCG0 = 9,    // 3: r.zr, r.r, q.q of the next projection's start
  S_PGP = 12,    // 1: p.Gp
  S_RZ = 13,     // 2: r.zr, r.r
  S_HZ = 15,     // 2: h1.z, h2.z
  S_SETUP = 17,  // 3: sum c, ||b||^2, ||c||^2
  S_K = 20,      // 4: H^T M^{-1} H
};

constexpr int kDeltaRefresh = 100;   // updates between exact FP64 recomputations
constexpr int kSetupRounds = 12;     // refinement rounds of one setup solve, at most
constexpr double kSetupRoundRed = 1e-5;   // residual reduction asked of one FP32 round

// start of the correction solve that follows `done` ADMM updates (reading A10 restated
// on corrections): 0 none, 1 the last correction (the linear extrapolation 2 z_k - z_{k-1}
// of the solutions), 2 twice the last minus the one before (the quadratic one)
__device__ __forceinline__ int extrap_for(int cg_warm, int64_t done) {
  return (cg_warm == 2 && done >= 3) ? 2 : (cg_warm >= 1 && done >= 2) ? 1 : 0;
}
__device__ __forceinline__ float start_of(float d1, float d2, int extrap) {
  return extrap == 2 ? 2.f * d1 - d2 : extrap == 1 ? d1 : 0.f;
}

// accumulator of the products with A after an update: A dx, A ds (FP32) and A W (FP64)
struct MaintSt {
  using G = XSW;
  float adx = 0.f, ads = 0.f;
  double aw = 0.0;
  __device__ __forceinline__ void add(float a, const XSW& g) {
    adx += a * g.dx;
    ads += a * g.ds;
    aw += (double)a * g.w;
  }
  template <int L>
  __device__ __forceinline__ void group() {
    adx = group_sum<L>(adx);
    ads = group_sum<L>(ads);
    aw = group_sum<L>(aw);
  }
};

struct DeltaSolver {
  const GridDelta& D;
  SolveCtl* C;
  double* red;   // shared scratch
  Thr th;
  unsigned long long bar_target = 0;
  unsigned long long* prof;
  unsigned long long t_last = 0;
  __device__ DeltaSolver(const GridDelta& d, double* r) : D(d), C(d.ctl), red(r) {
    prof = (blockIdx.x == 0 && threadIdx.x == 0) ? d.ctl->prof : nullptr;
    if (prof) t_last = globaltimer_ns();
  }

  __device__ __forceinline__ void mark(int b) {
    if (prof) {
      const unsigned long long t = globaltimer_ns();
      prof[b] += t - t_last;
      t_last = t;
    }
  }
  __device__ bool sync(int phase) {
    mark(phase);
    const bool ok = grid_sync(GridBarrier{D.bar, &C->err, C->bar_limit_ns}, bar_target);
    mark(P_BARRIER);
    return ok;
  }
  __device__ void flag(int code) {
    if (threadIdx.x == 0) atomicCAS(&C->err, 0, code);
  }

  // Grid totals of K slots plus E scalars derived from them by f(totals, extra) on
  // thread 0, broadcast to the CTA (every CTA computes the same values).
  template <int K, int E, typename F>
  __device__ void totals_x(double (&out)[K], double (&ext)[E], int slot, F f) {
    const int nb = gridDim.x;
    if (threadIdx.x < 32) {
      double v[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const double* pp = D.partials + (size_t)(slot + k) * nb;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < kGridTotalPer; ++q) {
          const int i = threadIdx.x + q * 32;
          acc += i < nb ? __ldcg(pp + i) : 0.0;
        }
        v[k] = warp_sum(acc);
      }
      if (threadIdx.x == 0) {
        double e[E];
        f(v, e);
#pragma unroll
        for (int k = 0; k < K; ++k) red[k] = v[k];
#pragma unroll
        for (int i = 0; i < E; ++i) red[K + i] = e[i];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = red[k];
#pragma unroll
    for (int i = 0; i < E; ++i) ext[i] = red[K + i];
    __syncthreads();
    mark(P_TOTALS);
  }

  // Start of a correction solve for row i (Sec. 4.4 with iterative refinement): the
  // FP64 residual r_0 = q - z_y - delta_0 - (A W)_i of the start point z_y + delta_0,
  // delta_0 = dz (set when the previous solve ended), W = A^T (z_y + delta_0); stores r_0
  // and zr_0 = D^{-1} r_0 in FP32 and adds r.zr, r.r, q.q to pc.
  __device__ __forceinline__ void start_row(int i, double qi, double zyi, double aw, double (&pc)[3]) const {
    const float d0 = D.dz[i];
    const double ri = qi - zyi - (double)d0 - aw;
    const float rf = (float)ri;
    const float zri = D.dinv[i] * rf;
    D.r[i] = rf;
    D.zd[i].x = zri;
    pc[0] += (double)(rf * zri);
    pc[1] += ri * ri;
    pc[2] += qi * qi;
  }

  // Jacobi-PCG (Sec. 4.4) on G delta = e from the start prepared by start_row (r, zr and
  // delta = dz in place, rz = r.zr), the FP64 path's two-phase iteration in FP32:
  //   phase A (rows of A):   p = zr + beta p;  Gp = p + A (u + beta t);  p.Gp
  //   phase B (rows of A^T): t <- u + beta t (= A^T p);  wdel += alpha t;  u <- A^T zr_new,
  //                          gathering zr_new = zr - alpha D^{-1} Gp;  rows of A:
  //                          dz += alpha p, r -= alpha Gp, zr_new = D^{-1} r;  r.zr, r.r
  // so that at the end wdel = A^T (delta - delta_0).  Stops when ||r||^2 <= bound2.
  // Returns iterations (>= 1), -1 on barrier failure, -2 past the cap.
  __device__ int pcg_run(double rz, double bound2, int maxit) {
    float* dz = D.dz; float* r = D.r; float* p = D.p; float* Gp = D.Gp;
    float2* ut = D.ut;
    float2* zd_cur = D.zd;
    float2* zd_nxt = D.zd2;
    {
      auto g = [&](int i) -> float { return zd_cur[i].x; };
      auto e = [&](int j, float v, float) { ut[j].x = v; };
      sell_rows_g<8, 1, float, float>(D.AT, g, g, e, BinaryTail{});
    }
    if (!sync(P_PCG_INIT)) return -1;
    float be = 0.f;
    int k = 0;
    for (;;) {
      if (k >= maxit) return -2;
      const bool first = k == 0;
      float a1 = 0.f;
      {
        auto g = [&](int j) -> float {
          const float2 w = ut[j];
          return first ? w.x : w.x + be * w.y;
        };
        struct RowOps { float zr, p, dinv; };
        auto pre = [&](int i) -> RowOps {
          RowOps o{0.f, 0.f, 0.f};
          if (i >= 0) { o.zr = zd_cur[i].x; o.p = p[i]; o.dinv = D.dinv[i]; }
          return o;
        };
        auto e = [&](int i, float v, float, RowOps o) {
          const float pi = first ? o.zr : o.zr + be * o.p;
          const float gp = pi + v;
          p[i] = pi;
          Gp[i] = gp;
          zd_cur[i].y = o.dinv * gp;
          a1 += pi * gp;
        };
        sell_rows_gp<8, 1, float, float>(D.A, g, g, pre, e, BinaryTail{});
      }
      {
        float a1v[1] = {a1};
        grid_partial_t<1, float>(a1v, D.partials, S_PGP, red);
      }
      if (!sync(P_CG_A)) return -1;
      double pgp[1], exa[1];
      totals_x<1, 1>(pgp, exa, S_PGP, [&](const double* v, double* e) { e[0] = rz / v[0]; });
      const float al = (float)exa[0];
      {
        auto g = [&](int i) -> float {
          const float2 w = zd_cur[i];
          return w.x - al * w.y;
        };
        auto pre = [&](int j) -> float2 {
          float2 w = make_float2(0.f, 0.f);
          if (j >= 0) w = ut[j];
          return w;
        };
        auto e = [&](int j, float v, float, float2 w) {
          const float t = first ? w.x : w.x + be * w.y;
          ut[j] = make_float2(v, t);
          D.wdel[j] = first ? al * t : D.wdel[j] + al * t;
        };
        sell_rows_gp<8, 1, float, float>(D.AT, g, g, pre, e, BinaryTail{});
      }
      mark(P_CG_AT);
      float a2[2] = {0.f, 0.f};
      for (int i = th.gtid; i < D.m; i += th.nthr) {
        dz[i] += al * p[i];
        const float ri = r[i] - al * Gp[i];
        const float zri = D.dinv[i] * ri;
        r[i] = ri;
        zd_nxt[i].x = zri;
        a2[0] += ri * zri;
        a2[1] += ri * ri;
      }
      grid_partial_t<2, float>(a2, D.partials, S_RZ, red);
      if (!sync(P_CG_UPD)) return -1;
      double t2[2], exb[2];
      totals_x<2, 2>(t2, exb, S_RZ, [&](const double* v, double* e) {
        e[0] = v[0] / rz;
        e[1] = v[1] > bound2 ? 1.0 : 0.0;
      });
      be = (float)exb[0];
      rz = t2[0];
      float2* sw = zd_cur; zd_cur = zd_nxt; zd_nxt = sw;
      ++k;
      if (exb[1] == 0.0) break;
    }
    return k;
  }

  // The nine sums of the Sec. 4.1 tests and Eq. inner-stop, in FP64:
  //   0 ||Qu-v||^2 (vector blocks), 1 ||Ax/tau - b||^2, 2 ||(A^T y + s)/tau - c||^2,
  //   3 ||Ax||^2, 4 ||A^T y + s||^2, 5 b^T y, 6 bbar^T y, 7 c^T x, 8 cbar^T x.
  __device__ __forceinline__ void row_sums(int i, double ax, double yi, double tau, double itau, double theta,
                                           double (&acc)[12]) const {
    const double bi = D.b[i], bb = D.bbar[i];
    const double ry = ax - bi * tau + bb * theta;
    const double pr = ax * itau - bi;
    acc[0] += ry * ry;
    acc[1] += pr * pr;
    acc[3] += ax * ax;
    acc[5] += bi * yi;
    acc[6] += bb * yi;
  }
  __device__ __forceinline__ void col_sums(int j, double aty, double tau, double itau, double theta,
                                           double (&acc)[12]) const {
    const double sj = D.s[j], cj = D.c[j], cb = D.cbar[j], xj = D.x[j];
    const double rx = -aty + cj * tau - cb * theta - sj;
    const double dr = (aty + sj) * itau - cj;
    acc[0] += rx * rx;
    acc[2] += dr * dr;
    acc[4] += (aty + sj) * (aty + sj);
    acc[7] += cj * xj;
    acc[8] += cb * xj;
  }
  __device__ __forceinline__ void put_sums(double (&acc)[12]) {
    grid_partial<12>(acc, D.partials, S_RES, red);
  }

  // After an update: Ax += A dx, As += A ds, A^T y += A^T dy (FP32 products of the
  // changes), the nine sums, and the start of the next projection (start_row with
  // A W gathered in the same pass).  Partials in S_RES..S_PCG0; no barrier.
  __device__ void maintained_phase(double tau, double theta) {
    double acc[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double pc[3] = {0.0, 0.0, 0.0};
    const double itau = 1.0 / tau;
    {
      auto gf = [&](int j) -> XSW { return D.xsw[j]; };
      auto pre = [](int) { return NoPre{}; };
      auto e = [&](int i, const MaintSt& st, NoPre) {
        const double ax = D.Ax[i] + (double)st.adx;
        const double as = D.As[i] + (double)st.ads;
        D.Ax[i] = ax;
        D.As[i] = as;
        const double yi = D.y[i];
        row_sums(i, ax, yi, tau, itau, theta, acc);
        start_row(i, yi - (ax + as), D.zy[i], st.aw, pc);
      };
      sell_fold<8, float, MaintSt>(D.A, gf, pre, e, BinaryTail{});
    }
    {
      auto g = [&](int i) -> float { return D.dy[i]; };
      auto e = [&](int j, float v, float) {
        const double aty = D.ATy[j] + (double)v;
        D.ATy[j] = aty;
        col_sums(j, aty, tau, itau, theta, acc);
      };
      sell_rows_g<8, 1, float, float>(D.AT, g, g, e, BinaryTail{});
    }
    acc[9] = pc[0]; acc[10] = pc[1]; acc[11] = pc[2];
    put_sums(acc);
  }

  // Exact FP64 products of the current iterate and the next projection's start, in two
  // phases: (1) Ax, As, A^T y and W = A^T (z_y + delta_0) with FP64 gathers, the nine sums;
  // (2) A W and start_row.  Returns false on barrier failure; the partials are in
  // S_RES..S_PCG0 after it.
  __device__ bool exact_phase(double tau, double theta, int phase) {
    double acc[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double itau = 1.0 / tau;
    {
      auto g0 = [&](int j) -> double { return D.x[j]; };
      auto g1 = [&](int j) -> double { return D.s[j]; };
      auto e = [&](int i, double ax, double as) {
        D.Ax[i] = ax;
        D.As[i] = as;
        row_sums(i, ax, D.y[i], tau, itau, theta, acc);
      };
      sell_rows_g<8, 2, double, float>(D.A, g0, g1, e);
    }
    {
      auto g0 = [&](int i) -> double { return D.y[i]; };
      auto g1 = [&](int i) -> double { return D.zy[i] + (double)D.dz[i]; };
      auto e = [&](int j, double aty, double w) {
        D.ATy[j] = aty;
        D.xsw[j].w = w;
        col_sums(j, aty, tau, itau, theta, acc);
      };
      sell_rows_g<8, 2, double, float>(D.AT, g0, g1, e);
    }
    if (!sync(phase)) return false;
    double pc[3] = {0.0, 0.0, 0.0};
    {
      auto g = [&](int j) -> double { return D.xsw[j].w; };
      auto e = [&](int i, double aw, double) {
        start_row(i, D.y[i] - (D.Ax[i] + D.As[i]), D.zy[i], aw, pc);
      };
      sell_rows_g<8, 1, double, float>(D.A, g, g, e);
    }
    acc[9] = pc[0]; acc[10] = pc[1]; acc[11] = pc[2];
    put_sums(acc);
    return sync(phase);
  }

  // Thread 0 only: the twelve sums -> e = (inner2 = ||Qu - v||^2, pres, dres, dgap, c^T x,
  // b^T y, finite flag, Sec. 4.1 test result with the given margin or 0, bound^2 of the
  // next PCG solve, whether its start is above the bound).  The PCG tolerance is cg_tol,
  // or with cg_rel > 0 max(cg_tol, cg_rel * relative KKT residual) (reading A10).
  __device__ __noinline__ void derive_sums(const double* a, double* e, bool with_tests, double margin,
                                           double tau, double kappa, double theta) {
    const double zbar = C->zbar, xi = C->xi, nb = C->nb, nc = C->nc, eps = C->eps;
    const double rt = a[5] - a[7] + zbar * theta - kappa;
    const double rth = -a[6] + a[8] - zbar * tau - xi;
    e[0] = a[0] + rt * rt + rth * rth;
    e[1] = sqrt(a[1]) / (1.0 + nb);
    e[2] = sqrt(a[2]) / (1.0 + nc);
    e[3] = fabs(a[7] / tau - a[5] / tau) / (1.0 + fabs(a[7] / tau) + fabs(a[5] / tau));
    e[4] = a[7];
    e[5] = a[5];
    e[6] = (isfinite(e[0]) && isfinite(e[1]) && isfinite(e[2]) && isfinite(a[9]) && isfinite(a[10])) ? 1.0 : 0.0;
    int st = 0;
    if (with_tests) {
      if (e[1] <= margin * eps && e[2] <= margin * eps && e[3] <= margin * eps) st = ABIP_OPTIMAL;
      else if (a[5] > 0 && sqrt(a[4]) <= margin * eps * a[5] / nb) st = ABIP_PRIMAL_INFEASIBLE;
      else if (a[7] < 0 && sqrt(a[3]) <= margin * eps * (-a[7]) / nc) st = ABIP_DUAL_INFEASIBLE;
    }
    e[7] = (double)st;
    const double kkt = fmax(e[1], fmax(e[2], e[3]));
    const double tol = C->cg_rel > 0.0 ? fmax(C->cg_tol, C->cg_rel * kkt) : C->cg_tol;
    const double bnd = tol * fmax(1.0, sqrt(a[11]));
    e[8] = bnd * bnd;
    e[9] = a[10] > e[8] ? 1.0 : 0.0;
  }

  // Thread 0 only: t = K^{-1} (w_{tau,theta} + H^T z) from v = H^T z, and the relaxed
  // barrier and dual steps of (tau, kappa) and theta (Sec. 4.2):
  // e = (t1, t2, tau, kappa, theta, mu/beta).
  __device__ __noinline__ void scalar_step(const double* v, double* e, double tau, double kappa,
                                           double theta, double mu) {
    const double alpha = C->alpha, beta = C->beta, xi = C->xi;
    const double v1 = tau + kappa + v[0], v2 = theta + xi + v[1];
    const double t1 = C->Kinv[0] * v1 + C->Kinv[1] * v2, t2 = C->Kinv[2] * v1 + C->Kinv[3] * v2;
    const double th_ = alpha * t1 + (1.0 - alpha) * tau;
    double tn, kn;
    barrier_step<double>(th_ - kappa, mu / beta, tn, kn);
    e[0] = t1; e[1] = t2; e[2] = tn; e[3] = kn;
    e[4] = alpha * t2 + (1.0 - alpha) * theta;
    e[5] = mu / beta;
  }

  // One FP64 solve with M (Sec. 4.4) at setup: [gy; gx] = M^{-1} [hy; hx], i.e.
  // G gy = hy - A hx and gx = hx + A^T gy, by FP32 PCG rounds on the FP64 residual until a
  // round starts below cg_tol; each round asks the FP32 iteration for a reduction of
  // kSetupRoundRed.  Uses zy, ATz, Ax, dz and xsw[].w as scratch.  Returns false on
  // failure (flag set).
  template <typename HY, typename HX>
  __device__ bool setup_solve(HY hy, HX hx, double* gy, double* gx) {
    const Thr t = th;
    for (int j = t.gtid; j < D.n; j += t.nthr) { gx[j] = hx(j); D.xsw[j].w = 0.0; }
    for (int i = t.gtid; i < D.m; i += t.nthr) { D.zy[i] = 0.0; D.dz[i] = 0.f; }
    if (!sync(P_SETUP)) return false;
    {
      auto g = [&](int j) -> double { return gx[j]; };
      auto e = [&](int i, double v, double) { D.Ax[i] = v; };
      sell_rows_g<8, 1, double, float>(D.A, g, g, e);
    }
    if (!sync(P_SETUP)) return false;
    int rounds = 0;
    for (;; ++rounds) {
      if (rounds >= kSetupRounds) { flag(DEV_ERR_PCG); sync(P_SETUP); return false; }
      // start residual of G gy = hy - A hx from the current gy (W = A^T gy)
      double pc[3] = {0.0, 0.0, 0.0};
      {
        auto g = [&](int j) -> double { return D.xsw[j].w; };
        auto e = [&](int i, double aw, double) { start_row(i, hy(i) - D.Ax[i], D.zy[i], aw, pc); };
        sell_rows_g<8, 1, double, float>(D.A, g, g, e);
      }
      grid_partial<3>(pc, D.partials, S_PCG0, red);
      if (!sync(P_SETUP)) return false;
      double tot[3], ex[2];
      totals_x<3, 2>(tot, ex, S_PCG0, [&](const double* v, double* e) {
        const double b = fmax(C->cg_tol * fmax(1.0, sqrt(v[2])), kSetupRoundRed * sqrt(v[1]));
        e[0] = b * b;
        e[1] = v[1] > C->cg_tol * C->cg_tol * fmax(1.0, v[2]) ? 1.0 : 0.0;
      });
      if (ex[1] == 0.0) break;   // converged: the FP64 residual is below cg_tol
      const int it = pcg_run(tot[0], ex[0], C->cg_max);
      if (it == -1) return false;
      if (it == -2) { flag(DEV_ERR_PCG); sync(P_SETUP); return false; }
      for (int i = t.gtid; i < D.m; i += t.nthr) {
        D.zy[i] += (double)D.dz[i];
        D.dz[i] = 0.f;
      }
      if (!sync(P_SETUP)) return false;
      {
        auto g = [&](int i) -> double { return D.zy[i]; };
        auto e = [&](int j, double v, double) { D.xsw[j].w = v; };
        sell_rows_g<8, 1, double, float>(D.AT, g, g, e);
      }
      if (!sync(P_SETUP)) return false;
    }
    for (int i = t.gtid; i < D.m; i += t.nthr) gy[i] = D.zy[i];
    for (int j = t.gtid; j < D.n; j += t.nthr) gx[j] += D.xsw[j].w;
    if (threadIdx.x == 0 && blockIdx.x == 0) C->setup_rounds += rounds + 1;
    return sync(P_SETUP);
  }

  // MODE_SETUP: bbar = b - A e, cbar = c - e, zbar = c^T e + 1 (Eq. bar-b-c-z-re), the
  // Jacobi diagonal 1 + sum_j A_ij^2, norms; M^{-1} h1 and M^{-1} h2 with h1 = [-b; c],
  // h2 = [bbar; -cbar] (Sec. 4.4, 4-block form) and H^T M^{-1} H, all in FP64.
  __device__ void setup() {
    const Thr t = th;
    double acc[3] = {0.0, 0.0, 0.0};
    {
      auto e = [&](int i, double rs, double sq) {
        D.bbar[i] = D.b[i] - rs;
        D.dinv[i] = (float)(1.0 / (1.0 + sq));
      };
      sell_rowstats<double, float>(D.A, e);
    }
    for (int i = t.gtid; i < D.m; i += t.nthr) acc[1] += D.b[i] * D.b[i];
    for (int j = t.gtid; j < D.n; j += t.nthr) {
      D.cbar[j] = D.c[j] - 1.0;
      acc[0] += D.c[j];
      acc[2] += D.c[j] * D.c[j];
    }
    grid_partial<3>(acc, D.partials, S_SETUP, red);
    if (!sync(P_SETUP)) return;
    double tot[3], none[1];
    totals_x<3, 1>(tot, none, S_SETUP, [](const double*, double* e) { e[0] = 0.0; });
    if (!setup_solve([&](int i) { return -D.b[i]; }, [&](int j) { return D.c[j]; }, D.g1y, D.g1x)) return;
    if (!setup_solve([&](int i) { return D.bbar[i]; }, [&](int j) { return -D.cbar[j]; }, D.g2y, D.g2x)) return;
    double k4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = t.gtid; i < D.m; i += t.nthr) {
      const double bi = D.b[i], bbi = D.bbar[i], g1 = D.g1y[i], g2 = D.g2y[i];
      k4[0] += -bi * g1; k4[1] += -bi * g2; k4[2] += bbi * g1; k4[3] += bbi * g2;
    }
    for (int j = t.gtid; j < D.n; j += t.nthr) {
      const double cj = D.c[j], cbj = D.cbar[j], g1 = D.g1x[j], g2 = D.g2x[j];
      k4[0] += cj * g1; k4[1] += cj * g2; k4[2] += -cbj * g1; k4[3] += -cbj * g2;
    }
    grid_partial<4>(k4, D.partials, S_K, red);
    if (!sync(P_SETUP)) return;
    double kt[4];
    totals_x<4, 1>(kt, none, S_K, [](const double*, double* e) { e[0] = 0.0; });
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      C->sum_c = tot[0]; C->sum_b2 = tot[1]; C->sum_c2 = tot[2];
      C->K[0] = 1.0 + kt[0];
      C->K[1] = tot[0] + 1.0 + kt[1];      // zbar = c^T e + 1
      C->K[2] = -(tot[0] + 1.0) + kt[2];
      C->K[3] = 1.0 + kt[3];
    }
  }

  // MODE_SOLVE: Algorithm 2 from the state in D / C.  Each ADMM update is four phases
  // plus the PCG iterations: [PCG: A^T zr_0, then (A, A^T) per iteration] -> [H^T z:
  // z_y += delta, A^T z_y = W + wdel] -> [update: prox and dual steps, A^T delta_0 of the
  // next solve] -> [products of the changes, the Sec. 4.1 sums and the next start residual].
  __device__ void solve() {
    const Thr t = th;
    const double alpha = C->alpha, gamma = C->gamma, eps = C->eps;
    double tau = C->tau, kappa = C->kappa, theta = C->theta, mu = C->mu;
    int64_t total = C->admm_iters;
    int64_t cgtot = C->cg_iters;
    int64_t refreshes = 0;
    int outer = C->outer_iters;
    int status = 0;
    int since_refresh = 0;
    int64_t next_confirm = 0;
    double tot[12];
    double inner2 = 0, pres = 0, dres = 0, dgap = 0, ctx = 0, bty = 0;
    double bound2 = 0.0, rz0 = 0.0;
    bool cold = true;   // the start residual is below the PCG bound

    // the twelve sums (after a barrier) -> the scalars, the next PCG start; the Sec. 4.1
    // tests with `margin` if asked.  Returns the test result, or -1 on a non-finite sum.
    auto absorb = [&](bool with_tests, double margin) -> int {
      double e[10];
      totals_x<12, 10>(tot, e, S_RES, [&](const double* a, double* ee) {
        derive_sums(a, ee, with_tests, margin, tau, kappa, theta);
      });
      inner2 = e[0]; pres = e[1]; dres = e[2]; dgap = e[3]; ctx = e[4]; bty = e[5];
      bound2 = e[8]; cold = e[9] == 0.0; rz0 = tot[9];
      if (e[6] == 0.0) { flag(DEV_ERR_NONFINITE); return -1; }
      return (int)e[7];
    };
    auto exact = [&](int phase) -> bool {
      ++refreshes;
      since_refresh = 0;
      return exact_phase(tau, theta, phase);
    };
    // After an update: maintained products (or the scheduled exact recomputation); the
    // Sec. 4.1 tests screened on them with a factor-4 margin and, when the screen passes,
    // decided on exact products (reading A5 cadence; check_every spaces the decisions).
    auto evaluate_update = [&]() -> bool {
      const bool want = C->stop_rule == 0;
      const bool exact_now = ++since_refresh >= kDeltaRefresh;
      if (exact_now) {
        if (!exact(P_RES)) return false;
      } else {
        maintained_phase(tau, theta);
        if (!sync(P_RES)) return false;
      }
      int st = absorb(want, exact_now ? 1.0 : 4.0);
      if (st < 0) return false;
      if (st != 0 && !exact_now) {
        if (total < next_confirm) return true;
        if (!exact(P_RES)) return false;
        st = absorb(true, 1.0);
        if (st < 0) return false;
        next_confirm = total + C->check_every;
      }
      status = want ? st : 0;
      return true;
    };

    if (!exact(P_RES)) return;
    if (absorb(false, 1.0) < 0) return;
    for (;;) {
      // inner stop, Eq. inner-stop: ||Q u - v||^2 <= mu
      if (inner2 <= mu) {
        const double gk = adaptive_gamma(gamma, C->gamma_max, eps, fmax(pres, fmax(dres, dgap)));
        const double sqrt_gk = sqrt(gk);
        mu *= gk;
        ++outer;
        if (C->stop_rule == 1 && mu < eps) { status = ABIP_OPTIMAL; break; }
        if (outer >= kMaxOuter) { status = ABIP_MAX_ITER; break; }   // mu has underflowed
        // warm start (Sec. 5 heuristic, or Eq. update-next-iterate), then exact products
        if (C->warmstart == 1) {
          for (int j = t.gtid; j < D.n; j += t.nthr) { D.x[j] *= sqrt_gk; D.s[j] *= sqrt_gk; }
          tau *= sqrt_gk; kappa *= sqrt_gk;
        } else {
          for (int j = t.gtid; j < D.n; j += t.nthr) {
            const double xj = D.x[j], sj = D.s[j];
            if (xj >= sj) D.s[j] = gk * sj; else D.x[j] = gk * xj;
          }
          if (tau >= kappa) kappa *= gk; else tau *= gk;
        }
        for (int i = t.gtid; i < D.m; i += t.nthr) D.y[i] *= sqrt_gk;
        theta *= sqrt_gk;
        if (!sync(P_WARM)) return;
        if (!exact(P_WARM)) return;
        if (absorb(false, 1.0) < 0) return;
        continue;
      }
      // ---- one ADMM update -------------------------------------------------
      // projection (Eq. Simple-Update:Affine) with w = u + v: w_y = y (r = 0),
      // w_x = x + s, w_tau = tau + kappa, w_theta = theta + xi;
      // z = M^{-1} w_yx: G z_y = q = y - Ax - As, z_x = w_x + A^T z_y.  The start
      // residual of the correction solve was formed with the last products.
      int it = 0;
      if (!cold) {
        it = pcg_run(rz0, bound2, C->cg_max);
        if (it == -1) return;
        if (it == -2) { flag(DEV_ERR_PCG); sync(P_CG_UPD); return; }
      }
      cgtot += it;
      // z_y += delta; A^T z_y = W + wdel; z_x = x + s + A^T z_y; H^T z; the corrections
      // history and the start of the next solve
      const int exn = extrap_for(C->cg_warm, total + 1);
      double hz[2] = {0.0, 0.0};
      for (int j = t.gtid; j < D.n; j += t.nthr) {
        const double a = it > 0 ? D.xsw[j].w + (double)D.wdel[j] : D.xsw[j].w;
        D.ATz[j] = a;
        const double zxj = (D.x[j] + D.s[j]) + a;
        hz[0] += D.c[j] * zxj;
        hz[1] -= D.cbar[j] * zxj;
      }
      for (int i = t.gtid; i < D.m; i += t.nthr) {
        const float d = D.dz[i];
        const double zyi = D.zy[i] + (double)d;
        D.zy[i] = zyi;
        const float dprev = D.d1[i];
        D.d2[i] = dprev;
        D.d1[i] = d;
        D.dz[i] = start_of(d, dprev, exn);
        hz[0] -= D.b[i] * zyi;
        hz[1] += D.bbar[i] * zyi;
      }
      grid_partial<2>(hz, D.partials, S_HZ, red);
      if (!sync(P_ZX)) return;
      double h[2], sc[6];
      totals_x<2, 6>(h, sc, S_HZ, [&](const double* v, double* e) { scalar_step(v, e, tau, kappa, theta, mu); });
      // u~_yx = z - [g1 g2] t; relaxation (Sec. 4.2); barrier and dual steps in FP64 (the
      // FP32-rounded changes feed the maintained products); and, independent of them, the
      // next W = A^T z_y + A^T delta_0 from an A^T pass
      const double t1 = sc[0], t2 = sc[1], cmu = sc[5], a1 = 1.0 - alpha;
      for (int i = t.gtid; i < D.m; i += t.nthr) {
        const double uy = D.zy[i] - D.g1y[i] * t1 - D.g2y[i] * t2;
        const double y0 = D.y[i];
        const double yn = alpha * uy + a1 * y0;
        D.y[i] = yn;
        D.dy[i] = (float)(yn - y0);
      }
      for (int j = t.gtid; j < D.n; j += t.nthr) {
        const double x0 = D.x[j], s0 = D.s[j];
        const double ux = (x0 + s0 + D.ATz[j]) - D.g1x[j] * t1 - D.g2x[j] * t2;
        const double xh = alpha * ux + a1 * x0;
        double xn, sn;
        barrier_step_newton(xh - s0, cmu, xn, sn);
        D.x[j] = xn;
        D.s[j] = sn;
        D.xsw[j].dx = (float)(xn - x0);
        D.xsw[j].ds = (float)(sn - s0);
      }
      {
        auto g = [&](int i) -> float { return D.dz[i]; };
        auto e = [&](int j, float v, float) { D.xsw[j].w = D.ATz[j] + (double)v; };
        sell_rows_g<8, 1, float, float>(D.AT, g, g, e, BinaryTail{});
      }
      tau = sc[2]; kappa = sc[3]; theta = sc[4];
      if (!sync(P_UPD)) return;
      ++total;
      if (!evaluate_update()) return;
      if (status != 0) break;
      if (total >= C->max_admm) { status = ABIP_MAX_ITER; break; }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      C->tau = tau; C->kappa = kappa; C->theta = theta; C->mu = mu;
      C->admm_iters = total; C->cg_iters = cgtot; C->outer_iters = outer; C->status = status;
      C->pres = pres; C->dres = dres; C->dgap = dgap; C->ctx = ctx; C->bty = bty; C->inner2 = inner2;
      C->refreshes = refreshes;
    }
  }
};

__global__ void __launch_bounds__(kGridThreads, 1) grid_delta_kernel(GridDelta d) {
  __shared__ double red[32 * 12];
  DeltaSolver S(d, red);
  if (d.ctl->mode == MODE_SETUP) S.setup();
  else S.solve();
}

}  // namespace

cudaError_t launch_grid_delta(const GridDelta& d, int grid, cudaStream_t st) {
  void* args[] = {const_cast<GridDelta*>(&d)};
  return cudaLaunchCooperativeKernel((const void*)grid_delta_kernel, dim3(grid), dim3(kGridThreads), args, 0, st);
}

int grid_delta_max_ctas(int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, grid_delta_kernel, kGridThreads, 0);
  return sms * per;
}

}  // namespace abip
