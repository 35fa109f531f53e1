// Persistent cooperative kernel running ABIP (Algorithm 2 with the over-relaxation
// of Sec. 4.2) on one sparse LP: Jacobi-PCG projection (Sec. 4.4), or the direct
// projection through a sparse LDL^T factor of the quasi-definite system (Sec. 4.4),
// and the Sec. 4.1 termination tests, entirely on the device.
//
// One launch covers setup (MODE_SETUP: embedding constants of Eq. bar-b-c-z-re,
// Jacobi diagonal, M^{-1} H and the 2x2 Schur complement) or the whole solve
// (MODE_SOLVE).  Phases are separated by a bounded grid barrier; every scalar the
// control flow depends on is reduced in a fixed order and recomputed identically
// by every CTA, so all CTAs take the same branch.
//
// Sparse products use SELL-32 (one warp per slice of 32 length-sorted rows, one
// thread per row): value and column loads are coalesced and each thread keeps U
// independent gathers in flight, which is what an L2-resident, latency-bound
// product needs on this part.
#include <cmath>

#include "abip_device.cuh"
#include "abip_internal.h"
#include "sell.cuh"

namespace abip {

namespace {

// reduction slots (a slot is never rewritten before a barrier separates its
// previous read)
enum Slot : int {
  S_PCG0 = 0,    // 3: r.zr, r.r, q.q
  S_PGP = 3,     // 1: p.Gp
  S_RZ = 4,      // 2: r.zr, r.r
  S_HZ = 6,      // 2: h1.z, h2.z
  S_RES = 8,     // 9: residual sums
  S_SETUP = 17,  // 3: sum c, ||b||^2, ||c||^2
  S_K = 20,      // 4: H^T M^{-1} H
};

constexpr int kMinBlocks = 1;   // resident CTAs per SM requested from the compiler

// Direct projection: the number of factor solves so far (the flag epoch of the last one),
// per CTA.  Thread 0 loads it at launch and advances it after a __syncthreads that
// follows every thread's read.
__shared__ unsigned long long s_ldl_epoch;

using namespace sell;

// ---------------------------------------------------------------------------
// Sparse direct projection (Sec. 4.4, the quasi-definite system K = [I A^T; A -I]).
// No grid barrier inside.  The factorisation publishes a column by a release store of
// its flag, acquired by its readers.  The sweeps publish each entry by storing the value
// itself over the kLdlEmpty pattern, and a reader waits until the pattern is gone: one
// relaxed 64-bit store and one load per dependency, no fences.  Free functions on one
// LdlView pointer, so that the grid kernel's parameters stay where they are.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_f64(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// Shared wait loop: until done() holds, bounded by the barrier wall-clock limit and left
// as soon as any thread has flagged an error; false in both cases.
template <typename Done>
__device__ __forceinline__ bool ldl_spin_until(Done done, SolveCtl* C) {
  const unsigned long long t0 = globaltimer_ns();
  const unsigned long long limit = C->bar_limit_ns ? C->bar_limit_ns : kBarrierLimitNs;
  for (unsigned spins = 0;; ++spins) {
    __nanosleep(16);
    if (done()) return true;
    if ((spins & 31u) == 31u) {
      if (ld_relaxed_i32(&C->err) != 0) return false;
      if (globaltimer_ns() - t0 > limit) {
        atomicCAS(&C->err, 0, (int)DEV_ERR_BARRIER_TIMEOUT);
        return false;
      }
    }
  }
}

// Factorisation: wait (this lane) until *f >= target.
__device__ __noinline__ bool ldl_spin(const unsigned long long* f, unsigned long long target, SolveCtl* C) {
  return ldl_spin_until([&] { return ld_acquire_u64(f) >= target; }, C);
}
__device__ __forceinline__ bool ldl_wait(const unsigned long long* f, unsigned long long target, SolveCtl* C) {
  return ld_acquire_u64(f) >= target || ldl_spin(f, target, C);
}
__device__ __forceinline__ void st_release(unsigned long long* f, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(f), "l"(v) : "memory");
}

// Sweeps: the value at p once it is no longer kLdlEmpty (kLdlEmpty if the wait failed).
__device__ __noinline__ unsigned long long ldl_spin_value(const unsigned long long* p, SolveCtl* C) {
  unsigned long long v = kLdlEmpty;
  ldl_spin_until([&] { v = ld_relaxed_u64(p); return v != kLdlEmpty; }, C);
  return v;
}
__device__ __forceinline__ bool ldl_take(const double* p, double& out, SolveCtl* C) {
  const unsigned long long* q = reinterpret_cast<const unsigned long long*>(p);
  unsigned long long v = ld_relaxed_u64(q);
  if (v == kLdlEmpty) v = ldl_spin_value(q, C);
  out = __longlong_as_double((long long)v);
  return v != kLdlEmpty;
}

// Left-looking LDL^T of P K P^T on the symbolic pattern: one warp per column, columns
// handed out in increasing order (warp w of W takes w, w + W, ...).  Column j needs the
// columns k < j of row j's entries, each published by its flag; the lowest unfinished
// column never waits, so the sweep always progresses.  For each such k:
//   D_j -= L(j,k)^2 D_k,   L(i,j) -= L(i,k) L(j,k) D_k  for the rows i > j of column k
// (those rows lie in column j's pattern), then L(i,j) /= D_j.  K is quasi-definite, so
// each pivot's sign is fixed (+ for an x node, - for a yhat node); a pivot of the other
// sign, or not finite, is a breakdown (DEV_ERR_LDL).  A failing warp leaves; the waits
// of the others then end on the error flag.
__device__ __noinline__ void ldl_factor(const LdlView* __restrict__ V) {
  const LdlDev& F = V->F;
  SolveCtl* C = V->ctl;
  const int n = V->n;
  const int lane = threadIdx.x & 31;
  const int W = (gridDim.x * blockDim.x) >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int j = gw; j < F.N; j += W) {
    const int64_t c0 = F.Lp[j], c1 = F.Lp[j + 1];
    const bool pos = F.perm[j] < n;
    double d = pos ? 1.0 : -1.0;
    bool ok = true;
    for (int64_t r = F.Rp[j]; r < F.Rp[j + 1]; ++r) {
      const int k = F.Rk[r];
      if (!__all_sync(0xffffffffu, ldl_wait(F.flag + k, 1ull, C))) { ok = false; break; }
      const int64_t pjk = F.Rpos[r];
      const double ljk = __ldcg(F.Lx + pjk);
      const double f = ljk * __ldcg(F.Dd + k);
      d -= ljk * f;
      const int64_t k1 = F.Lp[k + 1];
      bool found = true;
      for (int64_t e = pjk + 1 + lane; e < k1; e += 32) {
        const int i = F.Li[e];
        int64_t lo = c0, hi = c1;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (F.Li[mid] < i) lo = mid + 1;
          else hi = mid;
        }
        if (lo < c1 && F.Li[lo] == i) __stcg(F.Lx + lo, __ldcg(F.Lx + lo) - __ldcg(F.Lx + e) * f);
        else found = false;
      }
      if (!__all_sync(0xffffffffu, found)) {
        if (lane == 0) atomicCAS(&C->err, 0, (int)DEV_ERR_LDL);
        ok = false;
        break;
      }
    }
    if (ok && !(isfinite(d) && (pos ? d > 0.0 : d < 0.0))) {
      if (lane == 0) atomicCAS(&C->err, 0, (int)DEV_ERR_LDL);
      ok = false;
    }
    if (!ok) return;
    for (int64_t e = c0 + lane; e < c1; e += 32) __stcg(F.Lx + e, __ldcg(F.Lx + e) / d);
    if (lane == 0) __stcg(F.Dd + j, d);
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(F.flag + j, 1ull);
  }
}

// Solve K [x; yhat] = [r_x; r_y] with the factor: forward sweep L z = P r by rows in
// increasing order, backward sweep L^T w = D^{-1} z by columns in decreasing order, and
// [x; yhat] = P^T w.  Each warp takes its forward rows (w, w + W, ...) and then its
// backward columns (N-1-w, N-1-w-W, ...).  Everything a task reads belongs to an
// earlier task in that order (forward row p: rows k < p; backward column p: rows i > p
// and forward row p), so the lowest unfinished task never waits.  Solve `epoch` uses the
// buffer pair of its parity and empties the other pair for the next solve (the one
// before, which used it, is complete: a grid barrier separates every two solves).
// rhs(q) is r at node q; put(q, w) receives the solution at node q (lane 0 of the warp
// that finishes it).  On a failed wait the warp leaves with the error flag set; the
// caller's next grid barrier reports it.
template <typename RF, typename PF>
__device__ __forceinline__ void ldl_solve(const LdlView* __restrict__ V, unsigned long long epoch, RF rhs, PF put) {
  const LdlDev& F = V->F;
  SolveCtl* C = V->ctl;
  const int N = F.N;
  const int lane = threadIdx.x & 31;
  const int W = (gridDim.x * blockDim.x) >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const size_t cur = (size_t)(epoch & 1) * N, other = (size_t)((epoch & 1) ^ 1) * N;
  double* zf = F.zf + cur;
  double* wb = F.wb + cur;
  {
    unsigned long long* zo = reinterpret_cast<unsigned long long*>(F.zf + other);
    unsigned long long* wo = reinterpret_cast<unsigned long long*>(F.wb + other);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
      zo[i] = kLdlEmpty;
      wo[i] = kLdlEmpty;
    }
  }
  for (int p = gw; p < N; p += W) {
    const double rp = lane == 0 ? rhs(F.perm[p]) : 0.0;
    double acc = 0.0;
    bool ok = true;
    for (int64_t r = F.Rp[p] + lane; r < F.Rp[p + 1]; r += 32) {
      const double l = __ldcg(F.Lx + F.Rpos[r]);
      double zk;
      if (!ldl_take(zf + F.Rk[r], zk, C)) { ok = false; break; }
      acc += l * zk;
    }
    if (!__all_sync(0xffffffffu, ok)) return;
    acc = warp_sum(acc);
    if (lane == 0) st_relaxed_f64(zf + p, rp - acc);
  }
  for (int t = gw; t < N; t += W) {
    const int p = N - 1 - t;
    double acc = 0.0;
    bool ok = true;
    for (int64_t e = F.Lp[p] + lane; e < F.Lp[p + 1]; e += 32) {
      const double l = __ldcg(F.Lx + e);
      double wi;
      if (!ldl_take(wb + F.Li[e], wi, C)) { ok = false; break; }
      acc += l * wi;
    }
    double zp = 0.0;
    if (lane == 0 && ok) ok = ldl_take(zf + p, zp, C);
    if (!__all_sync(0xffffffffu, ok)) return;
    acc = warp_sum(acc);
    if (lane == 0) {
      const double w = zp / __ldcg(F.Dd + p) - acc;
      st_relaxed_f64(wb + p, w);
      put(F.perm[p], w);
    }
  }
}

// Start of a solve launch: both buffer pairs emptied (a launch that ended early may have
// left either half written); the caller's next grid barrier orders this before any sweep.
__device__ __noinline__ void ldl_reset(const LdlView* __restrict__ V) {
  const LdlDev& F = V->F;
  unsigned long long* z = reinterpret_cast<unsigned long long*>(F.zf);
  unsigned long long* w = reinterpret_cast<unsigned long long*>(F.wb);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * F.N; i += gridDim.x * blockDim.x) {
    z[i] = kLdlEmpty;
    w[i] = kLdlEmpty;
  }
}

// Setup solve `col` of the direct projection: M^{-1} h1 (col 0) or M^{-1} h2 (col 1)
// from K [x; yhat] = [h_x; h_y] with y = -yhat (h1 = [-b; c], h2 = [bbar; -cbar]).
__device__ __noinline__ void ldl_setup_solve(const LdlView* __restrict__ V, int col, unsigned long long epoch) {
  const int n = V->n;
  double* gy = col == 0 ? V->g1y : V->g2y;
  double* gx = col == 0 ? V->g1x : V->g2x;
  auto rhs = [&](int q) -> double {
    if (q < n) return col == 0 ? V->c[q] : -V->cbar[q];
    return col == 0 ? -V->b[q - n] : V->bbar[q - n];
  };
  auto put = [&](int q, double w) {
    if (q < n) gx[q] = w;
    else gy[q - n] = -w;
  };
  ldl_solve(V, epoch, rhs, put);
}

// Projection of one ADMM update by the factor: K [zx; -zy] = [w_x; w_y] with
// w = (y, x + s), and the two sums of H^T z into the partials (slot `slot`).
__device__ __noinline__ void ldl_update_solve(const LdlView* __restrict__ V, unsigned long long epoch, int slot,
                                              double* red) {
  const int n = V->n;
  double hz[2] = {0.0, 0.0};
  auto rhs = [&](int q) -> double { return q < n ? V->x[q] + V->s[q] : V->y[q - n]; };
  auto put = [&](int q, double w) {
    if (q < n) {
      V->zx[q] = w;
      hz[0] += V->c[q] * w;
      hz[1] -= V->cbar[q] * w;
    } else {
      const int i = q - n;
      V->zy[i] = -w;
      hz[0] += V->b[i] * w;
      hz[1] -= V->bbar[i] * w;
    }
  };
  ldl_solve(V, epoch, rhs, put);
  grid_partial_t<2, double>(hz, V->partials, slot, red);
}

template <typename T, typename V>
struct Solver {
  const GridData<T>& D;
  SolveCtl* C;
  double* red;   // shared scratch
  Thr th;
  unsigned long long bar_target = 0;
  unsigned long long* prof;
  unsigned long long t_last = 0;
  __device__ Solver(const GridData<T>& d, double* r) : D(d), C(d.ctl), red(r) {
    prof = (blockIdx.x == 0 && threadIdx.x == 0) ? d.ctl->prof : nullptr;
    if (prof) t_last = globaltimer_ns();
  }

  // phase timer: charge the time since the previous mark to bucket b (CTA 0, thread 0)
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
  template <int K>
  __device__ void totals(double (&out)[K], int slot) {
    grid_total<K>(out, D.partials, slot, red);
    mark(P_TOTALS);
  }

  // Grid totals of K slots plus E scalars derived from them by f(totals, extra),
  // which runs on thread 0 only and is broadcast with the totals.  Every scalar
  // that steers the iteration (CG step lengths, stop tests, the Sec. 4.1 tests,
  // the tau/kappa step) is formed this way: once per CTA, not once per thread,
  // which matters on a part whose FP64 rate is 1/64 of FP32.
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

  // A v, A^T v with the iteration type T; the residual products use double
  // accumulation (exact products of float data, summed in FP64)
  template <typename Epi>
  __device__ void rowsA(const T* v0, Epi& e) {
    auto g = [&](int j) { return v0[j]; };
    sell_rows_g<8, 1, T, V>(D.A, g, g, e);
  }
  template <typename Epi>
  __device__ void rowsAT(const T* v0, Epi& e) {
    auto g = [&](int j) { return v0[j]; };
    sell_rows_g<8, 1, T, V>(D.AT, g, g, e);
  }
  template <typename Epi>
  __device__ void rowsA2_d(const T* v0, const T* v1, Epi& e) {
    auto g0 = [&](int j) { return v0[j]; };
    auto g1 = [&](int j) { return v1[j]; };
    sell_rows_g<8, 2, double, V>(D.A, g0, g1, e);
  }
  template <typename Epi>
  __device__ void rowsAT_d(const T* v0, Epi& e) {
    auto g = [&](int j) { return v0[j]; };
    sell_rows_g<8, 1, double, V>(D.AT, g, g, e);
  }

  __device__ void flag(int code) {
    if (threadIdx.x == 0) atomicCAS(&C->err, 0, code);
  }

  // PCG start (reading A10): 0 the previous solution, 1 the linear extrapolation
  // 2 z - zp2, 2 the quadratic one 3 z - 3 zp2 + zp3 (zp2, zp3: the two solutions before)
  __device__ __forceinline__ static T start(const T* z, const T* zp2, const T* zp3, int extrap, int i) {
    if (extrap == 2) return T(3) * (z[i] - zp2[i]) + zp3[i];
    if (extrap == 1) return T(2) * z[i] - zp2[i];
    return z[i];
  }

  // Jacobi-PCG on G = I + A A^T (Sec. 4.4): z (in: warm start, out: solution),
  // right-hand side q_i = qf(i).  Stop when ||r|| <= tol * max(1, ||q||) (reading
  // A10).  Two phases and two grid barriers per iteration:
  //   phase A (rows of A):   p = zr + beta p;  Gp = p + A (u + beta t);  p.Gp
  //   phase B (rows of A^T): t <- u + beta t (= A^T p);  u <- A^T zr_new, gathering
  //                          zr_new = zr - alpha D^{-1} Gp;  and for the rows of A
  //                          z += alpha p, r -= alpha Gp, zr_new = D^{-1} r;  r.zr, r.r
  // zr is double-buffered so phase B gathers the old values while writing the new.
  // Returns iterations, or -1 on barrier failure / -2 past the cap.
  //
  // Start point: z itself, or with `extrap` the linear extrapolation 2 z - zp2 from
  // the two previous solutions (reading A10); when zp2 is given it receives the
  // previous z.  The extrapolated start is gathered on the fly in the first A^T
  // pass and stored by each row's owner in the first A pass.
  template <typename QF>
  __device__ int pcg(T* z, QF qf, double tol, int maxit, int extrap = 0, T* zp2 = nullptr, T* zp3 = nullptr) {
    using T2 = typename Vec2<T>::type;
    T* r = D.r; T* p = D.p; T* Gp = D.Gp;
    T2* ut = D.ut;                 // (u, t)
    T2* zd_cur = D.zd;             // (zr, D^{-1} Gp)
    T2* zd_nxt = D.zd2;
    T acc[3] = {T(0), T(0), T(0)};
    {
      // A^T z0 into ut[].x
      auto g = [&](int i) -> T { return start(z, zp2, zp3, extrap, i); };
      auto e = [&](int j, T v, T) { ut[j].x = v; };
      sell_rows_g<8, 1, T, V>(D.AT, g, g, e);
    }
    if (!sync(P_PCG_INIT)) return -1;
    {
      auto g = [&](int j) -> T { return ut[j].x; };
      auto e = [&](int i, T v, T) {
        const T qi = qf(i);
        const T zi = start(z, zp2, zp3, extrap, i);
        if (zp3) zp3[i] = zp2[i];
        if (zp2) zp2[i] = z[i];
        z[i] = zi;
        const T ri = qi - (zi + v);
        const T zri = D.dinv[i] * ri;
        r[i] = ri; zd_cur[i].x = zri;
        acc[0] += ri * zri;
        acc[1] += ri * ri;
        acc[2] += qi * qi;
      };
      sell_rows_g<8, 1, T, V>(D.A, g, g, e);
    }
    grid_partial_t<3, T>(acc, D.partials, S_PCG0, red);
    if (!sync(P_PCG_INIT)) return -1;
    double tot[3], ex0[2];
    totals_x<3, 2>(tot, ex0, S_PCG0, [&](const double* v, double* e) {
      const double bnd = tol * fmax(1.0, sqrt(v[2]));
      e[0] = bnd * bnd;                       // stop when ||r||^2 <= bound^2
      e[1] = v[1] > e[0] ? 1.0 : 0.0;
    });
    double rz = tot[0];
    const double bound2 = ex0[0];
    if (ex0[1] == 0.0) return 0;
    // u = A^T zr (so that A^T p_0 = u with p_0 = zr)
    {
      auto g = [&](int i) -> T { return zd_cur[i].x; };
      auto e = [&](int j, T v, T) { ut[j].x = v; };
      sell_rows_g<8, 1, T, V>(D.AT, g, g, e);
    }
    if (!sync(P_PCG_INIT)) return -1;
    T be = T(0);
    int k = 0;
    for (;;) {
      if (k >= maxit) return -2;
      const bool first = k == 0;
      T a1 = T(0);
      {
        // gather A^T p = u + be * t (one pair load per nonzero)
        auto g = [&](int j) -> T {
          const T2 w = ut[j];
          return first ? w.x : w.x + be * w.y;
        };
        struct RowOps { T zr, p, dinv; };
        auto pre = [&](int i) -> RowOps {
          RowOps o{T(0), T(0), T(0)};
          if (i >= 0) { o.zr = zd_cur[i].x; o.p = p[i]; o.dinv = D.dinv[i]; }
          return o;
        };
        auto e = [&](int i, T v, T, RowOps o) {
          const T pi = first ? o.zr : o.zr + be * o.p;
          const T gp = pi + v;
          p[i] = pi;
          Gp[i] = gp;
          zd_cur[i].y = o.dinv * gp;
          a1 += pi * gp;
        };
        sell_rows_gp<8, 1, T, V>(D.A, g, g, pre, e);
      }
      {
        T a1v[1] = {a1};
        grid_partial_t<1, T>(a1v, D.partials, S_PGP, red);
      }
      if (!sync(P_CG_A)) return -1;
      double pgp[1], exa[1];
      totals_x<1, 1>(pgp, exa, S_PGP, [&](const double* v, double* e) { e[0] = rz / v[0]; });
      const T al = (T)exa[0];
      {
        // gather zr_new = zr - al * D^{-1} Gp (one pair load per nonzero)
        auto g = [&](int i) -> T {
          const T2 w = zd_cur[i];
          return w.x - al * w.y;
        };
        auto pre = [&](int j) -> T2 {
          T2 w;
          w.x = T(0); w.y = T(0);
          if (j >= 0) w = ut[j];
          return w;
        };
        auto e = [&](int j, T v, T, T2 w) {
          T2 o;
          o.x = v;
          o.y = first ? w.x : w.x + be * w.y;
          ut[j] = o;
        };
        sell_rows_gp<8, 1, T, V>(D.AT, g, g, pre, e);
      }
      mark(P_CG_AT);
      T a2[2] = {T(0), T(0)};
      for (int i = th.gtid; i < D.m; i += th.nthr) {
        z[i] += al * p[i];
        const T ri = r[i] - al * Gp[i];
        const T zri = D.dinv[i] * ri;
        r[i] = ri; zd_nxt[i].x = zri;
        a2[0] += ri * zri;
        a2[1] += ri * ri;
      }
      grid_partial_t<2, T>(a2, D.partials, S_RZ, red);
      if (!sync(P_CG_UPD)) return -1;
      double t2[2], exb[2];
      totals_x<2, 2>(t2, exb, S_RZ, [&](const double* v, double* e) {
        e[0] = v[0] / rz;
        e[1] = v[1] > bound2 ? 1.0 : 0.0;
      });
      be = (T)exb[0];
      rz = t2[0];
      T2* sw = zd_cur; zd_cur = zd_nxt; zd_nxt = sw;
      ++k;
      if (exb[1] == 0.0) break;
    }
    return k;
  }

  // Residual products and every sum the Sec. 4.1 tests and Eq. inner-stop need,
  // for the current (y, x, s, tau, kappa, theta):  Ax, As (one 2-vector pass over
  // A), A^T y, then
  //   Q u - v  = (Ax - b tau + bbar theta,  -A^T y + c tau - cbar theta - s,
  //               b^T y - c^T x + zbar theta - kappa,  -bbar^T y + cbar^T x - zbar tau - xi)
  // Returns false on barrier failure.  tot[] receives
  //   0 ||Qu-v||^2 (vector blocks), 1 ||Ax/tau - b||^2, 2 ||(A^T y + s)/tau - c||^2,
  //   3 ||Ax||^2, 4 ||A^T y + s||^2, 5 b^T y, 6 bbar^T y, 7 c^T x, 8 cbar^T x.
  template <typename Acc, int E, typename F>
  __device__ bool residuals(double tau, double theta, double (&tot)[9], double (&ext)[E], F f,
                            int phase = P_RES) {
    Acc acc[9] = {Acc(0), Acc(0), Acc(0), Acc(0), Acc(0), Acc(0), Acc(0), Acc(0), Acc(0)};
    const Acc ta = (Acc)tau, th_ = (Acc)theta;
    {
      auto g0 = [&](int j) { return D.x[j]; };
      auto g1 = [&](int j) { return D.s[j]; };
      auto e = [&](int i, Acc ax, Acc as) {
        D.Ax[i] = (T)ax; D.As[i] = (T)as;
        const Acc bi = (Acc)D.b[i];
        const Acc ry = ax - bi * ta + (Acc)D.bbar[i] * th_;
        const Acc pr = ax / ta - bi;
        const Acc yi = (Acc)D.y[i];
        acc[0] += ry * ry;
        acc[1] += pr * pr;
        acc[3] += ax * ax;
        acc[5] += bi * yi;
        acc[6] += (Acc)D.bbar[i] * yi;
      };
      sell_rows_g<8, 2, Acc, V>(D.A, g0, g1, e);
    }
    {
      auto g = [&](int i) { return D.y[i]; };
      auto e = [&](int j, Acc aty, Acc) {
        D.ATy[j] = (T)aty;
        const Acc sj = (Acc)D.s[j], cj = (Acc)D.c[j];
        const Acc rx = -aty + cj * ta - (Acc)D.cbar[j] * th_ - sj;
        const Acc dr = (aty + sj) / ta - cj;
        const Acc xj = (Acc)D.x[j];
        acc[0] += rx * rx;
        acc[2] += dr * dr;
        acc[4] += (aty + sj) * (aty + sj);
        acc[7] += cj * xj;
        acc[8] += (Acc)D.cbar[j] * xj;
      };
      sell_rows_g<8, 1, Acc, V>(D.AT, g, g, e);
    }
    grid_partial_t<9, Acc>(acc, D.partials, S_RES, red);
    if (!sync(phase)) return false;
    totals_x<9, E>(tot, ext, S_RES, f);
    return true;
  }

  // MODE_SETUP: bbar = b - A e, cbar = c - e, zbar = c^T e + 1 (Eq. bar-b-c-z-re),
  // Jacobi diagonal 1 + sum_j A_ij^2, norms; then M^{-1} h1, M^{-1} h2 with
  // h1 = [-b; c], h2 = [bbar; -cbar] (Sec. 4.4, 4-block form) and H^T M^{-1} H.
  __device__ void setup() {
    const Thr t = th;
    double acc[3] = {0.0, 0.0, 0.0};
    {
      auto e = [&](int i, T rs, T sq) {
        D.bbar[i] = D.b[i] - rs;
        D.dinv[i] = T(1) / (T(1) + sq);
      };
      sell_rowstats<T, V>(D.A, e);
    }
    for (int i = t.gtid; i < D.m; i += t.nthr) acc[1] += (double)D.b[i] * (double)D.b[i];
    for (int j = t.gtid; j < D.n; j += t.nthr) {
      D.cbar[j] = D.c[j] - T(1);
      acc[0] += (double)D.c[j];
      acc[2] += (double)D.c[j] * (double)D.c[j];
    }
    grid_partial<3>(acc, D.partials, S_SETUP, red);
    if (!sync(P_SETUP)) return;
    double tot[3];
    totals<3>(tot, S_SETUP);
    if (D.ldl_N > 0) {
      // direct projection: factor P K P^T, then the two setup solves
      const unsigned long long e0 = s_ldl_epoch;
      ldl_factor(D.ldlv);
      if (!sync(P_SETUP)) return;
      for (int col = 0; col < 2; ++col) {
        ldl_setup_solve(D.ldlv, col, e0 + 1 + col);
        if (!sync(P_SETUP)) return;
      }
      if (threadIdx.x == 0) s_ldl_epoch = e0 + 2;   // every thread read s_ldl_epoch before the barriers
    }
    // two solves with M: a = h_y, d = h_x  ->  zy = G^{-1}(a - A d), zx = d + A^T zy
    for (int col = 0; col < 2 && D.ldl_N == 0; ++col) {
      T* gy = col == 0 ? D.g1y : D.g2y;
      T* gx = col == 0 ? D.g1x : D.g2x;
      for (int j = t.gtid; j < D.n; j += t.nthr) gx[j] = col == 0 ? D.c[j] : -D.cbar[j];
      for (int i = t.gtid; i < D.m; i += t.nthr) gy[i] = T(0);
      if (!sync(P_SETUP)) return;
      {
        auto e = [&](int i, T v, T) { D.Ax[i] = v; };
        rowsA(gx, e);
      }
      if (!sync(P_SETUP)) return;
      const int c0 = col;
      auto qf = [&](int i) -> T { return (c0 == 0 ? -D.b[i] : D.bbar[i]) - D.Ax[i]; };
      const int it = pcg(gy, qf, C->cg_tol, C->cg_max);
      if (it == -1) return;
      if (it == -2) { flag(DEV_ERR_PCG); sync(P_SETUP); return; }
      {
        auto e = [&](int j, T v, T) { gx[j] = gx[j] + v; };
        rowsAT(gy, e);
      }
      if (!sync(P_SETUP)) return;
    }
    // H^T M^{-1} H:  h1.g1, h1.g2, h2.g1, h2.g2
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
    totals<4>(kt, S_K);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      C->sum_c = tot[0]; C->sum_b2 = tot[1]; C->sum_c2 = tot[2];
      C->K[0] = 1.0 + kt[0];
      C->K[1] = tot[0] + 1.0 + kt[1];      // zbar = c^T e + 1
      C->K[2] = -(tot[0] + 1.0) + kt[2];
      C->K[3] = 1.0 + kt[3];
    }
  }

  // Thread 0 only: the nine residual sums -> e = (inner2 = ||Qu - v||^2, pres, dres,
  // dgap, c^T x, b^T y, finite flag, Sec. 4.1 test result with the given margin or 0).
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
    e[6] = (isfinite(e[0]) && isfinite(e[1]) && isfinite(e[2])) ? 1.0 : 0.0;
    int st = 0;
    if (with_tests) {
      if (e[1] <= margin * eps && e[2] <= margin * eps && e[3] <= margin * eps) st = ABIP_OPTIMAL;
      else if (a[5] > 0 && sqrt(a[4]) <= margin * eps * a[5] / nb) st = ABIP_PRIMAL_INFEASIBLE;
      else if (a[7] < 0 && sqrt(a[3]) <= margin * eps * (-a[7]) / nc) st = ABIP_DUAL_INFEASIBLE;
    }
    e[7] = (double)st;
  }

  // Thread 0 only: t = K^{-1} (w_{tau,theta} + H^T z) from v = H^T z, and the
  // relaxed barrier and dual steps of (tau, kappa) and theta (Sec. 4.2):
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

  // MODE_SOLVE: Algorithm 2 from the state in D / C.
  __device__ void solve() {
    const Thr t = th;
    const double alpha = C->alpha, gamma = C->gamma, eps = C->eps;
    const double cg_rel = C->cg_rel;
    double tau = C->tau, kappa = C->kappa, theta = C->theta, mu = C->mu;
    int64_t total = C->admm_iters;
    int64_t cgtot = C->cg_iters;
    int outer = C->outer_iters;
    int status = 0;
    double tot[9];
    double inner2 = 0, pres = 0, dres = 0, dgap = 0, ctx = 0, bty = 0;

    auto derive = [&](const double* a, double* e, bool with_tests, double margin) {
      derive_sums(a, e, with_tests, margin, tau, kappa, theta);
    };
    // Residual sums of the current iterate.  FP64 path: FP64 accumulation, tests
    // decided on them.  FP32 path: FP32 sums every update (inner test and screen);
    // when they pass a Sec. 4.1 test within a factor 4, the sums are recomputed with
    // FP64 accumulation (exact products of the FP32 data) and those decide.
    auto evaluate = [&](bool final_test) -> bool {
      const bool want = final_test && C->stop_rule == 0;
      double e[8];
      const double margin = sizeof(T) == 8 ? 1.0 : 4.0;
      auto f = [&](const double* a, double* ee) { derive(a, ee, want, margin); };
      bool ok;
      if (sizeof(T) == 8) ok = residuals<double>(tau, theta, tot, e, f);
      else ok = residuals<T>(tau, theta, tot, e, f);
      if (!ok) return false;
      inner2 = e[0]; pres = e[1]; dres = e[2]; dgap = e[3]; ctx = e[4]; bty = e[5];
      if (e[6] == 0.0) {
        flag(DEV_ERR_NONFINITE);
        return false;
      }
      if (want) {
        if (sizeof(T) == 8) {
          status = (int)e[7];
        } else if (e[7] != 0.0) {
          double d[9], e2[8];
          auto f2 = [&](const double* a, double* ee) { derive(a, ee, true, 1.0); };
          if (!residuals<double>(tau, theta, d, e2, f2)) return false;
          pres = e2[1]; dres = e2[2]; dgap = e2[3]; ctx = e2[4]; bty = e2[5];
          status = (int)e2[7];
        }
      }
      return true;
    };

    if (D.ldl_N > 0) ldl_reset(D.ldlv);   // evaluate's grid barrier follows
    if (!evaluate(false)) return;
    for (;;) {
      // inner stop, Eq. inner-stop: ||Q u - v||^2 <= mu
      if (inner2 <= mu) {
        const double gk = adaptive_gamma(gamma, C->gamma_max, eps, fmax(pres, fmax(dres, dgap)));
        const double sqrt_gk = sqrt(gk);
        mu *= gk;
        ++outer;
        if (C->stop_rule == 1 && mu < eps) { status = ABIP_OPTIMAL; break; }
        if (outer >= kMaxOuter) { status = ABIP_MAX_ITER; break; }   // mu has underflowed
        // warm start (Sec. 5 heuristic, or Eq. update-next-iterate)
        const T g = (T)gk, sg = (T)sqrt_gk;
        if (C->warmstart == 1) {
          for (int j = t.gtid; j < D.n; j += t.nthr) { D.x[j] *= sg; D.s[j] *= sg; }
          tau *= sqrt_gk; kappa *= sqrt_gk;
        } else {
          for (int j = t.gtid; j < D.n; j += t.nthr) {
            const T xj = D.x[j], sj = D.s[j];
            if (xj >= sj) D.s[j] = g * sj; else D.x[j] = g * xj;
          }
          if (tau >= kappa) kappa *= gk; else tau *= gk;
        }
        for (int i = t.gtid; i < D.m; i += t.nthr) D.y[i] *= sg;
        theta *= sqrt_gk;
        if (!sync(P_WARM)) return;
        if (!evaluate(false)) return;
        continue;
      }
      // ---- one ADMM update -------------------------------------------------
      // projection (Eq. Simple-Update:Affine) with w = u + v: w_y = y (r = 0),
      // w_x = x + s, w_tau = tau + kappa, w_theta = theta + xi.
      // z = M^{-1} w_yx: G zy = w_y - A w_x = y - Ax - As (PCG warm-started), zx = w_x + A^T zy.
      if (D.ldl_N > 0) {
        const unsigned long long e = s_ldl_epoch + 1;
        ldl_update_solve(D.ldlv, e, S_HZ, red);   // its block reduction syncs after every read of e
        if (threadIdx.x == 0) s_ldl_epoch = e;
      } else {
        T hz[2] = {T(0), T(0)};
        auto qf = [&](int i) -> T { return D.y[i] - (D.Ax[i] + D.As[i]); };
        // PCG tolerance: fixed, or (cg_rel > 0) loosened to cg_rel times the current
        // relative KKT residual, never below cg_tol (reading A10, performance mode)
        const double kkt = fmax(pres, fmax(dres, dgap));
        const double tol = cg_rel > 0.0 ? fmax(C->cg_tol, cg_rel * kkt) : C->cg_tol;
        const int extrap = (C->cg_warm == 2 && total >= 3) ? 2 : (C->cg_warm >= 1 && total >= 2) ? 1 : 0;
        const int it = pcg(D.zy, qf, tol, C->cg_max, extrap, D.zp2, D.zp3);
        if (it == -1) return;
        if (it == -2) { flag(DEV_ERR_PCG); sync(P_CG_UPD); return; }
        cgtot += it;
        {
          auto e = [&](int j, T v, T) {
            const T zxj = (D.x[j] + D.s[j]) + v;
            D.zx[j] = zxj;
            hz[0] += D.c[j] * zxj;
            hz[1] -= D.cbar[j] * zxj;
          };
          rowsAT(D.zy, e);
        }
        for (int i = t.gtid; i < D.m; i += t.nthr) {
          const T zyi = D.zy[i];
          hz[0] -= D.b[i] * zyi;
          hz[1] += D.bbar[i] * zyi;
        }
        grid_partial_t<2, T>(hz, D.partials, S_HZ, red);
      }
      if (!sync(P_ZX)) return;
      double h[2], sc[6];
      // thread 0: t = K^{-1} (w_{tau,theta} + H^T z), and the relaxed barrier and dual
      // steps of the scalar pair (tau, kappa) and of theta (Sec. 4.2)
      totals_x<2, 6>(h, sc, S_HZ, [&](const double* v, double* e) { scalar_step(v, e, tau, kappa, theta, mu); });
      // u~_yx = z - [g1 g2] t; relaxation (Sec. 4.2); barrier and dual steps
      const T a = (T)alpha, a1 = (T)(1.0 - alpha), t1T = (T)sc[0], t2T = (T)sc[1], cmu = (T)sc[5];
      for (int i = t.gtid; i < D.m; i += t.nthr) {
        const T uy = D.zy[i] - D.g1y[i] * t1T - D.g2y[i] * t2T;
        D.y[i] = a * uy + a1 * D.y[i];
      }
      for (int j = t.gtid; j < D.n; j += t.nthr) {
        const T ux = D.zx[j] - D.g1x[j] * t1T - D.g2x[j] * t2T;
        const T xh = a * ux + a1 * D.x[j];
        T xn, sn;
        barrier_step<T>(xh - D.s[j], cmu, xn, sn);
        D.x[j] = xn; D.s[j] = sn;
      }
      tau = sc[2]; kappa = sc[3]; theta = sc[4];
      if (!sync(P_UPD)) return;
      ++total;
      if (!evaluate(true)) return;
      if (status != 0) break;
      if (total >= C->max_admm) { status = ABIP_MAX_ITER; break; }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      C->tau = tau; C->kappa = kappa; C->theta = theta; C->mu = mu;
      C->admm_iters = total; C->cg_iters = cgtot; C->outer_iters = outer; C->status = status;
      C->pres = pres; C->dres = dres; C->dgap = dgap; C->ctx = ctx; C->bty = bty; C->inner2 = inner2;
    }
  }
};

template <typename T, typename V>
__global__ void __launch_bounds__(kGridThreads, kMinBlocks) grid_kernel(GridData<T> d) {
  __shared__ double red[32 * 12];
  if (threadIdx.x == 0) s_ldl_epoch = d.ctl->ldl_epoch;
  __syncthreads();
  Solver<T, V> S(d, red);
  if (d.ctl->mode == MODE_SETUP) S.setup();
  else S.solve();
  // the flag epochs of the direct projection carry into the next launch: the largest
  // count any CTA reached, so that a launch that ended early never reuses one
  __syncthreads();
  if (d.ldl_N > 0 && threadIdx.x == 0) atomicMax(&d.ctl->ldl_epoch, s_ldl_epoch);
}

template <typename T, typename V>
cudaError_t launch(const GridData<T>& d, int grid, cudaStream_t st) {
  void* args[] = {const_cast<GridData<T>*>(&d)};
  return cudaLaunchCooperativeKernel((const void*)grid_kernel<T, V>, dim3(grid), dim3(kGridThreads), args, 0, st);
}

template <typename T, typename V>
int max_ctas(int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, grid_kernel<T, V>, kGridThreads, 0);
  return sms * per;
}

}  // namespace

cudaError_t launch_grid_solver_f64(const GridData<double>& d, bool val_f64, int grid, cudaStream_t st) {
  return val_f64 ? launch<double, double>(d, grid, st) : launch<double, float>(d, grid, st);
}

int grid_solver_max_ctas(bool val_f64, int device) {
  return val_f64 ? max_ctas<double, double>(device) : max_ctas<double, float>(device);
}

}  // namespace abip
