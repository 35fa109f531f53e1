// Device-side building blocks shared by the ABIP kernels: bounded grid barrier,
// deterministic block and grid reductions, sub-warp CSR row products and the
// closed-form barrier step.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace abip {

// device error codes written to the kernel's status word
enum DevErr : int {
  DEV_OK = 0,
  DEV_ERR_BARRIER_TIMEOUT = 1,   // a grid barrier wait ran past its limit
  DEV_ERR_PCG = 2,               // PCG exceeded cg_max_iter
  DEV_ERR_NONFINITE = 3,         // a reduction produced NaN/Inf
  DEV_ERR_CHOLESKY = 4,          // non-positive pivot in the Cholesky factorisation
};

// Bound on mu decreases of one solve: gamma^kMaxOuter underflows any double, so
// a solve that reaches it stops with ABIP_MAX_ITER instead of looping.
constexpr int kMaxOuter = 4000;

// Default wall-clock limit of one barrier wait (nanoseconds).  A healthy barrier on
// a co-resident cooperative grid completes in microseconds.
constexpr unsigned long long kBarrierLimitNs = 4000000000ull;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

struct GridBarrier {
  unsigned long long* count;   // total arrivals since the launch (host zeroes it)
  int* err;                    // first device error (0 = none)
  unsigned long long limit_ns; // wall-clock limit of one wait; 0 = kBarrierLimitNs
};

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The
// arrival counter only grows: barrier number k of the launch completes when it
// reaches k * gridDim.x, so no reset is needed.  Thread 0 of each CTA arrives
// after a release fence and waits with a wall-clock limit (read on the first spin
// and every 64th after it), leaving early if any CTA has flagged an error.
// `target` is this CTA's running count (all CTAs pass the same barriers).  Returns
// false (in every thread) on timeout or error; the caller must then leave the kernel.
__device__ __forceinline__ bool grid_sync(const GridBarrier& gb, unsigned long long& target) {
  __shared__ int s_ok;
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(gb.count, 1ull);
    if (ld_acquire_u64(gb.count) < target) {
      const unsigned long long t0 = globaltimer_ns();
      const unsigned long long limit = gb.limit_ns ? gb.limit_ns : kBarrierLimitNs;
      unsigned spins = 0;
      while (ld_acquire_u64(gb.count) < target) {
        __nanosleep(32);
        if (ld_relaxed_i32(gb.err) != 0) { ok = 0; break; }
        if ((spins++ & 63u) == 0 && globaltimer_ns() - t0 > limit) {
          atomicCAS(gb.err, 0, (int)DEV_ERR_BARRIER_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (ld_relaxed_i32(gb.err) != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// reductions (fixed order => bitwise reproducible for a fixed launch shape)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over groups of `L` consecutive lanes (L a power of two <= 32); every lane of
// the group receives the group total.  All 32 lanes must call it.
template <int L, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce K doubles; thread 0 receives the totals in v.  `scratch` needs
// K * 32 doubles of shared memory.  blockDim.x must be a multiple of 32.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[k * 32 + wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = lane < nw ? scratch[k * 32 + lane] : 0.0;
      v[k] = warp_sum(t);
    }
  }
  __syncthreads();
}

// Block-reduce K doubles and broadcast the totals to every thread.
template <int K>
__device__ __forceinline__ void block_allsum(double (&v)[K], double* scratch) {
  block_sum<K>(v, scratch);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = scratch[k];
  __syncthreads();
}

// Grid reduction in two halves around a grid barrier:
//   grid_partial: block-reduce and store this CTA's K partials at slot*nblk + blockIdx
//   grid_total:   (after grid_sync) every CTA sums all partials in the same order.
template <int K>
__device__ __forceinline__ void grid_partial(double (&v)[K], double* partials, int slot0,
                                             double* scratch) {
  block_sum<K>(v, scratch);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)(slot0 + k) * gridDim.x + blockIdx.x] = v[k];
  }
}

constexpr int kGridTotalPer = 8;   // partials per lane of warp 0 in grid_total

// Warp 0 loads every slot's partials at once (kGridTotalPer per lane, one L2
// round trip), sums them in a fixed order and broadcasts the K totals through
// shared memory, so every CTA gets the same totals.  Needs gridDim.x <= 32 * kGridTotalPer.
// Same as grid_partial for per-thread values of type T: warp sums in T (FP32 in the
// mixed-precision path, where FP64 shuffle-adds would occupy the 1/64-rate FP64 pipe),
// the per-warp results summed in double.  The caller's next step is a grid barrier.
template <int K, typename T>
__device__ __forceinline__ void grid_partial_t(T (&v)[K], double* partials, int slot0, double* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[k * 32 + wid] = (double)v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = lane < nw ? scratch[k * 32 + lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) partials[(size_t)(slot0 + k) * gridDim.x + blockIdx.x] = t;
    }
  }
}

template <int K>
__device__ __forceinline__ void grid_total(double (&out)[K], const double* partials, int slot0,
                                           double* scratch) {
  const int nb = gridDim.x;
  if (threadIdx.x < 32) {
    double v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const double* p = partials + (size_t)(slot0 + k) * nb;
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < kGridTotalPer; ++q) {
        const int i = threadIdx.x + q * 32;
        t += i < nb ? __ldcg(p + i) : 0.0;
      }
      v[k] = warp_sum(t);
    }
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) scratch[k] = v[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = scratch[k];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// closed-form barrier step (Eq. Simple-Update:Barrier-X and Simple-Update:Dual)
// ---------------------------------------------------------------------------
// For omega = x_hat - s and c = mu/beta returns the minimiser x of
// -c log x + (x - omega)^2/2 and s_new = x - omega (so x * s_new = c), each root
// evaluated in the form without cancellation.
template <typename T>
__device__ __forceinline__ void barrier_step(T omega, T c, T& x, T& s) {
  const T D = sqrt(omega * omega + T(4) * c);
  if (omega >= T(0)) {
    x = T(0.5) * (omega + D);
    s = (T(2) * c) / (omega + D);
  } else {
    x = (T(2) * c) / (D - omega);
    s = T(0.5) * (D - omega);
  }
}

// The barrier and dual step of one column (Eqs. Simple-Update:Barrier-X and
// Simple-Update:Dual, reading A9) with few FP64 operations: the larger root L of
// t^2 - |omega| t - c = 0 from an FP32 square root, refined by one Newton step in FP64
// whose derivative 2L - |omega| = D is taken from the FP32 estimate; the smaller root
// c / L through an FP32 reciprocal refined by one Newton step.  Error below 2e-14
// relative to the closed form (checked over omega in +-[1e-12, 1e12], c in [1e-15, 1e2]);
// outside the range where the FP32 estimates are safe the closed form is used.
__device__ __forceinline__ void barrier_step_newton(double omega, double c, double& x, double& s) {
  const double disc = omega * omega + 4.0 * c;
  if (!(disc > 1e-30 && disc < 1e30)) {
    barrier_step<double>(omega, c, x, s);
    return;
  }
  const double aw = fabs(omega);
  const float d32 = sqrtf((float)disc);
  double L = 0.5 * (aw + (double)d32);
  L -= (L * (L - aw) - c) * (double)(1.0f / d32);
  const double r0 = (double)(1.0f / (float)L);
  const double small = c * (r0 + r0 * (1.0 - L * r0));
  if (omega >= 0.0) { x = L; s = small; }
  else { x = small; s = L; }
}

// ---------------------------------------------------------------------------
// decrease ratio of mu <- gamma mu (Sec. 5)
// ---------------------------------------------------------------------------
// Sec. 5 raises gamma as the iterate approaches the optimum but gives no rule (reading
// B11): with gamma_max > 0 the ratio moves from gamma to gamma_max linearly in log10 of
// rho = max(pres, dres, dgap) of the current iterate, from rho >= 1e-1 down to rho <= eps.
constexpr double kGammaFar = 1e-1;
__device__ __forceinline__ double adaptive_gamma(double gamma, double gamma_max, double eps, double rho) {
  if (!(gamma_max > 0.0)) return gamma;
  double t = log10(kGammaFar / fmax(rho, 1e-300)) / log10(kGammaFar / eps);
  t = fmin(1.0, fmax(0.0, t));
  return gamma + (gamma_max - gamma) * t;
}

template <typename T> __device__ __forceinline__ T ldv(const T* p) { return *p; }

template <typename V>
__device__ __forceinline__ double to_d(V v) { return static_cast<double>(v); }

}  // namespace abip
