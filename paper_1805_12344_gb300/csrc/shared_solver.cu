// Algorithm 2 for a batch of LPs that share one dense A (different b_k, c_k).
//
// With B instances side by side every product of the ADMM update becomes a GEMM
// with B (or 2B) right-hand columns: A [X S], A^T Y, G^{-1} Q and A^T Z_y.  The
// projection's G^{-1} = (I + A A^T)^{-1} (Sec. 4.4) is formed explicitly once, from
// the FP64 Cholesky factor, so that the per-update solve is one parallel GEMM
// instead of two sequential triangular sweeps.  Every vector is stored row-major as
// [length x B] (instance index fastest) so that GEMM operands, elementwise updates
// and per-instance column reductions all read contiguous memory.
//
// One update cycle (fixed launch sequence, per-instance masks):
//   products  AXS = A [X S], ATY = A^T Y            (GEMM, split-K, deterministic)
//   sums      the nine sums of the Sec. 4.1 tests and Eq. inner-stop, Q = Y - AX - AS
//   control   per instance: tests after an update, inner stop ||Qu-v||^2 <= mu,
//             mu decrease with warm start, or another update
//   [mixed]   FP64 confirmation of FP32 screens that pass
//   step      ZY = G^{-1} Q, ZX = X + S + A^T ZY    (GEMM)
//             H^T z, t = K^{-1}(w_tau,theta + H^T z), relaxation, barrier prox,
//             dual update (Eqs. Simple-Update:*, Sec. 4.2)
#include "abip_internal.h"
#include "abip_device.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

namespace abip {
namespace {

constexpr int kThr = 256;
constexpr int kThrWarps = kThr / 32;
constexpr int kMaxBatch = 64;        // instances per launch chunk (one column per thread lane group)
constexpr int kSumRowGroups = kThr / kMaxBatch;

// ---------------------------------------------------------------------------
// SIMT GEMM:  Cpart[z] = op(A)[M x K_z] * W[K_z x N], K split into gridDim.z chunks.
// op(A) = A (row-major, lda) or A^T.  W row-major (ldw).  Cpart: gridDim.z x M x N.
// 256 threads as 16 x 16, each TM x TN outputs at rows tr + 16u, columns tc + 16v.
// ---------------------------------------------------------------------------
template <typename T> struct GemmCfg;
template <> struct GemmCfg<float> { static constexpr int TM = 8, TN = 4, BK = 16; };
template <> struct GemmCfg<double> { static constexpr int TM = 4, TN = 4, BK = 16; };

template <typename T, bool TRANS>
__global__ void __launch_bounds__(kThr) gemm_kernel(const T* __restrict__ A, int64_t lda, int M, int N, int K,
                                                    const T* __restrict__ W, int64_t ldw, T* __restrict__ Cp,
                                                    int kchunk, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  constexpr int TM = GemmCfg<T>::TM, TN = GemmCfg<T>::TN, BK = GemmCfg<T>::BK;
  constexpr int BM = 16 * TM, BN = 16 * TN;
  __shared__ T As[BK][BM + 1];
  __shared__ T Ws[BK][BN + 1];
  const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
  const int i0 = blockIdx.x * BM, k0 = blockIdx.y * BN;
  const int jb = blockIdx.z * kchunk, je = min(K, jb + kchunk);
  T acc[TM][TN];
#pragma unroll
  for (int u = 0; u < TM; ++u)
#pragma unroll
    for (int v = 0; v < TN; ++v) acc[u][v] = T(0);
  for (int j0 = jb; j0 < je; j0 += BK) {
    if (!TRANS) {
      for (int e = tid; e < BM * BK; e += kThr) {
        const int r = e / BK, q = e % BK;
        const int gi = i0 + r, gj = j0 + q;
        As[q][r] = (gi < M && gj < je) ? A[(size_t)gi * lda + gj] : T(0);
      }
    } else {
      for (int e = tid; e < BM * BK; e += kThr) {
        const int q = e / BM, r = e % BM;
        const int gi = i0 + r, gj = j0 + q;
        As[q][r] = (gi < M && gj < je) ? A[(size_t)gj * lda + gi] : T(0);
      }
    }
    for (int e = tid; e < BK * BN; e += kThr) {
      const int q = e / BN, cc = e % BN;
      const int gj = j0 + q, gk = k0 + cc;
      Ws[q][cc] = (gj < je && gk < N) ? W[(size_t)gj * ldw + gk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < BK; ++q) {
      T a[TM], w[TN];
#pragma unroll
      for (int u = 0; u < TM; ++u) a[u] = As[q][tr + 16 * u];
#pragma unroll
      for (int v = 0; v < TN; ++v) w[v] = Ws[q][tc + 16 * v];
#pragma unroll
      for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int v = 0; v < TN; ++v) acc[u][v] += a[u] * w[v];
    }
    __syncthreads();
  }
  T* C = Cp + (size_t)blockIdx.z * M * N;
#pragma unroll
  for (int u = 0; u < TM; ++u) {
    const int gi = i0 + tr + 16 * u;
    if (gi >= M) continue;
#pragma unroll
    for (int v = 0; v < TN; ++v) {
      const int gk = k0 + tc + 16 * v;
      if (gk < N) C[(size_t)gi * N + gk] = acc[u][v];
    }
  }
}

// out[i][k] = sum_z Cpart[z][i][k] (+ diag [i == k]) (+ E[i][k]) (+ F[i][k]), fixed order.
template <typename T>
__global__ void reduce_kernel(const T* __restrict__ Cp, int splits, int M, int N, T* __restrict__ out,
                              T diag, const T* __restrict__ E, const T* __restrict__ F, int64_t lde,
                              const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const size_t MN = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    T v = Cp[e];
    for (int z = 1; z < splits; ++z) v += Cp[(size_t)z * MN + e];
    const int i = (int)(e / N), k = (int)(e % N);
    if (i == k) v += diag;
    if (E) v += E[(size_t)i * lde + k];
    if (F) v += F[(size_t)i * lde + k];
    out[e] = v;
  }
}

// Mixed path: v = sum_z Cpart[z][e] (FP32 partials of a product of deltas); out32[e] = v
// (or 0 where the instance is masked out) and acc64[e] += v (FP64 running product).
// Column k of an N-wide output belongs to instance k % B; the mask (insts non-null)
// keeps only instances whose action is SH_STEP.
__global__ void accum_kernel(const float* __restrict__ Cp, int splits, int M, int N, int B, double* acc64,
                             float* out32, const ShInst* __restrict__ insts) {
  const size_t MN = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    float v = Cp[e];
    for (int z = 1; z < splits; ++z) v += Cp[(size_t)z * MN + e];
    const bool on = !insts || insts[(int)(e % N) % B].action == SH_STEP;
    if (out32) out32[e] = on ? v : 0.0f;
    if (acc64 && on) acc64[e] += (double)v;
  }
}

// ---------------------------------------------------------------------------
// Blocked Cholesky G = L L^T and the explicit inverse of G (setup only, FP64)
// ---------------------------------------------------------------------------
// Right-looking, kCB-wide block columns (G row-major m x m, lower triangle read and
// overwritten by L).  For block column k0:
//   chol_diag_kernel   (one CTA):          factor the diagonal block L_kk in shared memory;
//   chol_panel_kernel  (CTA per kCB rows): L_ik = G_ik L_kk^{-T} for the rows below;
//   chol_update_kernel (CTA per tile):     G_ij -= L_ik L_jk^T on the trailing lower
//                                          triangle, kCB x kCB tiles, 4 x 4 outputs/thread.
// A non-positive or non-finite pivot sets *err; every later kernel then returns at once.
constexpr int kCB = 64;

__global__ void __launch_bounds__(kThr) chol_diag_kernel(double* __restrict__ L, int m, int k0, int* err) {
  __shared__ double T[kCB][kCB + 1];
  __shared__ int ok;
  if (*err) return;
  const int nb = min(kCB, m - k0);
  for (int e = threadIdx.x; e < nb * nb; e += kThr) {
    const int r = e / nb, c = e % nb;
    T[r][c] = c <= r ? L[(size_t)(k0 + r) * m + k0 + c] : 0.0;
  }
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      const double d = T[j][j];
      if (!(d > 0.0) || !isfinite(d)) ok = 0;
      T[j][j] = sqrt(d);
    }
    __syncthreads();
    if (!ok) break;
    const double djj = T[j][j];
    for (int i = j + 1 + threadIdx.x; i < nb; i += kThr) T[i][j] /= djj;
    __syncthreads();
    for (int e = threadIdx.x; e < (nb - j - 1) * (nb - j - 1); e += kThr) {
      const int i = j + 1 + e / (nb - j - 1), l = j + 1 + e % (nb - j - 1);
      if (l <= i) T[i][l] -= T[i][j] * T[l][j];
    }
    __syncthreads();
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, DEV_ERR_CHOLESKY);
    return;
  }
  for (int e = threadIdx.x; e < nb * nb; e += kThr) {
    const int r = e / nb, c = e % nb;
    if (c <= r) L[(size_t)(k0 + r) * m + k0 + c] = T[r][c];
  }
}

// rows k0 + kCB + blockIdx.x * kCB ...: x L_kk^T = g  (forward substitution per row)
constexpr size_t kCholSmem = 2 * sizeof(double) * kCB * (kCB + 1);   // two kCB x (kCB + 1) tiles

__global__ void __launch_bounds__(kThr) chol_panel_kernel(double* __restrict__ L, int m, int k0, const int* err) {
  extern __shared__ double chol_sm[];
  auto D = reinterpret_cast<double(*)[kCB + 1]>(chol_sm);
  auto X = reinterpret_cast<double(*)[kCB + 1]>(chol_sm + kCB * (kCB + 1));
  if (*err) return;
  const int nb = min(kCB, m - k0);
  const int r0 = k0 + nb + blockIdx.x * kCB;
  const int nr = min(kCB, m - r0);
  if (nr <= 0) return;
  for (int e = threadIdx.x; e < nb * nb; e += kThr) {
    const int r = e / nb, c = e % nb;
    D[r][c] = c <= r ? L[(size_t)(k0 + r) * m + k0 + c] : 0.0;
  }
  for (int e = threadIdx.x; e < nr * nb; e += kThr) {
    const int r = e / nb, c = e % nb;
    X[r][c] = L[(size_t)(r0 + r) * m + k0 + c];
  }
  __syncthreads();
  // four threads per row: column j of every row, then the rows' remaining columns
  const int row = threadIdx.x / 4, q = threadIdx.x % 4;
  for (int j = 0; j < nb; ++j) {
    if (row < nr && q == 0) X[row][j] /= D[j][j];
    __syncthreads();
    if (row < nr) {
      const double xj = X[row][j];
      for (int l = j + 1 + q; l < nb; l += 4) X[row][l] -= xj * D[l][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nr * nb; e += kThr) {
    const int r = e / nb, c = e % nb;
    L[(size_t)(r0 + r) * m + k0 + c] = X[r][c];
  }
}

// tile (bi, bj), bi >= bj, of the trailing matrix below and right of block column k0
__global__ void __launch_bounds__(kThr) chol_update_kernel(double* __restrict__ L, int m, int k0, const int* err) {
  extern __shared__ double chol_sm[];
  auto Pi = reinterpret_cast<double(*)[kCB + 1]>(chol_sm);
  auto Pj = reinterpret_cast<double(*)[kCB + 1]>(chol_sm + kCB * (kCB + 1));
  if (*err) return;
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  const int nb = min(kCB, m - k0);
  const int t0 = k0 + nb;
  const int i0 = t0 + bi * kCB, j0 = t0 + bj * kCB;
  const int ni = min(kCB, m - i0), nj = min(kCB, m - j0);
  for (int e = threadIdx.x; e < kCB * nb; e += kThr) {
    const int r = e / nb, c = e % nb;
    Pi[r][c] = r < ni ? L[(size_t)(i0 + r) * m + k0 + c] : 0.0;
    Pj[r][c] = r < nj ? L[(size_t)(j0 + r) * m + k0 + c] : 0.0;
  }
  __syncthreads();
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  double acc[4][4] = {};
  for (int l = 0; l < nb; ++l) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { a[u] = Pi[tr + 16 * u][l]; b[u] = Pj[tc + 16 * u][l]; }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = tr + 16 * u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = tc + 16 * v;
      if (i < ni && j < nj && j0 + j <= i0 + i) L[(size_t)(i0 + i) * m + j0 + j] -= acc[u][v];
    }
  }
}

// G = L L^T in place (lower triangle), err <- DEV_ERR_CHOLESKY on breakdown.
cudaError_t cholesky_blocked(double* G, int m, int* err, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(chol_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chol_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmem);
  if (e != cudaSuccess) return e;
  for (int k0 = 0; k0 < m; k0 += kCB) {
    chol_diag_kernel<<<1, kThr, 0, st>>>(G, m, k0, err);
    const int rest = m - k0 - kCB;
    if (rest <= 0) break;
    const int nt = (rest + kCB - 1) / kCB;
    chol_panel_kernel<<<nt, kThr, kCholSmem, st>>>(G, m, k0, err);
    chol_update_kernel<<<dim3(nt, nt), kThr, kCholSmem, st>>>(G, m, k0, err);
  }
  return cudaGetLastError();
}

// Column k of G^{-1} = L^{-T} L^{-1} e_k, one column per CTA pass (w in shared memory).
__global__ void __launch_bounds__(kThr) inverse_kernel(const double* __restrict__ L, int m, double* __restrict__ Ginv) {
  extern __shared__ double w[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int col = blockIdx.x; col < m; col += gridDim.x) {
    for (int i = threadIdx.x; i < m; i += kThr) w[i] = i == col ? 1.0 : 0.0;
    __syncthreads();
    // L z = e_col (z_i = 0 for i < col)
    for (int kb = (col / 32) * 32; kb < m; kb += 32) {
      const int nb = min(32, m - kb);
      if (wid == 0) {
        double wl = lane < nb ? w[kb + lane] : 0.0;
        for (int j = 0; j < nb; ++j) {
          if (lane == j) wl = wl / L[(size_t)(kb + j) * m + kb + j];
          const double wj = __shfl_sync(0xffffffffu, wl, j);
          if (lane > j && lane < nb) wl -= L[(size_t)(kb + lane) * m + kb + j] * wj;
        }
        if (lane < nb) w[kb + lane] = wl;
      }
      __syncthreads();
      const double wb = lane < nb ? w[kb + lane] : 0.0;
      for (int i = kb + nb + wid; i < m; i += kThrWarps) {
        double a = lane < nb ? L[(size_t)i * m + kb + lane] * wb : 0.0;
        a = warp_sum(a);
        if (lane == 0) w[i] -= a;
      }
      __syncthreads();
    }
    // L^T g = z
    const int nblk = (m + 31) / 32;
    for (int bk = nblk - 1; bk >= 0; --bk) {
      const int kb = bk * 32, nb = min(32, m - kb);
      if (wid == 0) {
        double wl = lane < nb ? w[kb + lane] : 0.0;
        for (int j = nb - 1; j >= 0; --j) {
          if (lane == j) wl = wl / L[(size_t)(kb + j) * m + kb + j];
          const double zj = __shfl_sync(0xffffffffu, wl, j);
          if (lane < j) wl -= L[(size_t)(kb + j) * m + kb + lane] * zj;
        }
        if (lane < nb) w[kb + lane] = wl;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < kb; i += kThr) {
        double a = 0.0;
        for (int j = 0; j < nb; ++j) a += L[(size_t)(kb + j) * m + i] * w[kb + j];
        w[i] -= a;
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < m; i += kThr) Ginv[(size_t)i * m + col] = w[i];
    __syncthreads();
  }
}

template <typename T>
__global__ void transpose_kernel(const double* __restrict__ A, int m, int n, T* __restrict__ AT) {
  __shared__ double t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = by + r, j = bx + threadIdx.x;
    t[r][threadIdx.x] = (i < m && j < n) ? A[(size_t)i * n + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = bx + r, i = by + threadIdx.x;
    if (j < n && i < m) AT[(size_t)j * m + i] = (T)t[threadIdx.x][r];
  }
}

template <typename T>
__global__ void convert_kernel(const double* __restrict__ src, T* __restrict__ dst, size_t len) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (T)src[e];
}

// bfloat16 terms of A (m x n) and A^T (n x m) for the tensor-core products: plane t holds
// the bfloat16 rounding of what planes 0 .. t-1 leave of A's FP32 value.  One plane is
// exact for an A representable in bfloat16, three for any A representable in FP32
// (the host picks `terms`).
// bfloat16 terms of A (m x n, K = n) and of A^T (n x m, K = m), tile-major (tc::a_tiled),
// the operands of the tensor-core products.
__global__ void bf16_copies_kernel(const double* __restrict__ A, int m, int n, int terms,
                                   __nv_bfloat16* __restrict__ A16, __nv_bfloat16* __restrict__ AT16) {
  const size_t tot = (size_t)m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    float rest = (float)A[e];
    const size_t ea = tc::a_tiled(i, j, n), eat = tc::a_tiled(j, i, m);
    for (int t = 0; t < terms; ++t) {
      const __nv_bfloat16 v = __float2bfloat16_rn(rest);
      rest -= __bfloat162float(v);
      A16[t * tot + ea] = v;
      AT16[t * tot + eat] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Per-instance column reductions.  A CTA covers a contiguous range of "virtual rows"
// 0 .. m+n-1 (rows < m are y-type, the rest x-type); thread (rg, k) handles instance
// k and rows rg, rg + 4, ...; partials[cta][k][NS] in double.
// ---------------------------------------------------------------------------
template <int NS>
__device__ void store_partials(double (&acc)[NS], double* sm, double* partials, int B) {
  const int k = threadIdx.x % kMaxBatch, rg = threadIdx.x / kMaxBatch;
#pragma unroll
  for (int q = 0; q < NS; ++q) sm[(rg * kMaxBatch + k) * NS + q] = acc[q];
  __syncthreads();
  if (rg == 0 && k < B) {
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      double v = sm[k * NS + q];
      for (int g = 1; g < kSumRowGroups; ++g) v += sm[(g * kMaxBatch + k) * NS + q];
      partials[((size_t)blockIdx.x * kMaxBatch + k) * NS + q] = v;
    }
  }
}

struct RowRange {
  int r0, r1;
};
__device__ __forceinline__ RowRange my_rows(int total) {
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int r0 = min(total, blockIdx.x * per);
  return {r0, min(total, r0 + per)};
}

// The nine sums (as in the per-CTA dense path) and Q = Y - AX - AS:
//   0 ||Qu-v||^2 (vector blocks), 1 ||Ax/tau - b||^2, 2 ||(A^T y + s)/tau - c||^2,
//   3 ||Ax||^2, 4 ||A^T y + s||^2, 5 b^T y, 6 bbar^T y, 7 c^T x, 8 cbar^T x.
// Mixed path (T = double, maintained products): also dQ = (float)(Q - Qprev).
template <typename T>
__global__ void __launch_bounds__(kThr) sums_kernel(ShView<T> V, const ShInst* __restrict__ st, double* partials,
                                                   T* __restrict__ Q, const int* __restrict__ gate,
                                                   const double* __restrict__ Qprev, float* __restrict__ dQ) {
  if (gate && *gate == 0) return;
  __shared__ double sm[kThr * 9];
  const int m = V.m, n = V.n, B = V.B;
  const int k = threadIdx.x % kMaxBatch, rg = threadIdx.x / kMaxBatch;
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const RowRange rr = my_rows(m + n);
  if (k < B) {
    const double ta = st[k].tau, th = st[k].theta;
    for (int r = rr.r0 + rg; r < rr.r1; r += kSumRowGroups) {
      if (r < m) {
        const size_t e = (size_t)r * B + k;
        const double ax = (double)V.AXS[(size_t)r * 2 * B + k], as = (double)V.AXS[(size_t)r * 2 * B + B + k];
        const double bi = (double)V.b[e], bb = (double)V.bbar[e], yi = (double)V.Y[e];
        const double ry = ax - bi * ta + bb * th;
        const double pr = ax / ta - bi;
        acc[0] += ry * ry; acc[1] += pr * pr; acc[3] += ax * ax;
        acc[5] += bi * yi; acc[6] += bb * yi;
        if (Q) Q[e] = (T)(yi - (ax + as));
        if (dQ) dQ[e] = (float)((yi - (ax + as)) - Qprev[e]);
      } else {
        const int j = r - m;
        const size_t e = (size_t)j * B + k;
        const double aty = (double)V.ATY[e];
        const double xj = (double)V.XS[(size_t)j * 2 * B + k], sj = (double)V.XS[(size_t)j * 2 * B + B + k];
        const double cj = (double)V.c[e], cb = (double)V.cbar[e];
        const double rx = -aty + cj * ta - cb * th - sj;
        const double dr = (aty + sj) / ta - cj;
        acc[0] += rx * rx; acc[2] += dr * dr; acc[4] += (aty + sj) * (aty + sj);
        acc[7] += cj * xj; acc[8] += cb * xj;
      }
    }
  }
  store_partials<9>(acc, sm, partials, B);
}

// H^T z for the projection result: hz0 = c^T zx - b^T zy, hz1 = -cbar^T zx + bbar^T zy.
template <typename T>
__global__ void __launch_bounds__(kThr) hz_kernel(ShView<T> V, double* partials) {
  __shared__ double sm[kThr * 2];
  const int m = V.m, n = V.n, B = V.B;
  const int k = threadIdx.x % kMaxBatch, rg = threadIdx.x / kMaxBatch;
  double acc[2] = {0, 0};
  const RowRange rr = my_rows(m + n);
  if (k < B) {
    for (int r = rr.r0 + rg; r < rr.r1; r += kSumRowGroups) {
      if (r < m) {
        const size_t e = (size_t)r * B + k;
        const double z = (double)V.ZY[e];
        acc[0] -= (double)V.b[e] * z;
        acc[1] += (double)V.bbar[e] * z;
      } else {
        const size_t e = (size_t)(r - m) * B + k;
        const double z = (double)V.ZX[e];
        acc[0] += (double)V.c[e] * z;
        acc[1] -= (double)V.cbar[e] * z;
      }
    }
  }
  store_partials<2>(acc, sm, partials, B);
}

// Mixed path: ZX = X + S + (A^T ZY maintained in FP64), H^T z from ZY and ZX, and
// Qprev = Q for the instances that take this update (their ZY now matches Q).
__global__ void __launch_bounds__(kThr) hz_delta_kernel(ShView<double> V, const double* __restrict__ ATZY,
                                                        double* Qprev, const ShInst* __restrict__ insts,
                                                        double* partials) {
  __shared__ double sm[kThr * 2];
  const int m = V.m, n = V.n, B = V.B;
  const int k = threadIdx.x % kMaxBatch, rg = threadIdx.x / kMaxBatch;
  double acc[2] = {0, 0};
  const RowRange rr = my_rows(m + n);
  if (k < B) {
    const bool step = insts[k].action == SH_STEP;
    for (int r = rr.r0 + rg; r < rr.r1; r += kSumRowGroups) {
      if (r < m) {
        const size_t e = (size_t)r * B + k;
        const double z = V.ZY[e];
        acc[0] -= V.b[e] * z;
        acc[1] += V.bbar[e] * z;
        if (step) Qprev[e] = V.Q[e];
      } else {
        const int j = r - m;
        const size_t e = (size_t)j * B + k;
        const double z = V.XS[(size_t)j * 2 * B + k] + V.XS[(size_t)j * 2 * B + B + k] + ATZY[e];
        V.ZX[e] = z;
        acc[0] += V.c[e] * z;
        acc[1] -= V.cbar[e] * z;
      }
    }
  }
  store_partials<2>(acc, sm, partials, B);
}

// End of an FP64 refresh: the exact Q becomes the reference for later deltas.
__global__ void refresh_finish_kernel(const double* __restrict__ Q, double* Qprev, float* dQ, size_t len,
                                      const int* __restrict__ gate) {
  if (*gate == 0) return;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x) {
    Qprev[e] = Q[e];
    dQ[e] = 0.0f;
  }
}

template <int NS>
__device__ void total_partials(const double* partials, int nparts, int k, double (&out)[NS]) {
#pragma unroll
  for (int q = 0; q < NS; ++q) out[q] = 0.0;
  for (int p = 0; p < nparts; ++p)
#pragma unroll
    for (int q = 0; q < NS; ++q) out[q] += partials[((size_t)p * kMaxBatch + k) * NS + q];
}

// totals[k][q] = sum over the reduction CTAs of partials[cta][k][q]: one CTA per instance,
// fixed assignment of partials to threads and a fixed-order block reduction.
template <int NS>
__global__ void __launch_bounds__(kThr) partials_total_kernel(const double* __restrict__ partials, int nparts,
                                                              double* __restrict__ totals) {
  __shared__ double red[32 * NS];
  const int k = blockIdx.x;
  double v[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) v[q] = 0.0;
  for (int p = threadIdx.x; p < nparts; p += kThr)
#pragma unroll
    for (int q = 0; q < NS; ++q) v[q] += partials[((size_t)p * kMaxBatch + k) * NS + q];
  block_sum<NS>(v, red);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NS; ++q) totals[k * NS + q] = v[q];
}

// Sec. 4.1 tests on the nine sums; 0 = none passes.
__device__ int sh_tests(const ShInst& I, const double (&a)[9], double margin, double eps) {
  const double tau = I.tau;
  const double ps = sqrt(a[1]) / (1.0 + I.nb), ds = sqrt(a[2]) / (1.0 + I.nc);
  const double gp = fabs(a[7] / tau - a[5] / tau) / (1.0 + fabs(a[7] / tau) + fabs(a[5] / tau));
  if (ps <= margin * eps && ds <= margin * eps && gp <= margin * eps) return ABIP_OPTIMAL;
  if (a[5] > 0 && sqrt(a[4]) <= margin * eps * a[5] / I.nb) return ABIP_PRIMAL_INFEASIBLE;
  if (a[7] < 0 && sqrt(a[3]) <= margin * eps * (-a[7]) / I.nc) return ABIP_DUAL_INFEASIBLE;
  return 0;
}

__device__ void sh_absorb(ShInst& I, const double (&a)[9], int n) {
  const double xi = -(double)n - 1.0;
  I.bty = a[5];
  I.ctx = a[7];
  const double rt = a[5] - a[7] + I.zbar * I.theta - I.kappa;
  const double rth = -a[6] + a[8] - I.zbar * I.tau - xi;
  I.inner2 = a[0] + rt * rt + rth * rth;
  I.pres = sqrt(a[1]) / (1.0 + I.nb);
  I.dres = sqrt(a[2]) / (1.0 + I.nc);
  I.dgap = fabs(I.ctx / I.tau - I.bty / I.tau) / (1.0 + fabs(I.ctx / I.tau) + fabs(I.bty / I.tau));
}

// Decide each instance's next move after its sums are in (thread = instance).
//   last == STEP: count the update, run the Sec. 4.1 tests (FP64: decide; FP32: screen
//   with margin 4 and ask for an FP64 confirmation), the update cap.
//   Then the inner stop: mu decrease with warm start (Algorithm 2, keep-larger
//   heuristic on (x, s) and (tau, kappa), sqrt(gamma) on y and theta) or another update.
__global__ void ctrl_eval_kernel(ShInst* insts, int B, int n, const double* partials, int nparts, ShParams P,
                                 int* flags) {
  const int k = threadIdx.x;
  if (k == 0) {
    flags[0] = 0;
    flags[2] += 1;   // cycle counter
    flags[1] = (P.mixed && P.refresh > 0 && flags[2] % P.refresh == 0) ? 1 : 0;
  }
  __syncthreads();
  if (k >= B) return;
  ShInst& I = insts[k];
  if (I.action == SH_DONE) return;
  double a[9];
  total_partials<9>(partials, nparts, k, a);
  sh_absorb(I, a, n);
  if (!isfinite(I.inner2)) { I.err = DEV_ERR_NONFINITE; I.action = SH_DONE; return; }
  if (I.last == SH_STEP) {
    I.total += 1;
    int status = 0;
    if (P.stop_rule == 0) {
      if (!P.mixed) {
        status = sh_tests(I, a, 1.0, P.eps);
      } else if (I.total >= I.next_confirm && sh_tests(I, a, 4.0, P.eps) != 0) {
        // decided on exact FP64 sums at the next scheduled refresh; the instance keeps
        // iterating meanwhile, so a refresh serves every instance that asked since the last
        I.pending = 1;
        I.next_confirm = I.total + P.confirm_gap;
      }
    }
    if (status != 0) { I.status = status; I.action = SH_DONE; return; }
    if (I.total >= P.max_admm) { I.status = ABIP_MAX_ITER; I.action = SH_DONE; return; }
  }
  atomicAdd(&flags[0], 1);
  if (I.inner2 <= I.mu) {
    I.gam = adaptive_gamma(P.gamma, P.gamma_max, P.eps, fmax(I.pres, fmax(I.dres, I.dgap)));
    I.mu *= I.gam;
    I.outer += 1;
    I.level_start = I.total;
    if (P.stop_rule == 1 && I.mu < P.eps) { I.status = ABIP_OPTIMAL; I.action = SH_DONE; return; }
    if (I.outer >= kMaxOuter) { I.status = ABIP_MAX_ITER; I.action = SH_DONE; return; }
    const double sg = sqrt(I.gam);
    if (P.warmstart == 1) {
      I.tau *= sg;
      I.kappa *= sg;
    } else if (I.tau >= I.kappa) {
      I.kappa *= I.gam;
    } else {
      I.tau *= I.gam;
    }
    I.theta *= sg;
    I.action = SH_WARM;
  } else {
    I.action = SH_STEP;
  }
}

// At a scheduled FP64 refresh: the instances whose maintained screen passed since the last
// one are decided on the exact sums of their current state (mixed path).
__global__ void ctrl_confirm_kernel(ShInst* insts, int B, const double* partials, int nparts, ShParams P,
                                    const int* flags) {
  const int k = threadIdx.x;
  if (flags[1] == 0 || k >= B) return;
  ShInst& I = insts[k];
  // an instance that warm-starts this cycle already carries the new tau, kappa, theta while
  // its vectors are rescaled only later in the cycle: it stays pending for the next refresh
  if (I.action != SH_STEP || !I.pending) return;
  I.pending = 0;
  double a[9];
  total_partials<9>(partials, nparts, k, a);
  const int status = sh_tests(I, a, 1.0, P.eps);
  if (status != 0) {
    sh_absorb(I, a, P.n);   // report the exact sums of the state that passed
    I.status = status;
    I.action = SH_DONE;
  }
}

// After H^T z: t = K^{-1}(tau + kappa + hz0, theta + xi + hz1), then the scalar part of
// the update (relaxation and the tau / kappa barrier step, theta).
__global__ void ctrl_step_kernel(ShInst* insts, int B, int n, const double* partials, int nparts, ShParams P) {
  const int k = threadIdx.x;
  if (k >= B) return;
  ShInst& I = insts[k];
  I.last = I.action;
  if (I.action != SH_STEP) return;
  double hz[2];
  total_partials<2>(partials, nparts, k, hz);
  const double xi = -(double)n - 1.0;
  const double v1 = I.tau + I.kappa + hz[0], v2 = I.theta + xi + hz[1];
  const double t1 = I.Kinv[0] * v1 + I.Kinv[1] * v2, t2 = I.Kinv[2] * v1 + I.Kinv[3] * v2;
  I.t1 = t1;
  I.t2 = t2;
  const double th = P.alpha * t1 + (1.0 - P.alpha) * I.tau;
  double tn, kn;
  barrier_step<double>(th - I.kappa, I.mu / P.beta, tn, kn);
  I.cmu = I.mu / P.beta;
  I.tau = tn;
  I.kappa = kn;
  I.theta = P.alpha * t2 + (1.0 - P.alpha) * I.theta;
}

// Elementwise part of the update (STEP) or of the warm start (WARM), per (row, instance).
// Mixed path (dXS non-null): also the FP32 changes of x and s (zero where the instance
// did not move), the input of the maintained product A [dX dS].
//   ATZY, ATG1, ATG2 (mixed path, else null): A^T y of the new state follows from the
//   update's linearity in y: y <- alpha (zy - g1y t1 - g2y t2) + (1 - alpha) y gives
//   A^T y <- alpha (A^T zy - (A^T g1y) t1 - (A^T g2y) t2) + (1 - alpha) A^T y, with A^T zy
//   maintained for the projection and A^T g1y, A^T g2y formed once at setup; the warm
//   start scales it with y.  This replaces a product with A^T per cycle.
template <typename T>
__global__ void update_kernel(ShView<T> V, const ShInst* __restrict__ insts, ShParams P, float* dXS,
                              const T* __restrict__ ATZY, const T* __restrict__ ATG1, const T* __restrict__ ATG2) {
  const int m = V.m, n = V.n, B = V.B;
  const size_t tot = (size_t)(m + n) * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / B), k = (int)(e % B);
    const ShInst& I = insts[k];
    const int act = I.last;
    if (r >= m && dXS) {
      const int j = r - m;
      dXS[(size_t)j * 2 * B + k] = 0.0f;
      dXS[(size_t)j * 2 * B + B + k] = 0.0f;
    }
    const T x0 = r < m ? T(0) : V.XS[(size_t)(r - m) * 2 * B + k];
    const T s0 = r < m ? T(0) : V.XS[(size_t)(r - m) * 2 * B + B + k];
    if (act == SH_STEP) {
      const T t1 = (T)I.t1, t2 = (T)I.t2, a = (T)P.alpha, a1 = (T)(1.0 - P.alpha);
      if (r < m) {
        const size_t q = (size_t)r * B + k;
        const T uy = V.ZY[q] - V.G1[(size_t)r * B + k] * t1 - V.G2[(size_t)r * B + k] * t2;
        V.Y[q] = a * uy + a1 * V.Y[q];
      } else {
        const int j = r - m;
        const size_t q = (size_t)j * B + k;
        const size_t gx = (size_t)(m + j) * B + k;
        const T ux = V.ZX[q] - V.G1[gx] * t1 - V.G2[gx] * t2;
        T* xp = V.XS + (size_t)j * 2 * B + k;
        T* sp = xp + B;
        const T xh = a * ux + a1 * *xp;
        T xn, sn;
        if (dXS) barrier_step_newton(xh - *sp, (T)I.cmu, xn, sn);   // mixed: few FP64 operations
        else barrier_step<T>(xh - *sp, (T)I.cmu, xn, sn);
        *xp = xn;
        *sp = sn;
        if (ATG1) V.ATY[q] = a * (ATZY[q] - ATG1[q] * t1 - ATG2[q] * t2) + a1 * V.ATY[q];
      }
    } else if (act == SH_WARM) {
      const T sg = (T)sqrt(I.gam), g = (T)I.gam;
      if (r < m) {
        V.Y[(size_t)r * B + k] *= sg;
      } else {
        const int j = r - m;
        T* xp = V.XS + (size_t)j * 2 * B + k;
        T* sp = xp + B;
        if (P.warmstart == 1) { *xp *= sg; *sp *= sg; }
        else if (*xp >= *sp) *sp *= g;
        else *xp *= g;
        if (ATG1) V.ATY[(size_t)j * B + k] *= sg;
      }
    }
    if ((act == SH_STEP || act == SH_WARM) && r >= m && dXS) {
      {
        const int j = r - m;
        dXS[(size_t)j * 2 * B + k] = (float)(V.XS[(size_t)j * 2 * B + k] - x0);
        dXS[(size_t)j * 2 * B + B + k] = (float)(V.XS[(size_t)j * 2 * B + B + k] - s0);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Setup kernels
// ---------------------------------------------------------------------------
// Per instance: bbar = b - A e (Ae given), cbar = c - e; partial sums of c^T e, ||b||^2,
// ||c||^2 and, once g1 and g2 exist, the four entries of H^T M^{-1} H.
__global__ void __launch_bounds__(kThr) setup_sums_kernel(ShView<double> V, const double* __restrict__ Ae,
                                                          double* partials, int phase) {
  __shared__ double sm[kThr * 7];
  const int m = V.m, n = V.n, B = V.B;
  const int k = threadIdx.x % kMaxBatch, rg = threadIdx.x / kMaxBatch;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const RowRange rr = my_rows(m + n);
  if (k < B) {
    for (int r = rr.r0 + rg; r < rr.r1; r += kSumRowGroups) {
      if (r < m) {
        const size_t e = (size_t)r * B + k;
        const double bi = V.b[e];
        if (phase == 0) {
          V.bbar[e] = bi - Ae[r];
          acc[1] += bi * bi;
        } else {
          const double g1 = V.G1[e], g2 = V.G2[e], bb = V.bbar[e];
          acc[3] += -bi * g1; acc[4] += -bi * g2; acc[5] += bb * g1; acc[6] += bb * g2;
        }
      } else {
        const int j = r - m;
        const size_t e = (size_t)j * B + k;
        const double cj = V.c[e];
        if (phase == 0) {
          V.cbar[e] = cj - 1.0;
          acc[0] += cj;
          acc[2] += cj * cj;
        } else {
          const size_t g = (size_t)r * B + k;
          const double g1 = V.G1[g], g2 = V.G2[g], cb = V.cbar[e];
          acc[3] += cj * g1; acc[4] += cj * g2; acc[5] += -cb * g1; acc[6] += -cb * g2;
        }
      }
    }
  }
  store_partials<7>(acc, sm, partials, B);
}

// K = I + S + H^T M^{-1} H, S = [[0, zbar], [-zbar, 0]]; Algorithm 2's start.
__global__ void setup_ctrl_kernel(ShInst* insts, int B, const double* partials, int nparts, int phase, ShParams P) {
  const int k = threadIdx.x;
  if (k >= B) return;
  ShInst& I = insts[k];
  double a[7];
  total_partials<7>(partials, nparts, k, a);
  if (phase == 0) {
    I.zbar = a[0] + 1.0;
    I.nb = sqrt(a[1]);
    I.nc = sqrt(a[2]);
    I.tau = 1.0; I.kappa = 1.0; I.theta = 1.0; I.mu = P.beta;
    I.total = 0; I.level_start = 0; I.next_confirm = 0;
    I.outer = 0; I.status = 0; I.action = SH_STEP; I.last = SH_INIT; I.err = 0; I.pending = 0;
    return;
  }
  const double K0 = 1.0 + a[3], K1 = I.zbar + a[4], K2 = -I.zbar + a[5], K3 = 1.0 + a[6];
  const double det = K0 * K3 - K1 * K2;
  I.Kinv[0] = K3 / det; I.Kinv[1] = -K1 / det; I.Kinv[2] = -K2 / det; I.Kinv[3] = K0 / det;
  if (!isfinite(det) || det == 0.0) { I.err = DEV_ERR_NONFINITE; I.action = SH_DONE; }
}

// Right-hand columns of the two M-solves: W2 = [c_k | -cbar_k] (n x 2B) and, after
// P = A W2, R = [-b_k - P_1 | bbar_k - ... ] so that G^{-1} R gives the y parts:
//   h1 = [-b; c]: a - A d = -b - A c;   h2 = [bbar; -cbar]: a - A d = bbar + A cbar.
__global__ void setup_rhs_kernel(ShView<double> V, double* W2, const double* P2, double* R, int stage) {
  const int m = V.m, n = V.n, B = V.B;
  const size_t tot = stage == 0 ? (size_t)n * B : (size_t)m * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / B), k = (int)(e % B);
    if (stage == 0) {
      W2[(size_t)r * 2 * B + k] = V.c[e];
      W2[(size_t)r * 2 * B + B + k] = -V.cbar[e];
    } else {
      R[(size_t)r * 2 * B + k] = -V.b[e] - P2[(size_t)r * 2 * B + k];
      R[(size_t)r * 2 * B + B + k] = V.bbar[e] - P2[(size_t)r * 2 * B + B + k];
    }
  }
}

// G1, G2 ([(m+n) x B]) from ZY2 (m x 2B) and ZX2 (n x 2B).
__global__ void setup_g_kernel(ShView<double> V, const double* ZY2, const double* ZX2) {
  const int m = V.m, n = V.n, B = V.B;
  const size_t tot = (size_t)(m + n) * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / B), k = (int)(e % B);
    const double* src = r < m ? ZY2 + (size_t)r * 2 * B : ZX2 + (size_t)(r - m) * 2 * B;
    V.G1[e] = src[k];
    V.G2[e] = src[B + k];
  }
}

// Start of Algorithm 2: y = 0, x = s = e.
template <typename T>
__global__ void init_state_kernel(ShView<T> V) {
  const int m = V.m, n = V.n, B = V.B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)m * B; e += (size_t)gridDim.x * blockDim.x)
    V.Y[e] = T(0);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * 2 * B; e += (size_t)gridDim.x * blockDim.x)
    V.XS[e] = T(1);
}

// Row sums A e (FP64), one warp per row.
__global__ void rowsum_kernel(const double* __restrict__ A, int m, int n, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; i < m; i += gridDim.x * (blockDim.x / 32)) {
    double a = 0.0;
    for (int j = lane; j < n; j += 32) a += A[(size_t)i * n + j];
    a = warp_sum(a);
    if (lane == 0) out[i] = a;
  }
}

// Outputs: the scaled candidate or certificate (Sec. 4.1), written FP64 [len x B].
template <typename T>
__global__ void output_kernel(ShView<T> V, const ShInst* __restrict__ insts, double* X, double* Yo, double* S) {
  const int m = V.m, n = V.n, B = V.B;
  const size_t tot = (size_t)(m + n) * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / B), k = (int)(e % B);
    const ShInst& I = insts[k];
    double sx = 1.0 / I.tau, sy = 1.0 / I.tau;
    if (I.status == ABIP_PRIMAL_INFEASIBLE) { sx = 1.0; sy = 1.0 / I.bty; }
    if (I.status == ABIP_DUAL_INFEASIBLE) { sx = -1.0 / I.ctx; sy = 1.0; }
    if (r < m) {
      Yo[(size_t)r * B + k] = (double)V.Y[(size_t)r * B + k] * sy;
    } else {
      const int j = r - m;
      X[(size_t)j * B + k] = (double)V.XS[(size_t)j * 2 * B + k] * sx;
      S[(size_t)j * B + k] = (double)V.XS[(size_t)j * 2 * B + B + k] * sy;
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct GemmPlan {
  int splits = 1, kchunk = 0;
  dim3 grid;
};

template <typename T>
GemmPlan plan_gemm(int M, int N, int K, int sms) {
  constexpr int BM = 16 * GemmCfg<T>::TM, BN = 16 * GemmCfg<T>::TN, BK = GemmCfg<T>::BK;
  GemmPlan g;
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  int splits = std::max(1, (2 * sms + tiles - 1) / tiles);
  const int kblocks = (K + BK - 1) / BK;
  splits = std::min(splits, std::max(1, kblocks / 4));
  const int kchunk = ((kblocks + splits - 1) / splits) * BK;
  g.splits = (K + kchunk - 1) / kchunk;
  g.kchunk = kchunk;
  g.grid = dim3((M + BM - 1) / BM, (N + BN - 1) / BN, g.splits);
  return g;
}

template <typename T>
cudaError_t gemm(bool trans, const T* A, int64_t lda, int M, int N, int K, const T* W, int64_t ldw, T* out,
                 T* work, size_t work_elems, int sms, cudaStream_t st, T diag = T(0), const T* E = nullptr,
                 const T* F = nullptr, int64_t lde = 0, const int* gate = nullptr) {
  const GemmPlan g = plan_gemm<T>(M, N, K, sms);
  if ((size_t)g.splits * M * N > work_elems) return cudaErrorInvalidValue;
  if (trans) gemm_kernel<T, true><<<g.grid, kThr, 0, st>>>(A, lda, M, N, K, W, ldw, work, g.kchunk, gate);
  else gemm_kernel<T, false><<<g.grid, kThr, 0, st>>>(A, lda, M, N, K, W, ldw, work, g.kchunk, gate);
  const size_t MN = (size_t)M * N;
  const int rb = (int)std::min<size_t>((MN + kThr - 1) / kThr, (size_t)sms * 8);
  reduce_kernel<T><<<std::max(rb, 1), kThr, 0, st>>>(work, g.splits, M, N, out, diag, E, F, lde, gate);
  return cudaGetLastError();
}

// FP32 product of deltas, accumulated into an FP64 running product (mixed path).
cudaError_t gemm_acc(bool trans, const float* A, int64_t lda, int M, int N, int K, const float* W, int64_t ldw,
                     int B, double* acc64, float* out32, const ShInst* mask, float* work, size_t work_elems, int sms,
                     cudaStream_t st) {
  const GemmPlan g = plan_gemm<float>(M, N, K, sms);
  if ((size_t)g.splits * M * N > work_elems) return cudaErrorInvalidValue;
  if (trans) gemm_kernel<float, true><<<g.grid, kThr, 0, st>>>(A, lda, M, N, K, W, ldw, work, g.kchunk, nullptr);
  else gemm_kernel<float, false><<<g.grid, kThr, 0, st>>>(A, lda, M, N, K, W, ldw, work, g.kchunk, nullptr);
  const size_t MN = (size_t)M * N;
  const int rb = (int)std::min<size_t>((MN + kThr - 1) / kThr, (size_t)sms * 8);
  accum_kernel<<<std::max(rb, 1), kThr, 0, st>>>(work, g.splits, M, N, B, acc64, out32, mask);
  return cudaGetLastError();
}

// Tensor-core product of deltas (tcgen05, A in `terms` bfloat16 planes, W split in three
// bfloat16 terms), accumulated into an FP64 running product like gemm_acc.
struct TcPlan {
  int splits = 1, kchunk = 0;
};
TcPlan plan_tc(int M, int N, int K, int sms, int terms) {
  // one wave: CTAs per SM from the staged shared memory, split K to fill the SMs
  TcPlan p;
  const int occ = std::max(1, (int)((227 * 1024) / tc::tc2_smem_bytes(N, terms)));
  const int tiles = M / tc::kTM, kblocks = K / tc::kTK;
  int splits = std::max(1, (sms * occ) / tiles);
  splits = std::min(splits, std::max(1, kblocks / 4));
  p.kchunk = ((kblocks + splits - 1) / splits) * tc::kTK;
  p.splits = (K + p.kchunk - 1) / p.kchunk;
  return p;
}
bool tc_shape_ok(int m, int n, int B) {
  return m % tc::kTM == 0 && n % tc::kTM == 0 && B % 16 == 0 && 2 * B <= 256;
}

// the tcgen05 kernel instance for (stages, terms); nullptr if there is none
using TcKernel = void (*)(const __nv_bfloat16*, int64_t, int, int, int, const __nv_bfloat16*, float*, int, int*);
TcKernel tc_kernel_for(int stages, int terms) {
  if (terms == 1) {
    switch (stages) {
      case 6: return tc::tc_gemm2_kernel<6, 1>;
      case 5: return tc::tc_gemm2_kernel<5, 1>;
      case 4: return tc::tc_gemm2_kernel<4, 1>;
      case 3: return tc::tc_gemm2_kernel<3, 1>;
      case 2: return tc::tc_gemm2_kernel<2, 1>;
      default: return nullptr;
    }
  }
  if (terms == 3) {
    switch (stages) {
      case 6: return tc::tc_gemm2_kernel<6, 3>;
      case 5: return tc::tc_gemm2_kernel<5, 3>;
      case 4: return tc::tc_gemm2_kernel<4, 3>;
      case 3: return tc::tc_gemm2_kernel<3, 3>;
      case 2: return tc::tc_gemm2_kernel<2, 3>;
      default: return nullptr;
    }
  }
  return nullptr;
}

cudaError_t gemm_tc(const __nv_bfloat16* A16, int64_t aplane, int terms, int M, int N, int K,
                    const float* W, int64_t ldw, int B, double* acc64, float* out32, const ShInst* mask, float* work,
                    size_t work_elems, __nv_bfloat16* wt, int sms, int* err, cudaStream_t st) {
  const TcPlan p = plan_tc(M, N, K, sms, terms);
  if ((size_t)p.splits * M * N > work_elems) return cudaErrorInvalidValue;
  const TcKernel kern = tc_kernel_for(tc::tc2_stages(N, terms), terms);
  if (!kern) return cudaErrorInvalidValue;
  tc::split3_kernel<<<dim3((K + 31) / 32, (N + 31) / 32), dim3(32, 8), 0, st>>>(W, ldw, K, N, wt);
  const dim3 grid(M / tc::kTM, p.splits);
  kern<<<grid, tc::kTCThreads, tc::tc2_smem_bytes(N, terms), st>>>(A16, aplane, M, N, K, wt, work, p.kchunk, err);
  const size_t MN = (size_t)M * N;
  const int rb = (int)std::min<size_t>((MN + kThr - 1) / kThr, (size_t)sms * 8);
  accum_kernel<<<std::max(rb, 1), kThr, 0, st>>>(work, p.splits, M, N, B, acc64, out32, mask);
  return cudaGetLastError();
}

template <typename T>
size_t gemm_work(int M, int N, int K, int sms) {
  const GemmPlan g = plan_gemm<T>(M, N, K, sms);
  return (size_t)g.splits * M * N;
}

struct Bump {
  char* base = nullptr;
  size_t off = 0;
  template <typename U>
  U* take(size_t n) {
    const size_t at = off;
    off += ((n * sizeof(U) + 255) / 256) * 256;
    return base ? reinterpret_cast<U*>(base + at) : nullptr;
  }
};

}  // namespace

// One chunk of <= 64 instances sharing A.
int shared_batch_run(const SharedBatchArgs& a, std::vector<SharedBatchResult>& out, std::string& err) {
  const int m = a.m, n = a.n, B = a.count;
  const bool mixed = a.prm.mixed != 0;
  if (B < 1 || B > kMaxBatch) { err = "shared batch: a chunk holds 1..64 instances"; return ABIP_E_INVALID_ARG; }
  // the update cycles are captured in a CUDA graph, which the legacy default stream cannot
  // record: without a caller stream the solve runs on its own (it is synchronous, and its
  // inputs are staged through host memory first)
  cudaStream_t st = a.stream;
  cudaStream_t owned = nullptr;
  if (!st) {
    if (cudaStreamCreateWithFlags(&owned, cudaStreamNonBlocking) != cudaSuccess) {
      err = "shared batch: cannot create a stream";
      return ABIP_E_CUDA;
    }
    st = owned;
  }
  if ((size_t)m * 8 > 200 * 1024) {
    err = "shared batch: m <= 25600";
    if (owned) cudaStreamDestroy(owned);
    return ABIP_E_UNSUPPORTED;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // CTAs of the per-instance column reductions (their partials are totalled per instance
  // by partials_total_kernel before the control kernels read them)
  const int red_ctas = std::max(1, std::min(sms * 2, (m + n + 63) / 64));
  const size_t wk64 = std::max({gemm_work<double>(m, m, n, sms), gemm_work<double>(m, 2 * B, n, sms),
                                gemm_work<double>(m, 2 * B, m, sms), gemm_work<double>(n, 2 * B, m, sms),
                                gemm_work<double>(n, B, m, sms), gemm_work<double>(m, B, m, sms)});
  const bool tc = mixed && a.prm.tc != 0 && tc_shape_ok(m, n, B);
  const int terms = a.prm.tc == 3 ? 3 : 1;   // bfloat16 planes of A on the tensor-core path
  const size_t aplane = (size_t)m * n;
  size_t wk32 = mixed ? std::max({gemm_work<float>(m, 2 * B, n, sms), gemm_work<float>(n, B, m, sms),
                                  gemm_work<float>(m, B, m, sms)})
                      : 0;
  if (tc)
    wk32 = std::max({wk32, (size_t)plan_tc(m, 2 * B, n, sms, terms).splits * m * 2 * B,
                     (size_t)plan_tc(n, B, m, sms, terms).splits * n * B});
  ShView<double> V{};
  __nv_bfloat16 *A16 = nullptr, *AT16 = nullptr, *WT16 = nullptr;
  double *A64 = nullptr, *AT64 = nullptr, *G = nullptr, *Ginv64 = nullptr, *Ae = nullptr, *work64 = nullptr;
  double* totals = nullptr;
  double *partials = nullptr, *W2 = nullptr, *P2 = nullptr, *R = nullptr, *ZY2 = nullptr, *ZX2 = nullptr;
  double *Xo = nullptr, *Yo = nullptr, *So = nullptr, *ATZY = nullptr, *Qprev = nullptr;
  double *ATG1 = nullptr, *ATG2 = nullptr;
  float *A32 = nullptr, *Ginv32 = nullptr, *work32 = nullptr, *dXS = nullptr, *dQ = nullptr,
        *dZY = nullptr;
  ShInst* insts = nullptr;
  int *flags = nullptr, *derr = nullptr;
  Bump bp;
  auto layout = [&]() {
    bp.off = 0;
    A64 = bp.take<double>((size_t)m * n);
    AT64 = bp.take<double>((size_t)n * m);
    G = bp.take<double>((size_t)m * m);
    Ginv64 = bp.take<double>((size_t)m * m);
    Ae = bp.take<double>(m);
    work64 = bp.take<double>(wk64);
    partials = bp.take<double>((size_t)red_ctas * kMaxBatch * 9);
    totals = bp.take<double>((size_t)kMaxBatch * 9);
    insts = bp.take<ShInst>(kMaxBatch);
    flags = bp.take<int>(8);
    derr = bp.take<int>(8);
    W2 = bp.take<double>((size_t)n * 2 * B);
    P2 = bp.take<double>((size_t)m * 2 * B);
    R = bp.take<double>((size_t)m * 2 * B);
    ZY2 = bp.take<double>((size_t)m * 2 * B);
    ZX2 = bp.take<double>((size_t)n * 2 * B);
    Xo = bp.take<double>((size_t)n * B);
    Yo = bp.take<double>((size_t)m * B);
    So = bp.take<double>((size_t)n * B);
    V.m = m; V.n = n; V.B = B;
    V.A = A64;
    V.Ginv = Ginv64;
    V.b = bp.take<double>((size_t)m * B); V.bbar = bp.take<double>((size_t)m * B);
    V.c = bp.take<double>((size_t)n * B); V.cbar = bp.take<double>((size_t)n * B);
    V.G1 = bp.take<double>((size_t)(m + n) * B); V.G2 = bp.take<double>((size_t)(m + n) * B);
    V.Y = bp.take<double>((size_t)m * B); V.XS = bp.take<double>((size_t)n * 2 * B);
    V.AXS = bp.take<double>((size_t)m * 2 * B); V.ATY = bp.take<double>((size_t)n * B);
    V.Q = bp.take<double>((size_t)m * B); V.ZY = bp.take<double>((size_t)m * B); V.ZX = bp.take<double>((size_t)n * B);
    if (tc) {
      A16 = bp.take<__nv_bfloat16>(terms * aplane);
      AT16 = bp.take<__nv_bfloat16>(terms * aplane);
      WT16 = bp.take<__nv_bfloat16>(3 * std::max((size_t)2 * B * n, (size_t)B * m));
    }
    if (mixed) {
      ATZY = bp.take<double>((size_t)n * B);
      ATG1 = bp.take<double>((size_t)n * B);
      ATG2 = bp.take<double>((size_t)n * B);
      Qprev = bp.take<double>((size_t)m * B);
      A32 = bp.take<float>((size_t)(tc ? 1 : m) * (tc ? 1 : n));
      Ginv32 = bp.take<float>((size_t)m * m);
      work32 = bp.take<float>(wk32);
      dXS = bp.take<float>((size_t)n * 2 * B);
      dQ = bp.take<float>((size_t)m * B);
      dZY = bp.take<float>((size_t)m * B);
    }
  };
  layout();
  const size_t bytes = bp.off;
  void* arena = nullptr;
  if (cudaMalloc(&arena, bytes) != cudaSuccess) {
    err = "shared batch: cannot allocate " + std::to_string(bytes) + " bytes";
    cudaGetLastError();
    if (owned) cudaStreamDestroy(owned);
    return ABIP_E_OOM;
  }
  bp.base = static_cast<char*>(arena);
  layout();
  int rc = ABIP_OK;
  int64_t launches = 0;
  auto ck = [&](cudaError_t e, const char* what) {
    if (rc == ABIP_OK && e != cudaSuccess) {
      err = std::string("shared batch ") + what + ": " + cudaGetErrorString(e);
      rc = ABIP_E_CUDA;
    }
  };
  const int eb = std::max(1, std::min(sms * 8, (int)(((size_t)(m + n) * 2 * B + kThr - 1) / kThr)));
  cudaEvent_t e0 = nullptr, es = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&es);
  cudaEventCreate(&e1);
  // ---- inputs: A (m x n FP64) and the per-instance vectors in [len x B] layout
  {
    std::vector<double> hb((size_t)m * B), hc((size_t)n * B);
    for (int k = 0; k < B; ++k) {
      for (int i = 0; i < m; ++i) hb[(size_t)i * B + k] = a.b[k][i];
      for (int j = 0; j < n; ++j) hc[(size_t)j * B + k] = a.c[k][j];
    }
    ck(cudaMemcpyAsync(A64, a.A, (size_t)m * n * 8, cudaMemcpyHostToDevice, st), "upload A");
    ck(cudaMemcpyAsync(V.b, hb.data(), hb.size() * 8, cudaMemcpyHostToDevice, st), "upload b");
    ck(cudaMemcpyAsync(V.c, hc.data(), hc.size() * 8, cudaMemcpyHostToDevice, st), "upload c");
    ck(cudaMemsetAsync(derr, 0, 8 * sizeof(int), st), "memset");
    ck(cudaMemsetAsync(flags, 0, 8 * sizeof(int), st), "memset");
    ck(cudaStreamSynchronize(st), "upload");   // the host staging vectors go out of scope here
  }
  cudaEventRecord(e0, st);
  // ---- setup (FP64): embedding constants (Eq. bar-b-c-z-re)
  rowsum_kernel<<<std::max(1, std::min(sms * 4, (m + 7) / 8)), kThr, 0, st>>>(A64, m, n, Ae);
  setup_sums_kernel<<<red_ctas, kThr, 0, st>>>(V, Ae, partials, 0);
  setup_ctrl_kernel<<<1, kMaxBatch, 0, st>>>(insts, B, partials, red_ctas, 0, a.prm);
  // G = I + A A^T (Sec. 4.4), its Cholesky factor and the explicit inverse
  transpose_kernel<double><<<dim3((n + 31) / 32, (m + 31) / 32), dim3(32, 8), 0, st>>>(A64, m, n, AT64);
  ck(gemm<double>(false, A64, n, m, m, n, AT64, m, G, work64, wk64, sms, st, 1.0), "Gram");
  ck(cholesky_blocked(G, m, derr, st), "Cholesky");
  const size_t inv_smem = (size_t)m * 8;
  ck(cudaFuncSetAttribute(inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_smem), "smem");
  inverse_kernel<<<std::min(m, sms * 2), kThr, inv_smem, st>>>(G, m, Ginv64);
  // M^{-1} h1, M^{-1} h2 for every instance: z_y = G^{-1}(a - A d), z_x = d + A^T z_y
  setup_rhs_kernel<<<eb, kThr, 0, st>>>(V, W2, nullptr, nullptr, 0);
  ck(gemm<double>(false, A64, n, m, 2 * B, n, W2, 2 * B, P2, work64, wk64, sms, st), "A W2");
  setup_rhs_kernel<<<eb, kThr, 0, st>>>(V, nullptr, P2, R, 1);
  ck(gemm<double>(false, Ginv64, m, m, 2 * B, m, R, 2 * B, ZY2, work64, wk64, sms, st), "Ginv R");
  ck(gemm<double>(true, A64, n, n, 2 * B, m, ZY2, 2 * B, ZX2, work64, wk64, sms, st, 0.0, W2, nullptr, 2 * B),
     "A^T ZY2");
  setup_g_kernel<<<eb, kThr, 0, st>>>(V, ZY2, ZX2);
  setup_sums_kernel<<<red_ctas, kThr, 0, st>>>(V, Ae, partials, 1);
  setup_ctrl_kernel<<<1, kMaxBatch, 0, st>>>(insts, B, partials, red_ctas, 1, a.prm);
  init_state_kernel<double><<<eb, kThr, 0, st>>>(V);
  if (mixed) {
    // A^T g1y, A^T g2y per instance: the y-parts of M^{-1} h1, M^{-1} h2 (rows 0..m-1 of G1, G2)
    ck(gemm<double>(true, A64, n, n, B, m, V.G1, B, ATG1, work64, wk64, sms, st), "A^T G1");
    ck(gemm<double>(true, A64, n, n, B, m, V.G2, B, ATG2, work64, wk64, sms, st), "A^T G2");
    const int cb = sms * 8;
    if (tc) {
      bf16_copies_kernel<<<cb, kThr, 0, st>>>(A64, m, n, terms, A16, AT16);
      for (int N : {B, 2 * B}) {
        const TcKernel kern = tc_kernel_for(tc::tc2_stages(N, terms), terms);
        if (!kern) ck(cudaErrorInvalidValue, "tc stages");
        else ck(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tc::tc2_smem_bytes(N, terms)), "tc smem");
      }
    } else {
      convert_kernel<float><<<cb, kThr, 0, st>>>(A64, A32, (size_t)m * n);
    }
    convert_kernel<float><<<cb, kThr, 0, st>>>(Ginv64, Ginv32, (size_t)m * m);
  }
  ck(cudaGetLastError(), "setup launches");
  cudaEventRecord(es, st);
  int herr = 0;
  ck(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st), "setup status");
  ck(cudaStreamSynchronize(st), "setup");
  if (rc == ABIP_OK && herr != 0) {
    err = "shared batch: Cholesky factorisation of I + A A^T broke down";
    rc = ABIP_E_NUMERICAL;
  }
  const int* gate = flags + 1;
  // Mixed path: exact FP64 products of the current state (gated on flags[1]); they reset
  // the maintained AX, AS, A^T y, Q, ZY = G^{-1} Q and A^T ZY and decide the instances
  // whose FP32-maintained screen asked for a confirmation.
  auto refresh = [&]() {
    ck(gemm<double>(false, A64, n, m, 2 * B, n, V.XS, 2 * B, V.AXS, work64, wk64, sms, st, 0.0, nullptr, nullptr, 0,
                    gate), "refresh A [X S]");
    ck(gemm<double>(true, A64, n, n, B, m, V.Y, B, V.ATY, work64, wk64, sms, st, 0.0, nullptr, nullptr, 0, gate),
       "refresh A^T Y");
    sums_kernel<double><<<red_ctas, kThr, 0, st>>>(V, insts, partials, V.Q, gate, nullptr, nullptr);
    partials_total_kernel<9><<<B, kThr, 0, st>>>(partials, red_ctas, totals);
    ctrl_confirm_kernel<<<1, kMaxBatch, 0, st>>>(insts, B, totals, 1, a.prm, flags);
    ck(gemm<double>(false, Ginv64, m, m, B, m, V.Q, B, V.ZY, work64, wk64, sms, st, 0.0, nullptr, nullptr, 0, gate),
       "refresh Ginv Q");
    ck(gemm<double>(true, A64, n, n, B, m, V.ZY, B, ATZY, work64, wk64, sms, st, 0.0, nullptr, nullptr, 0, gate),
       "refresh A^T ZY");
    refresh_finish_kernel<<<eb, kThr, 0, st>>>(V.Q, Qprev, dQ, (size_t)m * B, gate);
    launches += 12;
  };
  // ---- Algorithm 2, all instances in lockstep
  auto cycle64 = [&]() {
    ck(gemm<double>(false, A64, n, m, 2 * B, n, V.XS, 2 * B, V.AXS, work64, wk64, sms, st), "A [X S]");
    ck(gemm<double>(true, A64, n, n, B, m, V.Y, B, V.ATY, work64, wk64, sms, st), "A^T Y");
    sums_kernel<double><<<red_ctas, kThr, 0, st>>>(V, insts, partials, V.Q, nullptr, nullptr, nullptr);
    partials_total_kernel<9><<<B, kThr, 0, st>>>(partials, red_ctas, totals);
    ctrl_eval_kernel<<<1, kMaxBatch, 0, st>>>(insts, B, n, totals, 1, a.prm, flags);
    ck(gemm<double>(false, Ginv64, m, m, B, m, V.Q, B, V.ZY, work64, wk64, sms, st), "Ginv Q");
    ck(gemm<double>(true, A64, n, n, B, m, V.ZY, B, V.ZX, work64, wk64, sms, st, 0.0, V.XS, V.XS + B, 2 * B),
       "A^T ZY");
    hz_kernel<double><<<red_ctas, kThr, 0, st>>>(V, partials);
    partials_total_kernel<2><<<B, kThr, 0, st>>>(partials, red_ctas, totals);
    ctrl_step_kernel<<<1, kMaxBatch, 0, st>>>(insts, B, n, totals, 1, a.prm);
    update_kernel<double><<<eb, kThr, 0, st>>>(V, insts, a.prm, nullptr, nullptr, nullptr, nullptr);
    launches += 15;
  };
  // with_refresh: this cycle's number is a multiple of a.prm.refresh, so ctrl_eval_kernel
  // opens the gate of the FP64 refresh; other cycles leave its kernels out altogether
  auto cycle_mixed = [&](bool with_refresh) {
    sums_kernel<double><<<red_ctas, kThr, 0, st>>>(V, insts, partials, V.Q, nullptr, Qprev, dQ);
    partials_total_kernel<9><<<B, kThr, 0, st>>>(partials, red_ctas, totals);
    ctrl_eval_kernel<<<1, kMaxBatch, 0, st>>>(insts, B, n, totals, 1, a.prm, flags);
    launches += 3;
    if (with_refresh) refresh();
    // projection on the change of Q: ZY += G^{-1} dQ, A^T ZY += A^T (G^{-1} dQ)
    ck(gemm_acc(false, Ginv32, m, m, B, m, dQ, B, B, V.ZY, dZY, insts, work32, wk32, sms, st), "Ginv dQ");
    if (tc) ck(gemm_tc(AT16, aplane, terms, n, B, m, dZY, B, B, ATZY, nullptr, nullptr, work32, wk32, WT16, sms,
                       derr + 1, st),
               "A^T dZY");
    else ck(gemm_acc(true, A32, n, n, B, m, dZY, B, B, ATZY, nullptr, nullptr, work32, wk32, sms, st), "A^T dZY");
    hz_delta_kernel<<<red_ctas, kThr, 0, st>>>(V, ATZY, Qprev, insts, partials);
    partials_total_kernel<2><<<B, kThr, 0, st>>>(partials, red_ctas, totals);
    ctrl_step_kernel<<<1, kMaxBatch, 0, st>>>(insts, B, n, totals, 1, a.prm);
    update_kernel<double><<<eb, kThr, 0, st>>>(V, insts, a.prm, dXS, ATZY, ATG1, ATG2);
    // maintained products of the new state: AX, AS += A [dX dS] (A^T Y in update_kernel)
    if (tc)
      ck(gemm_tc(A16, aplane, terms, m, 2 * B, n, dXS, 2 * B, B, V.AXS, nullptr, nullptr, work32, wk32, WT16, sms,
                 derr + 1, st),
         "A dXS");
    else
      ck(gemm_acc(false, A32, n, m, 2 * B, n, dXS, 2 * B, B, V.AXS, nullptr, nullptr, work32, wk32, sms, st), "A dXS");
    launches += tc ? 12 : 10;
  };
  if (mixed && rc == ABIP_OK) {
    // exact products of the starting point
    ck(cudaMemsetAsync(flags + 1, 0xff, sizeof(int), st), "gate");
    refresh();
  }
  int* hflags = nullptr;
  cudaMallocHost(&hflags, 8 * sizeof(int));
  const int64_t max_cycles = 2 * a.prm.max_admm + 2 * (int64_t)kMaxOuter + 16;
  int64_t cycles = 0;
  constexpr int kGroup = 16;
  // The scheduled FP64 refresh falls on cycles numbered by multiples of a.prm.refresh (a
  // multiple of kGroup), i.e. on the last cycle of a group: groups are launched from one
  // of two CUDA graphs, without a refresh or with one in the last cycle (every decision
  // inside them taken on the device); direct launches if a capture or an instantiation
  // fails.
  const bool aligned = mixed && a.prm.refresh > 0 && a.prm.refresh % kGroup == 0;
  auto group = [&](bool refresh_last) {
    for (int g = 0; g < kGroup; ++g) {
      if (mixed) cycle_mixed(aligned ? (refresh_last && g == kGroup - 1) : true);
      else cycle64();
    }
  };
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int64_t group_launches[2] = {0, 0};
  bool graphs = rc == ABIP_OK;
  for (int v = 0; v < (aligned ? 2 : 1) && graphs; ++v) {
    const int rc0 = rc;
    const int64_t l0 = launches;
    cudaGraph_t graph = nullptr;
    graphs = false;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      group(v == 1);
      const cudaError_t ec = cudaStreamEndCapture(st, &graph);
      if (ec == cudaSuccess && graph && rc == ABIP_OK && cudaGraphInstantiate(&gexec[v], graph, 0) == cudaSuccess) {
        group_launches[v] = launches - l0;
        graphs = true;
      } else {
        gexec[v] = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
    }
    launches = l0;
    if (!graphs) {   // fall back to direct launches
      rc = rc0;
      err.clear();
      cudaGetLastError();
    }
  }
  while (rc == ABIP_OK) {
    const bool refresh_last = aligned && (cycles + kGroup) % a.prm.refresh == 0;
    const int v = refresh_last ? 1 : 0;
    if (graphs) {
      ck(cudaGraphLaunch(gexec[v], st), "cycle graph");
      launches += group_launches[v];
    } else {
      group(refresh_last);
    }
    cycles += kGroup;
    ck(cudaGetLastError(), "cycle launches");
    ck(cudaMemcpyAsync(hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st), "flags");
    ck(cudaStreamSynchronize(st), "cycle");
    if (rc != ABIP_OK || hflags[0] == 0) break;
    if (cycles > max_cycles) { err = "shared batch: cycle guard reached"; rc = ABIP_E_NUMERICAL; }
  }
  cudaFreeHost(hflags);
  for (cudaGraphExec_t ge : gexec)
    if (ge) cudaGraphExecDestroy(ge);
  if (rc == ABIP_OK && tc) {
    int herr2 = 0;
    ck(cudaMemcpy(&herr2, derr + 1, sizeof(int), cudaMemcpyDeviceToHost), "tensor-core status");
    if (rc == ABIP_OK && herr2 != 0) {
      err = herr2 == tc::kErrShape ? "shared batch: tensor-core product called with an unsupported shape"
                                   : "shared batch: a tensor-core wait ran past its limit";
      rc = herr2 == tc::kErrShape ? ABIP_E_INVALID_ARG : ABIP_E_TIMEOUT;
    }
  }
  // ---- outputs
  if (rc == ABIP_OK) {
    output_kernel<double><<<eb, kThr, 0, st>>>(V, insts, Xo, Yo, So);
    cudaEventRecord(e1, st);
    std::vector<ShInst> hi(B);
    std::vector<double> hx((size_t)n * B), hy((size_t)m * B), hs((size_t)n * B);
    ck(cudaMemcpyAsync(hi.data(), insts, sizeof(ShInst) * B, cudaMemcpyDeviceToHost, st), "results");
    ck(cudaMemcpyAsync(hx.data(), Xo, hx.size() * 8, cudaMemcpyDeviceToHost, st), "x");
    ck(cudaMemcpyAsync(hy.data(), Yo, hy.size() * 8, cudaMemcpyDeviceToHost, st), "y");
    ck(cudaMemcpyAsync(hs.data(), So, hs.size() * 8, cudaMemcpyDeviceToHost, st), "s");
    ck(cudaStreamSynchronize(st), "outputs");
    float ms_setup = 0.f, ms_iter = 0.f;
    cudaEventElapsedTime(&ms_setup, e0, es);
    cudaEventElapsedTime(&ms_iter, es, e1);
    out.resize(B);
    for (int k = 0; k < B && rc == ABIP_OK; ++k) {
      SharedBatchResult& r = out[k];
      r.inst = hi[k];
      r.setup_s = ms_setup * 1e-3;
      r.kernel_s = ms_iter * 1e-3;
      r.launches = launches;
      r.tensor_cores = tc;
      r.x.resize(n); r.y.resize(m); r.s.resize(n);
      for (int j = 0; j < n; ++j) { r.x[j] = hx[(size_t)j * B + k]; r.s[j] = hs[(size_t)j * B + k]; }
      for (int i = 0; i < m; ++i) r.y[i] = hy[(size_t)i * B + k];
      if (hi[k].err != 0) {
        err = "shared batch instance " + std::to_string(k) + ": non-finite reduction";
        rc = ABIP_E_NUMERICAL;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(es);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(arena);
  if (owned) cudaStreamDestroy(owned);
  return rc;
}

}  // namespace abip
