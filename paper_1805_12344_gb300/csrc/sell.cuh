// Sliced-ELL (SELL) row products shared by the persistent grid kernels: the
// thread geometry of a persistent launch, row products with L lanes per row and
// U gathers in flight per lane, and per-row statistics for the setup.
#pragma once

#include <cstdint>

#include "abip_device.cuh"
#include "abip_internal.h"

namespace abip {
namespace sell {

struct Thr {
  int gtid, nthr, gw, nwarp, lane;
  __device__ Thr() {
    gtid = blockIdx.x * blockDim.x + threadIdx.x;
    nthr = gridDim.x * blockDim.x;
    gw = gtid >> 5;
    nwarp = nthr >> 5;
    lane = threadIdx.x & 31;
  }
};

// Row products for every row of a SELL matrix with L lanes per row:
// dot0 = sum_k A_ik g0(k), dot1 = sum_k A_ik g1(k) (NV = 2), accumulated in Acc;
// epi(row, dot0, dot1, pv) runs on the first lane of the row with pv = pre(row),
// which is loaded when the slice starts so the row's own operands arrive while
// the gathers are in flight.  g0/g1 map a column index to the gathered value.
// Each lane keeps U gathers in flight.
template <int L, int U, int NV, typename Acc, typename V, typename G0, typename G1, typename Pre, typename Epi>
__device__ __forceinline__ void sell_rows_L(const SellMat& S, G0& g0, G1& g1, Pre& pre, Epi& epi) {
  const Thr th;
  constexpr int C = 32 / L;
  const V* __restrict__ val = static_cast<const V*>(S.val);
  const int s1 = __ldg(S.wsl + th.gw + 1);
  for (int sl = __ldg(S.wsl + th.gw); sl < s1; ++sl) {
    const int64_t base = __ldg(S.sp + sl);
    const int w = (int)((__ldg(S.sp + sl + 1) - base) >> 5);
    const int row = __ldg(S.perm + sl * C + th.lane / L);
    const bool owner = row >= 0 && (th.lane % L) == 0;
    const auto pv = pre(owner ? row : -1);
    const int32_t* __restrict__ ci = S.ci + base + th.lane;
    const V* __restrict__ va = val + base + th.lane;
    Acc a0 = Acc(0), a1 = Acc(0);
    int k = 0;
    for (; k + U <= w; k += U) {
      int j[U];
      Acc a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        j[u] = __ldg(ci + (k + u) * 32);
        a[u] = static_cast<Acc>(__ldg(va + (k + u) * 32));
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        a0 += a[u] * static_cast<Acc>(g0(j[u]));
        if (NV == 2) a1 += a[u] * static_cast<Acc>(g1(j[u]));
      }
    }
    for (; k < w; ++k) {
      const int j = __ldg(ci + k * 32);
      const Acc a = static_cast<Acc>(__ldg(va + k * 32));
      a0 += a * static_cast<Acc>(g0(j));
      if (NV == 2) a1 += a * static_cast<Acc>(g1(j));
    }
    if (L > 1) {
      a0 = group_sum<L>(a0);
      if (NV == 2) a1 = group_sum<L>(a1);
    }
    if (owner) epi(row, a0, a1, pv);
  }
}

struct NoPre {};

template <int U, int NV, typename Acc, typename V, typename G0, typename G1, typename Pre, typename Epi>
__device__ __forceinline__ void sell_rows_gp(const SellMat& S, G0& g0, G1& g1, Pre& pre, Epi& epi) {
  switch (S.lanes) {
    case 1: sell_rows_L<1, U, NV, Acc, V>(S, g0, g1, pre, epi); break;
    case 2: sell_rows_L<2, U, NV, Acc, V>(S, g0, g1, pre, epi); break;
    case 4: sell_rows_L<4, U, NV, Acc, V>(S, g0, g1, pre, epi); break;
    case 8: sell_rows_L<8, U, NV, Acc, V>(S, g0, g1, pre, epi); break;
    case 16: sell_rows_L<16, U, NV, Acc, V>(S, g0, g1, pre, epi); break;
    default: sell_rows_L<32, U, NV, Acc, V>(S, g0, g1, pre, epi); break;
  }
}

// Row products without prefetched row operands: epi(row, dot0, dot1).
template <int U, int NV, typename Acc, typename V, typename G0, typename G1, typename Epi>
__device__ __forceinline__ void sell_rows_g(const SellMat& S, G0& g0, G1& g1, Epi& epi) {
  auto pre = [](int) { return NoPre{}; };
  auto e = [&](int row, Acc a0, Acc a1, NoPre) { epi(row, a0, a1); };
  sell_rows_gp<U, NV, Acc, V>(S, g0, g1, pre, e);
}

// Row products with two vectors stored interleaved: gp(k) returns the pair
// (v0_k, v1_k) in one load (float2 / double2); epi(row, dot0, dot1) on the first
// lane of the row.  Each lane keeps U pair gathers in flight.
template <int L, int U, typename Acc, typename V, typename GP, typename Epi>
__device__ __forceinline__ void sell_pair_L(const SellMat& S, GP& gp, Epi& epi) {
  const Thr th;
  constexpr int C = 32 / L;
  const V* __restrict__ val = static_cast<const V*>(S.val);
  const int s1 = __ldg(S.wsl + th.gw + 1);
  for (int sl = __ldg(S.wsl + th.gw); sl < s1; ++sl) {
    const int64_t base = __ldg(S.sp + sl);
    const int w = (int)((__ldg(S.sp + sl + 1) - base) >> 5);
    const int row = __ldg(S.perm + sl * C + th.lane / L);
    const bool owner = row >= 0 && (th.lane % L) == 0;
    const int32_t* __restrict__ ci = S.ci + base + th.lane;
    const V* __restrict__ va = val + base + th.lane;
    Acc a0 = Acc(0), a1 = Acc(0);
    int k = 0;
    for (; k + U <= w; k += U) {
      int j[U];
      Acc a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        j[u] = __ldg(ci + (k + u) * 32);
        a[u] = static_cast<Acc>(__ldg(va + (k + u) * 32));
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const auto g = gp(j[u]);
        a0 += a[u] * static_cast<Acc>(g.x);
        a1 += a[u] * static_cast<Acc>(g.y);
      }
    }
    for (; k < w; ++k) {
      const int j = __ldg(ci + k * 32);
      const Acc a = static_cast<Acc>(__ldg(va + k * 32));
      const auto g = gp(j);
      a0 += a * static_cast<Acc>(g.x);
      a1 += a * static_cast<Acc>(g.y);
    }
    if (L > 1) {
      a0 = group_sum<L>(a0);
      a1 = group_sum<L>(a1);
    }
    if (owner) epi(row, a0, a1);
  }
}

template <int U, typename Acc, typename V, typename GP, typename Epi>
__device__ __forceinline__ void sell_rows_pair(const SellMat& S, GP& gp, Epi& epi) {
  switch (S.lanes) {
    case 1: sell_pair_L<1, U, Acc, V>(S, gp, epi); break;
    case 2: sell_pair_L<2, U, Acc, V>(S, gp, epi); break;
    case 4: sell_pair_L<4, U, Acc, V>(S, gp, epi); break;
    case 8: sell_pair_L<8, U, Acc, V>(S, gp, epi); break;
    case 16: sell_pair_L<16, U, Acc, V>(S, gp, epi); break;
    default: sell_pair_L<32, U, Acc, V>(S, gp, epi); break;
  }
}

// Per-row sum and sum of squares of a SELL matrix with L lanes per row (setup only).
template <int L, typename T, typename V, typename Epi>
__device__ void sell_rowstats_L(const SellMat& S, Epi& epi) {
  const Thr th;
  constexpr int C = 32 / L;
  const V* val = static_cast<const V*>(S.val);
  const int s1 = S.wsl[th.gw + 1];
  for (int sl = S.wsl[th.gw]; sl < s1; ++sl) {
    const int64_t base = S.sp[sl];
    const int w = (int)((S.sp[sl + 1] - base) >> 5);
    const int row = S.perm[sl * C + th.lane / L];
    T sum = T(0), sq = T(0);
    for (int k = 0; k < w; ++k) {
      const T a = static_cast<T>(val[base + k * 32 + th.lane]);
      sum += a;
      sq += a * a;
    }
    if (L > 1) {
      sum = group_sum<L>(sum);
      sq = group_sum<L>(sq);
    }
    if (row >= 0 && (th.lane % L) == 0) epi(row, sum, sq);
  }
}

template <typename T, typename V, typename Epi>
__device__ void sell_rowstats(const SellMat& S, Epi& epi) {
  switch (S.lanes) {
    case 1: sell_rowstats_L<1, T, V>(S, epi); break;
    case 2: sell_rowstats_L<2, T, V>(S, epi); break;
    case 4: sell_rowstats_L<4, T, V>(S, epi); break;
    case 8: sell_rowstats_L<8, T, V>(S, epi); break;
    case 16: sell_rowstats_L<16, T, V>(S, epi); break;
    default: sell_rowstats_L<32, T, V>(S, epi); break;
  }
}

}  // namespace sell
}  // namespace abip
