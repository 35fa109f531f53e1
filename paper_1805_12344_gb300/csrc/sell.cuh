// Sliced-ELL (SELL) row products shared by the persistent grid kernels: the
// thread geometry of a persistent launch, one generic traversal that folds each
// row's stored entries into per-lane accumulators with U gathers in flight per
// lane, and the row products and per-row statistics built on it.
#pragma once

#include <cstdint>
#include <type_traits>

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

// One batch of B entries starting at entry k of the lane's row: the B index and value
// loads, then the B gathers, are issued before the first is used.  Positions at or past
// the slice's width w (none when the batch is full) repeat its last entry with value 0,
// so every gathered index is in range.
template <int B, typename V, typename St, typename GF>
__device__ __forceinline__ void sell_batch(const int32_t* __restrict__ ci, const V* __restrict__ va, int k, int w,
                                           GF& gf, St& st) {
  int j[B];
  V a[B];
#pragma unroll
  for (int u = 0; u < B; ++u) {
    const int kk = min(k + u, w - 1);
    j[u] = __ldg(ci + kk * 32);
    a[u] = k + u < w ? __ldg(va + kk * 32) : V(0);
  }
#pragma unroll
  for (int u = 0; u < B; ++u) st.add(a[u], gf(j[u]));
}

// How a traversal takes the entries of a slice past its last full batch of U: one at a
// time (SerialTail), or in batches of U/2, U/4, ..., 1 (BinaryTail: every load issued
// once, at most log2(U) rounds of loads in flight).  Measured on the 100000 x 400000 LP:
// the binary tail with one lane per row of A is 4 % faster in the mixed-precision kernel;
// the FP64 kernel, with twice the gathered bytes per entry, is 2-4 % faster with the
// serial one.
struct SerialTail { static constexpr bool binary = false; };
struct BinaryTail { static constexpr bool binary = true; };

// Generic SELL traversal over the slices of this warp (S.wsl), L lanes per row.
// For every row: the lane's entries (column j, value a) are folded into an
// accumulator St by st.add(a, gf(j)); the L lanes of the row are combined by
// st.template group<L>(); epi(row, st, pv) runs on the row's first lane with
// pv = pre(row), loaded when the slice starts so the row's own operands arrive while
// the gathers are in flight.  Entries go in batches of U (the U index and value loads,
// then the U gathers, issued before the first is used), the rest of a slice one entry
// at a time (measured on the 100000 x 400000 LP: faster than masked batches, which
// repeat loads).
//   St: default-constructible (zero); add(V a, const G& g) for the gathered type G;
//       template <int L> group().
template <int L, int U, typename V, typename St, typename GF, typename Pre, typename Epi, typename Tail>
__device__ __forceinline__ void sell_fold_L(const SellMat& S, GF& gf, Pre& pre, Epi& epi, Tail) {
  static_assert(!Tail::binary || U == 8, "the binary tail is written for batches of 8");
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
    St st;
    int k = 0;
    for (; k + U <= w; k += U) sell_batch<U, V>(ci, va, k, w, gf, st);
    if constexpr (Tail::binary) {
      if (w - k >= 4) { sell_batch<4, V>(ci, va, k, w, gf, st); k += 4; }
      if (w - k >= 2) { sell_batch<2, V>(ci, va, k, w, gf, st); k += 2; }
      if (k < w) st.add(__ldg(va + k * 32), gf(__ldg(ci + k * 32)));
    } else {
      for (; k < w; ++k) st.add(__ldg(va + k * 32), gf(__ldg(ci + k * 32)));
    }
    if (L > 1) st.template group<L>();
    if (owner) epi(row, st, pv);
  }
}

template <int U, typename V, typename St, typename GF, typename Pre, typename Epi, typename Tail = SerialTail>
__device__ __forceinline__ void sell_fold(const SellMat& S, GF& gf, Pre& pre, Epi& epi, Tail t = Tail{}) {
  switch (S.lanes) {
    case 1: sell_fold_L<1, U, V, St>(S, gf, pre, epi, t); break;
    case 2: sell_fold_L<2, U, V, St>(S, gf, pre, epi, t); break;
    case 4: sell_fold_L<4, U, V, St>(S, gf, pre, epi, t); break;
    case 8: sell_fold_L<8, U, V, St>(S, gf, pre, epi, t); break;
    case 16: sell_fold_L<16, U, V, St>(S, gf, pre, epi, t); break;
    default: sell_fold_L<32, U, V, St>(S, gf, pre, epi, t); break;
  }
}


// One or two dot products accumulated in Acc from a gathered pair (x: first vector,
// y: second vector, unused when NV = 1).
template <typename Acc, typename P, int NV>
struct DotSt {
  using G = P;
  Acc a0 = Acc(0), a1 = Acc(0);
  template <typename V>
  __device__ __forceinline__ void add(V a, const G& g) {
    const Acc av = static_cast<Acc>(a);
    a0 += av * static_cast<Acc>(g.x);
    if (NV == 2) a1 += av * static_cast<Acc>(g.y);
  }
  template <int L>
  __device__ __forceinline__ void group() {
    a0 = group_sum<L>(a0);
    if (NV == 2) a1 = group_sum<L>(a1);
  }
};

template <typename T>
struct Two {
  T x, y;
};
template <typename T>
struct One {
  T x, y;   // y is never read (NV = 1); kept so DotSt compiles for both shapes
};

template <typename P, int NV>
struct MakePair;
template <typename P>
struct MakePair<P, 2> {
  template <typename G0, typename G1>
  __device__ __forceinline__ static P get(G0& g0, G1& g1, int j) {
    P p;
    p.x = g0(j);
    p.y = g1(j);
    return p;
  }
};
template <typename P>
struct MakePair<P, 1> {
  template <typename G0, typename G1>
  __device__ __forceinline__ static P get(G0& g0, G1&, int j) {
    P p;
    p.x = g0(j);
    return p;
  }
};

// Row products for every row of a SELL matrix: dot0 = sum_k A_ik g0(k), dot1 = sum_k
// A_ik g1(k) (NV = 2), accumulated in Acc; epi(row, dot0, dot1, pv) with pv = pre(row)
// on the first lane of the row.  g0/g1 map a column index to the gathered value.
template <int U, int NV, typename Acc, typename V, typename G0, typename G1, typename Pre, typename Epi,
          typename Tail = SerialTail>
__device__ __forceinline__ void sell_rows_gp(const SellMat& S, G0& g0, G1& g1, Pre& pre, Epi& epi, Tail t = Tail{}) {
  using R0 = decltype(g0(0));
  using R1 = decltype(g1(0));
  using R = typename std::conditional<(sizeof(R0) >= sizeof(R1)), R0, R1>::type;
  using P = typename std::conditional<NV == 2, Two<R>, One<R>>::type;
  auto gf = [&](int j) -> P { return MakePair<P, NV>::get(g0, g1, j); };
  auto e = [&](int row, const DotSt<Acc, P, NV>& st, decltype(pre(0)) pv) { epi(row, st.a0, st.a1, pv); };
  sell_fold<U, V, DotSt<Acc, P, NV>>(S, gf, pre, e, t);
}

struct NoPre {};

// Row products without prefetched row operands: epi(row, dot0, dot1).
template <int U, int NV, typename Acc, typename V, typename G0, typename G1, typename Epi,
          typename Tail = SerialTail>
__device__ __forceinline__ void sell_rows_g(const SellMat& S, G0& g0, G1& g1, Epi& epi, Tail t = Tail{}) {
  auto pre = [](int) { return NoPre{}; };
  auto e = [&](int row, Acc a0, Acc a1, NoPre) { epi(row, a0, a1); };
  sell_rows_gp<U, NV, Acc, V>(S, g0, g1, pre, e, t);
}

// Row products with two vectors stored interleaved: gp(k) returns the pair
// (v0_k, v1_k) in one load (float2 / double2); epi(row, dot0, dot1).
template <int U, typename Acc, typename V, typename GP, typename Epi>
__device__ __forceinline__ void sell_rows_pair(const SellMat& S, GP& gp, Epi& epi) {
  using P = decltype(gp(0));
  auto pre = [](int) { return NoPre{}; };
  auto e = [&](int row, const DotSt<Acc, P, 2>& st, NoPre) { epi(row, st.a0, st.a1); };
  sell_fold<U, V, DotSt<Acc, P, 2>>(S, gp, pre, e);
}

// Per-row sum and sum of squares of a SELL matrix, accumulated in T (setup only).
template <typename T>
struct StatSt {
  struct G {};
  T sum = T(0), sq = T(0);
  template <typename V>
  __device__ __forceinline__ void add(V a, const G&) {
    const T t = static_cast<T>(a);
    sum += t;
    sq += t * t;
  }
  template <int L>
  __device__ __forceinline__ void group() {
    sum = group_sum<L>(sum);
    sq = group_sum<L>(sq);
  }
};

template <typename T, typename V, typename Epi>
__device__ void sell_rowstats(const SellMat& S, Epi& epi) {
  using St = StatSt<T>;
  auto gf = [](int) { return typename St::G{}; };
  auto pre = [](int) { return NoPre{}; };
  auto e = [&](int row, const St& st, NoPre) { epi(row, st.sum, st.sq); };
  sell_fold<8, V, St>(S, gf, pre, e);
}

}  // namespace sell
}  // namespace abip
