// Host side of the sliced-ELL (SELL) layout the persistent grid kernels traverse
// (sell.cuh): CSR on the host, its transpose, the SELL form with L lanes per row, the
// number of lanes per row, and the partition of slices among the warps of the grid.
// Included by the C ABI's setup of the sparse path only.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace abip {
namespace sell_host {

struct HostCSR {
  int m = 0, n = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> v;
};

// CSR of A^T by a stable counting sort over columns (row order kept within each column).
inline HostCSR transpose(const HostCSR& A) {
  HostCSR T;
  T.m = A.n;
  T.n = A.m;
  const int64_t nnz = A.rp[A.m];
  T.rp.assign(A.n + 1, 0);
  for (int64_t k = 0; k < nnz; ++k) T.rp[A.ci[k] + 1]++;
  for (int j = 0; j < A.n; ++j) T.rp[j + 1] += T.rp[j];
  std::vector<int64_t> pos(T.rp.begin(), T.rp.end() - 1);
  T.ci.resize(nnz);
  T.v.resize(nnz);
  for (int i = 0; i < A.m; ++i)
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const int64_t at = pos[A.ci[k]]++;
      T.ci[at] = i;
      T.v[at] = A.v[k];
    }
  return T;
}

// SELL form of a CSR matrix with L lanes per row (see SellMat): rows sorted by
// length (longest first, ties in row order), slices of C = 32/L sorted rows;
// within a slice, lane r*L + q holds entries q, q+L, q+2L, ... of row r, stored
// chunk-major and padded to the slice's longest lane with value 0 and a column the
// row already uses (or column 0), so every gather stays in range.
struct HostSell {
  int rows = 0, nslices = 0, lanes = 1;
  std::vector<int64_t> sp;
  std::vector<int32_t> ci;
  std::vector<double> v;
  std::vector<int32_t> perm;
};

// Loads a lane issues for a slice of width w in the device traversal (sell.cuh).
inline double slice_cost(int64_t w) { return (double)w; }

// Contiguous slice ranges per global warp with about equal work (loads of the slice + 2
// for the row bookkeeping).
inline std::vector<int32_t> warp_partition(const HostSell& S, int nwarp) {
  std::vector<int32_t> w(nwarp + 1, 0);
  double total = 0;
  for (int sl = 0; sl < S.nslices; ++sl) total += slice_cost((S.sp[sl + 1] - S.sp[sl]) / 32) + 2.0;
  const double per = total / nwarp;
  double acc = 0;
  int k = 1;
  for (int sl = 0; sl < S.nslices; ++sl) {
    acc += slice_cost((S.sp[sl + 1] - S.sp[sl]) / 32) + 2.0;
    while (k < nwarp && acc >= per * k - 1e-9) w[k++] = sl + 1;
  }
  while (k <= nwarp) w[k++] = S.nslices;
  return w;
}

// lanes per row: the smallest power of two that leaves at most about `per_lane` entries
// per lane.  On the 100000 x 400000 benchmark LP (25 entries per row of A, 6.25 of A^T):
// the FP64 kernel takes 16 (2 lanes for A; 6 % more updates per second than 4 or 8 lanes),
// the mixed-precision kernel, whose traversals batch the tail of a slice, 32 (1 lane for
// A; 4 % faster than 2 lanes, 8 % faster than 4).
inline int sell_lanes(const HostCSR& M, double per_lane) {
  const double mean = M.m > 0 ? (double)M.rp[M.m] / M.m : 0.0;
  int L = 1;
  while (L < 32 && mean > per_lane * L) L *= 2;
  return L;
}

inline HostSell to_sell(const HostCSR& M, int L) {
  HostSell S;
  S.rows = M.m;
  S.lanes = L;
  const int C = 32 / L;
  S.nslices = (M.m + C - 1) / C;
  std::vector<int32_t> order(M.m);
  for (int i = 0; i < M.m; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return (M.rp[a + 1] - M.rp[a]) > (M.rp[b + 1] - M.rp[b]);
  });
  S.perm.assign((size_t)S.nslices * C, -1);
  for (int p = 0; p < M.m; ++p) S.perm[p] = order[p];
  S.sp.assign(S.nslices + 1, 0);
  for (int sl = 0; sl < S.nslices; ++sl) {
    const int r0 = order[(size_t)sl * C];
    const int64_t len = M.rp[r0 + 1] - M.rp[r0];
    const int64_t w = (len + L - 1) / L;          // chunks per lane
    S.sp[sl + 1] = S.sp[sl] + 32 * w;
  }
  S.ci.assign(S.sp[S.nslices], 0);
  S.v.assign(S.sp[S.nslices], 0.0);
  for (int sl = 0; sl < S.nslices; ++sl) {
    const int64_t base = S.sp[sl];
    const int64_t w = (S.sp[sl + 1] - base) / 32;
    for (int r = 0; r < C; ++r) {
      const int row = S.perm[(size_t)sl * C + r];
      const int64_t len = row >= 0 ? M.rp[row + 1] - M.rp[row] : 0;
      const int32_t pad_col = len > 0 ? M.ci[M.rp[row] + len - 1] : 0;
      for (int q = 0; q < L; ++q) {
        for (int64_t c = 0; c < w; ++c) {
          const int64_t k = c * L + q;             // entry of the row
          const int64_t at = base + c * 32 + r * L + q;
          if (k < len) {
            S.ci[at] = M.ci[M.rp[row] + k];
            S.v[at] = M.v[M.rp[row] + k];
          } else {
            S.ci[at] = pad_col;
            S.v[at] = 0.0;
          }
        }
      }
    }
  }
  return S;
}

}  // namespace sell_host
}  // namespace abip
