// Host symbolic analysis of the sparse direct projection (Sec. 4.4): the projection's
// linear system with M = [[I, A], [-A^T, I]] is rewritten, with yhat = -y, as the
// quasi-definite system
//
//     K [x; yhat] = [r_x; r_y],      K = [[I_n, A^T], [A, -I_m]],
//
// whose symmetric permutations all have an LDL^T factorisation with D_p > 0 for the
// pivots of the I_n block and D_p < 0 for those of the -I_m block (quasi-definite
// matrices are strongly factorisable).  This file orders K by minimum degree, reads
// the pattern of L off the elimination graph, and builds the arrays the device
// factorisation and solves use.  Integer work only: the same result on every host.
//
// Node numbering of K: x_j is node j (0 <= j < n), yhat_i is node n + i.
#pragma once

#include <algorithm>
#include <climits>
#include <cstdint>
#include <functional>
#include <queue>
#include <string>
#include <utility>
#include <vector>

#include "sell_host.h"

namespace abip {
namespace ldl_host {

// Limits of the analysis: past them the factor is not worth forming on this path.
constexpr int64_t kMaxFactorNnz = 400000000;        // entries of L (3.2 GB of FP64 values)
constexpr int64_t kMaxWork = 1000000000;            // merge steps of the elimination graph (a few seconds)

struct Symbolic {
  int n = 0, m = 0, N = 0;
  std::vector<int32_t> perm;   // perm[p]: node of the p-th pivot
  std::vector<int32_t> iperm;  // iperm[node] = p
  std::vector<int64_t> Lp;     // N + 1: column p of L (strictly lower) is Li[Lp[p] .. Lp[p+1])
  std::vector<int32_t> Li;     // row indices, increasing within a column
  std::vector<int64_t> Rp;     // N + 1: row p of L (strictly lower) is Rk[Rp[p] .. Rp[p+1])
  std::vector<int32_t> Rk;     // columns k < p of row p, increasing
  std::vector<int32_t> Rpos;   // position of L(p, k) in Li
  int64_t work = 0;            // merge steps the ordering took
};

// Minimum-degree elimination of the graph of K.  The graph's edges are x_j -- yhat_i for
// every stored A_ij.  Eliminating a node joins its remaining neighbours into a clique;
// the neighbours at that moment are the pattern of its column of L.  Ties are broken by
// the smaller node number.  Once the remaining graph is complete (the least degree is
// the number of other remaining nodes) the rest is ordered by node number.
// Returns false (with `why`) past kMaxFactorNnz or kMaxWork.
inline bool analyze(const sell_host::HostCSR& A, Symbolic& S, std::string& why) {
  if ((int64_t)A.m + A.n > (int64_t)INT32_MAX) { why = "m + n does not fit the factor's 32-bit indices"; return false; }
  const int m = A.m, n = A.n, N = m + n;
  S.n = n; S.m = m; S.N = N;
  std::vector<std::vector<int32_t>> adj(N);
  {
    const sell_host::HostCSR AT = sell_host::transpose(A);
    for (int j = 0; j < n; ++j) {
      auto& a = adj[j];
      for (int64_t k = AT.rp[j]; k < AT.rp[j + 1]; ++k) a.push_back(n + AT.ci[k]);
      std::sort(a.begin(), a.end());
      a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    for (int i = 0; i < m; ++i) {
      auto& a = adj[n + i];
      for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) a.push_back(A.ci[k]);
      std::sort(a.begin(), a.end());
      a.erase(std::unique(a.begin(), a.end()), a.end());
    }
  }
  using Entry = std::pair<int64_t, int32_t>;   // (degree, node)
  std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> heap;
  for (int v = 0; v < N; ++v) heap.push(Entry((int64_t)adj[v].size(), v));
  std::vector<char> gone(N, 0);
  std::vector<std::vector<int32_t>> pat(N);   // pattern of each node's column, node numbers
  S.perm.clear();
  S.perm.reserve(N);
  int64_t nnz = 0, work = 0;
  int remaining = N;
  std::vector<int32_t> merged;
  while (remaining > 0) {
    const Entry e = heap.top();
    heap.pop();
    const int v = e.second;
    if (gone[v] || e.first != (int64_t)adj[v].size()) continue;   // stale entry
    if (e.first == remaining - 1 && remaining > 1) {
      // complete graph: the rest in node order, each column holding every later node
      std::vector<int32_t> rest;
      for (int u = 0; u < N; ++u)
        if (!gone[u]) rest.push_back(u);
      const int64_t r = (int64_t)rest.size();
      nnz += r * (r - 1) / 2;
      if (nnz > kMaxFactorNnz) { why = "the factor would hold more than 4e8 nonzeros"; return false; }
      for (int64_t a = 0; a < r; ++a) {
        pat[rest[a]].assign(rest.begin() + a + 1, rest.end());
        S.perm.push_back(rest[a]);
        gone[rest[a]] = 1;
      }
      remaining = 0;
      break;
    }
    // eliminate v
    std::vector<int32_t>& nb = adj[v];
    nnz += (int64_t)nb.size();
    if (nnz > kMaxFactorNnz) { why = "the factor would hold more than 4e8 nonzeros"; return false; }
    for (const int32_t u : nb) {
      const std::vector<int32_t>& au = adj[u];
      merged.clear();
      merged.reserve(au.size() + nb.size());
      size_t a = 0, b = 0;
      while (a < au.size() || b < nb.size()) {
        int32_t w;
        if (b >= nb.size() || (a < au.size() && au[a] < nb[b])) w = au[a++];
        else if (a >= au.size() || nb[b] < au[a]) w = nb[b++];
        else { w = au[a]; ++a; ++b; }
        if (w != u && w != v) merged.push_back(w);
      }
      work += (int64_t)(au.size() + nb.size());
      adj[u].swap(merged);
      heap.push(Entry((int64_t)adj[u].size(), u));
    }
    if (work > kMaxWork) { why = "the minimum-degree ordering exceeded its work limit"; return false; }
    pat[v].swap(nb);
    nb.clear();
    nb.shrink_to_fit();
    gone[v] = 1;
    S.perm.push_back(v);
    --remaining;
  }
  S.work = work;
  S.iperm.assign(N, 0);
  for (int p = 0; p < N; ++p) S.iperm[S.perm[p]] = p;
  // columns of L in pivot numbering, rows increasing
  S.Lp.assign(N + 1, 0);
  for (int p = 0; p < N; ++p) S.Lp[p + 1] = S.Lp[p] + (int64_t)pat[S.perm[p]].size();
  S.Li.resize(S.Lp[N]);
  for (int p = 0; p < N; ++p) {
    const std::vector<int32_t>& pv = pat[S.perm[p]];
    int32_t* dst = S.Li.data() + S.Lp[p];
    for (size_t k = 0; k < pv.size(); ++k) dst[k] = S.iperm[pv[k]];
    std::sort(dst, dst + pv.size());
    if (!pv.empty() && dst[0] <= p) { why = "internal: a column pattern reaches above its pivot"; return false; }
  }
  // rows of L: counting sort of the column entries by row
  S.Rp.assign(N + 1, 0);
  for (int64_t e = 0; e < S.Lp[N]; ++e) ++S.Rp[S.Li[e] + 1];
  for (int p = 0; p < N; ++p) S.Rp[p + 1] += S.Rp[p];
  S.Rk.resize(S.Lp[N]);
  S.Rpos.resize(S.Lp[N]);
  std::vector<int64_t> next(S.Rp.begin(), S.Rp.end() - 1);
  for (int p = 0; p < N; ++p)
    for (int64_t e = S.Lp[p]; e < S.Lp[p + 1]; ++e) {
      const int64_t at = next[S.Li[e]]++;
      S.Rk[at] = p;
      S.Rpos[at] = (int32_t)e;
    }
  return true;
}

// Strictly-lower values of P K P^T on the pattern of L (fill entries 0): column p holds
// K(node(i), node(p)) for its rows i, i.e. A_ij between x_j and yhat_i (duplicates of a
// stored entry summed).  The diagonal of K is +1 (x) / -1 (yhat) and is not stored.
inline std::vector<double> initial_values(const sell_host::HostCSR& A, const Symbolic& S) {
  const int n = S.n;
  std::vector<double> Lx(S.Li.size(), 0.0);
  auto put = [&](int node_row, int node_col, double v) {
    int p = S.iperm[node_col], r = S.iperm[node_row];
    if (r < p) std::swap(r, p);
    const int32_t* b = S.Li.data() + S.Lp[p];
    const int32_t* e = S.Li.data() + S.Lp[p + 1];
    const int32_t* at = std::lower_bound(b, e, r);
    Lx[(size_t)(at - S.Li.data())] += v;   // present: every edge of K is in the pattern
  };
  for (int i = 0; i < A.m; ++i)
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) put(n + i, A.ci[k], A.v[k]);
  return Lx;
}

}  // namespace ldl_host
}  // namespace abip
