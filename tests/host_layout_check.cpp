// Invariants of the host-side layouts the sparse kernels read, on seeded random CSR
// matrices (empty rows, ragged lengths, some stored duplicates): the SELL form with L lanes
// per row holds every row's entries in order with zero-valued in-range padding, the warp
// partition covers the slices in order, and the direct projection's arrays hold K's
// entries at their pivot pair with the row structure the exact transpose of the columns.
// Built and run by tests/test_host_layout_cpu.py; prints "ok" and exits 0, or names the
// first broken invariant and exits 1.
#include <cstdio>
#include <cstdlib>
#include <set>
#include <string>
#include <vector>

#include "../paper_1805_12344_gb300/csrc/ldl_host.h"
#include "../paper_1805_12344_gb300/csrc/sell_host.h"

using abip::sell_host::HostCSR;

static uint64_t g_state = 0;
static uint64_t next_u64() {            // splitmix64
  uint64_t z = (g_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static int below(int k) { return (int)(next_u64() % (uint64_t)k); }

static int fail(const std::string& what) {
  std::printf("FAIL %s\n", what.c_str());
  return 1;
}

static HostCSR random_csr(int m, int n, int maxlen) {
  HostCSR A;
  A.m = m;
  A.n = n;
  A.rp.assign(m + 1, 0);
  for (int i = 0; i < m; ++i) {
    const int len = below(5) == 0 ? 0 : below(maxlen + 1);
    std::set<int> cols;
    while ((int)cols.size() < std::min(len, n)) cols.insert(below(n));
    const bool dup = below(6) == 0;               // a stored duplicate of the row's first entry
    for (int j : cols) {
      A.ci.push_back(j);
      A.v.push_back((double)(below(2001) - 1000) / 64.0 + (below(2) ? 0.25 : -0.5));
      if (dup && j == *cols.begin()) {
        A.ci.push_back(j);
        A.v.push_back(0.125 * (1 + below(8)));
      }
    }
    A.rp[i + 1] = (int64_t)A.ci.size();
  }
  return A;
}

static int check_sell(const HostCSR& A, int L) {
  using namespace abip::sell_host;
  const HostSell S = to_sell(A, L);
  const int C = 32 / L;
  if (S.nslices != (A.m + C - 1) / C) return fail("slice count");
  std::vector<int> seen(A.m, 0);
  for (size_t p = 0; p < S.perm.size(); ++p) {
    const int r = S.perm[p];
    if ((int)p < A.m) {
      if (r < 0 || r >= A.m || seen[r]++) return fail("perm is not a permutation of the rows");
      if (p > 0) {
        const int q = S.perm[p - 1];
        const int64_t lq = A.rp[q + 1] - A.rp[q], lr = A.rp[r + 1] - A.rp[r];
        if (lq < lr || (lq == lr && q > r)) return fail("rows not sorted by length, stably");
      }
    } else if (r != -1) {
      return fail("perm tail is not -1");
    }
  }
  for (int sl = 0; sl < S.nslices; ++sl) {
    const int64_t base = S.sp[sl], span = S.sp[sl + 1] - base;
    if (span % 32 != 0) return fail("slice span not a multiple of 32");
    const int64_t w = span / 32;
    for (int r = 0; r < C; ++r) {
      const int row = S.perm[(size_t)sl * C + r];
      const int64_t len = row >= 0 ? A.rp[row + 1] - A.rp[row] : 0;
      if ((len + L - 1) / L > w) return fail("slice narrower than one of its rows");
      for (int q = 0; q < L; ++q)
        for (int64_t c = 0; c < w; ++c) {
          const int64_t k = c * L + q, at = base + c * 32 + r * L + q;
          if (k < len) {
            if (S.ci[at] != A.ci[A.rp[row] + k] || S.v[at] != A.v[A.rp[row] + k]) return fail("entry misplaced");
          } else {
            if (S.v[at] != 0.0) return fail("padding value not zero");
            if (S.ci[at] < 0 || S.ci[at] >= std::max(A.n, 1)) return fail("padding column out of range");
            if (len > 0 && S.ci[at] != A.ci[A.rp[row] + len - 1]) return fail("padding column not the row's last");
          }
        }
    }
  }
  for (int nw : {1, 3, 24, 3648}) {
    const std::vector<int32_t> wp = warp_partition(S, nw);
    if ((int)wp.size() != nw + 1 || wp[0] != 0 || wp[nw] != S.nslices) return fail("partition ends");
    double total = 0, most = 0;
    for (int sl = 0; sl < S.nslices; ++sl) {
      const double c = slice_cost((S.sp[sl + 1] - S.sp[sl]) / 32) + 2.0;
      total += c;
      most = std::max(most, c);
    }
    for (int k = 0; k < nw; ++k) {
      if (wp[k + 1] < wp[k]) return fail("partition not monotone");
      double load = 0;
      for (int sl = wp[k]; sl < wp[k + 1]; ++sl) load += slice_cost((S.sp[sl + 1] - S.sp[sl]) / 32) + 2.0;
      if (load > total / nw + most + 1e-9) return fail("partition unbalanced");
    }
  }
  return 0;
}

static int check_ldl(const HostCSR& A) {
  using namespace abip::ldl_host;
  Symbolic S;
  std::string why;
  if (!analyze(A, S, why)) return fail("analyze: " + why);
  const int N = S.N;
  const std::vector<double> Lx = initial_values(A, S);
  std::vector<double> want(Lx.size(), 0.0);
  auto pos = [&](int p, int r) -> int64_t {
    for (int64_t e = S.Lp[p]; e < S.Lp[p + 1]; ++e)
      if (S.Li[e] == r) return e;
    return -1;
  };
  for (int i = 0; i < A.m; ++i)
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      int p = S.iperm[A.ci[k]], r = S.iperm[A.n + i];
      if (r < p) std::swap(p, r);
      const int64_t e = pos(p, r);
      if (e < 0) return fail("an entry of K is missing from the pattern");
      want[e] += A.v[k];
    }
  for (size_t e = 0; e < Lx.size(); ++e)
    if (Lx[e] != want[e]) return fail("initial value misplaced");
  for (int p = 0; p < N; ++p) {
    if (S.perm[S.iperm[p]] != p) return fail("iperm is not the inverse of perm");
    for (int64_t e = S.Lp[p]; e < S.Lp[p + 1]; ++e) {
      if (S.Li[e] <= p || S.Li[e] >= N) return fail("column entry not below the pivot");
      if (e > S.Lp[p] && S.Li[e] <= S.Li[e - 1]) return fail("column rows not increasing");
    }
  }
  std::vector<int64_t> count(N, 0);
  for (int p = 0; p < N; ++p)
    for (int64_t r = S.Rp[p]; r < S.Rp[p + 1]; ++r) {
      const int k = S.Rk[r];
      const int32_t e = S.Rpos[r];
      if (k >= p || S.Li[e] != p || e < S.Lp[k] || e >= S.Lp[k + 1]) return fail("row entry does not point at L(p, k)");
      if (r > S.Rp[p] && S.Rk[r] <= S.Rk[r - 1]) return fail("row columns not increasing");
      ++count[k];
    }
  for (int k = 0; k < N; ++k)
    if (count[k] != S.Lp[k + 1] - S.Lp[k]) return fail("rows do not cover every column entry once");
  return 0;
}

int main() {
  int cases = 0;
  for (uint64_t seed = 1; seed <= 40; ++seed) {
    g_state = seed * 1000003ull;
    const int m = 1 + below(90), n = m + below(120), maxlen = 1 + below(std::min(n, 70));
    const HostCSR A = random_csr(m, n, maxlen);
    const HostCSR T = abip::sell_host::transpose(A);
    const HostCSR TT = abip::sell_host::transpose(T);
    if (TT.rp != A.rp || TT.ci != A.ci || TT.v != A.v) return fail("transpose twice is not the identity");
    for (int L : {1, 2, 4, 8, 16, 32}) {
      if (check_sell(A, L) || check_sell(T, L)) return 1;
      ++cases;
    }
    if (check_ldl(A)) return 1;
  }
  std::printf("ok %d\n", cases);
  return 0;
}
