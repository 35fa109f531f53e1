// Host presolve of the general LP  min c^T x, A x = b, l <= x <= w  (Sec. 4.5): the
// reductions P1-P7, the reformulation in the standard form the solver takes, a Ruiz
// equilibration (the Remark closing Sec. 4.5) and the postsolve.  Host code only; the
// order of every step is fixed so that the result does not depend on the machine:
//
//  1. Passes until one changes nothing: columns in index order for P3 (l_j > w_j:
//     infeasible) and P4 (l_j = w_j: fixed); rows in index order for P1 (no entry in an
//     active column: dropped when |b_i| <= tol (1 + ||b||_inf), else infeasible) and P6
//     (one entry a_ik: x_k = b_i / a_ik, infeasible when outside [l_k, w_k] by more than
//     tol max(1, |x_k|), else clamped to the bounds); columns in index order for P2 (no
//     entry in an active row: x_j at the bound that minimises c_j x_j, dual infeasible
//     toward an infinite one; c_j = 0 takes the point of [l_j, w_j] nearest 0).  A fixed
//     column leaves the problem: b_r -= a_rj x_j over its active rows, the objective
//     constant gains c_j x_j.
//  2. P7: the over-determined part of the Dulmage-Mendelsohn decomposition of the
//     remaining pattern (rows reached from the rows a maximum matching leaves unmatched,
//     along alternating paths) has rank below its row count; in index order, a row of it
//     that is a combination of the rows kept before it (residual of the orthogonal
//     projection <= tol max(1, ||row||)) is dropped when b agrees with the same
//     combination within tol (1 + ||b||_inf), else the LP is infeasible.
//  3. Standard form, per remaining column in index order: l finite: x = l + xbar, and
//     when w is finite a new row xbar + t = w - l with a new column t (rows after the
//     equality rows, columns after the structural ones); l = -inf, w finite: x = w - xbar
//     (column and cost negated); free (P5): x = x+ - x-.
//  4. `ruiz` passes of D_i /= sqrt(max_j |s_ij|), E_j /= sqrt(max_i |s_ij|) on the scaled
//     matrix S; then Ahat = D A E, bhat = D b, chat = E c.
//  5. Postsolve: x = E xhat, y = D yhat mapped back through 3; fixed columns restored;
//     y = 0 on dropped rows; singleton rows in reverse removal order take
//     y_i = (c_k - sum_{r != i} a_rk y_r) / a_ik (zero reduced cost of the column they
//     fixed); z = c - A^T y.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "abip_internal.h"

struct abip_presolved {
  int status = 0;
  int m0 = 0, n0 = 0;
  // original data, by columns (postsolve)
  std::vector<int64_t> cp;
  std::vector<int32_t> ri;
  std::vector<double> cv;
  std::vector<double> c0;
  // reductions
  std::vector<double> fixed_val;        // per original column (valid where fixed_flag)
  std::vector<char> fixed_flag;
  std::vector<std::pair<int, int>> singleton;   // (row, column) in removal order
  std::vector<int> rows;                // original index of each kept equality row
  struct Col { int j; int kind; double bound; };   // kind 0: l + xbar, 1: w - xbar, 2: free (+, -)
  std::vector<Col> cols;
  // standard form (scaled)
  int m = 0, n = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> v, b, c, D, E;
  double offset = 0.0;
  abip_presolve_info info{};
};

namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();

struct Csr {
  int m = 0, n = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> v;
};

int to_csr(const abip_matrix* A, Csr& M, std::string& why) {
  if (A->on_device) { why = "presolve takes host matrices only (on_device = 0)"; return ABIP_E_INVALID_ARG; }
  if (A->m < 0 || A->n < 1) { why = "need m >= 0 and n >= 1"; return ABIP_E_DIM; }
  if (A->dtype != ABIP_F32 && A->dtype != ABIP_F64) { why = "unknown dtype"; return ABIP_E_INVALID_ARG; }
  M.m = A->m;
  M.n = A->n;
  M.rp.assign(M.m + 1, 0);
  auto val = [&](int64_t k) -> double {
    return A->dtype == ABIP_F64 ? static_cast<const double*>(A->val)[k] : (double)static_cast<const float*>(A->val)[k];
  };
  if (A->fmt == ABIP_DENSE_ROWMAJOR) {
    if (!A->val && M.m > 0) { why = "A.val is NULL"; return ABIP_E_INVALID_ARG; }
    if (A->ld < A->n) { why = "ld < n"; return ABIP_E_DIM; }
    for (int i = 0; i < M.m; ++i) {
      for (int j = 0; j < M.n; ++j) {
        const double a = val((int64_t)i * A->ld + j);
        if (!std::isfinite(a)) { why = "A has non-finite entries"; return ABIP_E_INVALID_ARG; }
        if (a != 0.0) { M.ci.push_back(j); M.v.push_back(a); }
      }
      M.rp[i + 1] = (int64_t)M.ci.size();
    }
  } else if (A->fmt == ABIP_CSR) {
    if (A->nnz < 0 || (M.m > 0 && !A->row_ptr) || (A->nnz > 0 && (!A->col_idx || !A->val))) {
      why = "malformed CSR";
      return ABIP_E_DIM;
    }
    if (M.m > 0 && (A->row_ptr[0] != 0 || A->row_ptr[M.m] != A->nnz)) { why = "malformed CSR"; return ABIP_E_DIM; }
    for (int i = 0; i < M.m; ++i) {
      if (A->row_ptr[i + 1] < A->row_ptr[i]) { why = "malformed CSR"; return ABIP_E_DIM; }
      std::vector<std::pair<int32_t, double>> row;
      for (int64_t k = A->row_ptr[i]; k < A->row_ptr[i + 1]; ++k) {
        const int32_t j = A->col_idx[k];
        const double a = val(k);
        if (j < 0 || j >= M.n) { why = "CSR column index out of range"; return ABIP_E_DIM; }
        if (!std::isfinite(a)) { why = "A has non-finite entries"; return ABIP_E_INVALID_ARG; }
        if (a != 0.0) row.emplace_back(j, a);
      }
      std::stable_sort(row.begin(), row.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
      for (size_t q = 0; q < row.size(); ++q) {
        if (q > 0 && row[q].first == row[q - 1].first) { why = "CSR has a repeated column in a row"; return ABIP_E_DIM; }
        M.ci.push_back(row[q].first);
        M.v.push_back(row[q].second);
      }
      M.rp[i + 1] = (int64_t)M.ci.size();
    }
  } else {
    why = "unknown matrix format";
    return ABIP_E_INVALID_ARG;
  }
  return ABIP_OK;
}

// Columns of a CSR matrix (CSC arrays), rows in increasing order within each column.
void to_csc(const Csr& M, std::vector<int64_t>& cp, std::vector<int32_t>& ri, std::vector<double>& cv) {
  cp.assign(M.n + 1, 0);
  for (int32_t j : M.ci) cp[j + 1]++;
  for (int j = 0; j < M.n; ++j) cp[j + 1] += cp[j];
  ri.resize(M.ci.size());
  cv.resize(M.ci.size());
  std::vector<int64_t> at(cp.begin(), cp.end() - 1);
  for (int i = 0; i < M.m; ++i)
    for (int64_t k = M.rp[i]; k < M.rp[i + 1]; ++k) {
      const int64_t q = at[M.ci[k]]++;
      ri[q] = i;
      cv[q] = M.v[k];
    }
}

// Maximum matching of the rows of a pattern (augmenting paths by depth-first search
// from each row in turn); col_of_row[i] = -1 where unmatched.
void max_matching(int m, int n, const std::vector<std::vector<int>>& adj, std::vector<int>& col_of_row,
                  std::vector<int>& row_of_col) {
  col_of_row.assign(m, -1);
  row_of_col.assign(n, -1);
  std::vector<int> seen(n, -1);
  std::vector<std::pair<int, size_t>> stack;
  std::vector<int> path_col;
  for (int r0 = 0; r0 < m; ++r0) {
    // a free column of the row itself first (most rows of a full-rank pattern find one)
    bool direct = false;
    for (int j : adj[r0])
      if (row_of_col[j] < 0) {
        col_of_row[r0] = j;
        row_of_col[j] = r0;
        direct = true;
        break;
      }
    if (direct) continue;
    // iterative DFS over alternating paths: row -> column -> matched row ...
    stack.clear();
    path_col.clear();
    stack.emplace_back(r0, 0);
    bool found = false;
    while (!stack.empty() && !found) {
      auto& [r, k] = stack.back();
      if (k >= adj[r].size()) {
        stack.pop_back();
        if (!path_col.empty()) path_col.pop_back();
        continue;
      }
      const int j = adj[r][k++];
      if (seen[j] == r0) continue;
      seen[j] = r0;
      path_col.push_back(j);
      if (row_of_col[j] < 0) {
        found = true;
        break;
      }
      stack.emplace_back(row_of_col[j], 0);
    }
    if (!found) continue;
    // augment along the path: stack rows[t] takes path_col[t]
    for (size_t t = 0; t < stack.size(); ++t) {
      const int r = stack[t].first, j = path_col[t];
      col_of_row[r] = j;
      row_of_col[j] = r;
    }
  }
}

}  // namespace

namespace abip {
void set_global_error(const std::string& msg);
}

extern "C" {

int abip_presolve(const abip_matrix* A, const double* b, const double* c, const double* l, const double* w,
                  double tol, int32_t ruiz, abip_presolved** out, abip_presolve_info* info) {
  auto bad = [&](int code, const std::string& msg) {
    abip::set_global_error(msg);
    return code;
  };
  if (!A || !c || !l || !w || !out || (A->m > 0 && !b)) return bad(ABIP_E_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (!(tol > 0.0) || !(tol < 1.0)) return bad(ABIP_E_INVALID_ARG, "tol must be in (0, 1)");
  if (ruiz < 0) return bad(ABIP_E_INVALID_ARG, "ruiz must be >= 0");
  Csr M;
  std::string why;
  int rc = to_csr(A, M, why);
  if (rc) return bad(rc, why);
  const int m0 = M.m, n0 = M.n;
  for (int i = 0; i < m0; ++i)
    if (!std::isfinite(b[i])) return bad(ABIP_E_INVALID_ARG, "b has non-finite entries");
  for (int j = 0; j < n0; ++j) {
    if (!std::isfinite(c[j])) return bad(ABIP_E_INVALID_ARG, "c has non-finite entries");
    if (std::isnan(l[j]) || std::isnan(w[j]) || l[j] == kInf || w[j] == -kInf)
      return bad(ABIP_E_INVALID_ARG, "bounds must be l < +inf, w > -inf, not NaN");
  }
  auto* P = new abip_presolved();
  P->m0 = m0;
  P->n0 = n0;
  to_csc(M, P->cp, P->ri, P->cv);
  P->c0.assign(c, c + n0);
  P->fixed_val.assign(n0, 0.0);
  P->fixed_flag.assign(n0, 0);
  std::vector<double> bw(b, b + m0);
  double bmax = 0.0;
  for (int i = 0; i < m0; ++i) bmax = std::max(bmax, std::fabs(b[i]));
  const double bscale = 1.0 + bmax;
  std::vector<char> row_on(m0, 1), col_on(n0, 1);
  abip_presolve_info& I = P->info;
  std::memset(&I, 0, sizeof(I));
  double offset = 0.0;

  auto fix = [&](int j, double val) {
    col_on[j] = 0;
    P->fixed_flag[j] = 1;
    P->fixed_val[j] = val;
    offset += P->c0[j] * val;
    for (int64_t k = P->cp[j]; k < P->cp[j + 1]; ++k)
      if (row_on[P->ri[k]]) bw[P->ri[k]] -= P->cv[k] * val;
  };
  auto done = [&](int status, const std::string& msg) {
    P->status = status;
    I.status = status;
    abip::set_global_error(msg);
    if (info) *info = I;
    *out = P;
    return ABIP_OK;
  };

  bool changed = true;
  while (changed) {
    changed = false;
    for (int j = 0; j < n0; ++j) {                       // P3, P4
      if (!col_on[j]) continue;
      if (l[j] > w[j]) return done(ABIP_PRIMAL_INFEASIBLE, "P3: l > w at column " + std::to_string(j));
      if (l[j] == w[j]) {
        fix(j, l[j]);
        I.fixed_cols++;
        changed = true;
      }
    }
    for (int i = 0; i < m0; ++i) {                       // P1, P6
      if (!row_on[i]) continue;
      int cnt = 0, k = -1;
      double a = 0.0;
      for (int64_t q = M.rp[i]; q < M.rp[i + 1]; ++q)
        if (col_on[M.ci[q]]) {
          if (++cnt == 1) { k = M.ci[q]; a = M.v[q]; }
          if (cnt > 1) break;
        }
      if (cnt == 0) {
        if (std::fabs(bw[i]) > tol * bscale)
          return done(ABIP_PRIMAL_INFEASIBLE, "P1: empty row " + std::to_string(i) + " with b != 0");
        row_on[i] = 0;
        I.empty_rows++;
        changed = true;
      } else if (cnt == 1) {
        double val = bw[i] / a;
        const double slack = tol * std::max(1.0, std::fabs(val));
        if (val < l[k] - slack || val > w[k] + slack)
          return done(ABIP_PRIMAL_INFEASIBLE, "P6: row " + std::to_string(i) + " fixes column " + std::to_string(k) +
                                                 " outside its bounds");
        val = std::min(std::max(val, l[k]), w[k]);
        row_on[i] = 0;
        P->singleton.emplace_back(i, k);
        fix(k, val);
        I.singleton_rows++;
        changed = true;
      }
    }
    for (int j = 0; j < n0; ++j) {                       // P2
      if (!col_on[j]) continue;
      bool any = false;
      for (int64_t q = P->cp[j]; q < P->cp[j + 1] && !any; ++q) any = row_on[P->ri[q]] != 0;
      if (any) continue;
      double val;
      if (P->c0[j] > 0) {
        if (!std::isfinite(l[j])) return done(ABIP_DUAL_INFEASIBLE, "P2: empty column " + std::to_string(j) + " unbounded below");
        val = l[j];
      } else if (P->c0[j] < 0) {
        if (!std::isfinite(w[j])) return done(ABIP_DUAL_INFEASIBLE, "P2: empty column " + std::to_string(j) + " unbounded below");
        val = w[j];
      } else {
        val = std::min(std::max(0.0, l[j]), w[j]);
      }
      fix(j, val);
      I.empty_cols++;
      changed = true;
    }
  }

  // P7
  std::vector<int> rows, cols, colpos(n0, -1);
  for (int i = 0; i < m0; ++i) if (row_on[i]) rows.push_back(i);
  for (int j = 0; j < n0; ++j) if (col_on[j]) { colpos[j] = (int)cols.size(); cols.push_back(j); }
  {
    const int mr = (int)rows.size(), nc = (int)cols.size();
    std::vector<std::vector<int>> adj(mr);
    for (int t = 0; t < mr; ++t)
      for (int64_t q = M.rp[rows[t]]; q < M.rp[rows[t] + 1]; ++q)
        if (colpos[M.ci[q]] >= 0) adj[t].push_back(colpos[M.ci[q]]);
    std::vector<int> cor, roc;
    max_matching(mr, nc, adj, cor, roc);
    std::vector<char> rseen(mr, 0), cseen(nc, 0);
    std::vector<int> st;
    for (int t = 0; t < mr; ++t) if (cor[t] < 0) { rseen[t] = 1; st.push_back(t); }
    while (!st.empty()) {
      const int t = st.back();
      st.pop_back();
      for (int jj : adj[t]) {
        if (cseen[jj]) continue;
        cseen[jj] = 1;
        const int r = roc[jj];
        if (r >= 0 && !rseen[r]) { rseen[r] = 1; st.push_back(r); }
      }
    }
    std::vector<int> over;
    for (int t = 0; t < mr; ++t) if (rseen[t]) over.push_back(t);
    if (!over.empty()) {
      std::vector<int> bc(nc, -1);                 // column of the block -> dense index
      int nb = 0;
      for (int jj = 0; jj < nc; ++jj) if (cseen[jj]) bc[jj] = nb++;
      // kept rows: orthonormal basis Q (rows, MGS) with K = R Q, R lower triangular
      std::vector<std::vector<double>> Q, R;
      std::vector<double> bk;
      for (int t : over) {
        std::vector<double> v(nb, 0.0);
        for (int64_t q = M.rp[rows[t]]; q < M.rp[rows[t] + 1]; ++q)
          if (colpos[M.ci[q]] >= 0) v[bc[colpos[M.ci[q]]]] = M.v[q];
        double nrm = 0.0;
        for (double x : v) nrm += x * x;
        nrm = std::sqrt(nrm);
        std::vector<double> coef(Q.size(), 0.0);
        for (int pass = 0; pass < 2; ++pass)       // MGS with one reorthogonalisation
          for (size_t u = 0; u < Q.size(); ++u) {
            double d = 0.0;
            for (int e = 0; e < nb; ++e) d += Q[u][e] * v[e];
            coef[u] += d;
            for (int e = 0; e < nb; ++e) v[e] -= d * Q[u][e];
          }
        double res = 0.0;
        for (double x : v) res += x * x;
        res = std::sqrt(res);
        if (res > tol * std::max(1.0, nrm)) {
          for (double& x : v) x /= res;
          Q.push_back(v);
          coef.push_back(res);
          R.push_back(coef);
          bk.push_back(bw[rows[t]]);
          continue;
        }
        // row = coef^T Q = coef^T R^{-1} K: alpha solves R^T alpha = coef
        const size_t kq = Q.size();
        std::vector<double> alpha(coef);
        for (size_t u = kq; u-- > 0;) {
          double s = alpha[u];
          for (size_t q2 = u + 1; q2 < kq; ++q2) s -= R[q2][u] * alpha[q2];
          alpha[u] = s / R[u][u];
        }
        double bt = 0.0;
        for (size_t u = 0; u < kq; ++u) bt += alpha[u] * bk[u];
        if (std::fabs(bw[rows[t]] - bt) > tol * bscale)
          return done(ABIP_PRIMAL_INFEASIBLE, "P7: dependent row " + std::to_string(rows[t]) + " with inconsistent b");
        row_on[rows[t]] = 0;
        I.dependent_rows++;
      }
      rows.clear();
      for (int i = 0; i < m0; ++i) if (row_on[i]) rows.push_back(i);
    }
  }

  // standard form
  const int mk = (int)rows.size();
  std::vector<int> rowpos(m0, -1);
  for (int t = 0; t < mk; ++t) rowpos[rows[t]] = t;
  std::vector<double> bs(mk);
  for (int t = 0; t < mk; ++t) bs[t] = bw[rows[t]];
  // structural columns as lists of (row position, value)
  std::vector<std::vector<std::pair<int, double>>> scol;
  std::vector<double> cost;
  std::vector<std::pair<int, double>> up;        // (structural column, w - l)
  for (int j : cols) {
    std::vector<std::pair<int, double>> e;
    for (int64_t q = P->cp[j]; q < P->cp[j + 1]; ++q)
      if (rowpos[P->ri[q]] >= 0) e.emplace_back(rowpos[P->ri[q]], P->cv[q]);
    if (std::isfinite(l[j])) {
      for (auto& [r, a] : e) bs[r] -= a * l[j];
      offset += P->c0[j] * l[j];
      P->cols.push_back({j, 0, l[j]});
      scol.push_back(e);
      cost.push_back(P->c0[j]);
      if (std::isfinite(w[j])) up.emplace_back((int)scol.size() - 1, w[j] - l[j]);
    } else if (std::isfinite(w[j])) {
      for (auto& [r, a] : e) bs[r] -= a * w[j];
      offset += P->c0[j] * w[j];
      P->cols.push_back({j, 1, w[j]});
      for (auto& pr : e) pr.second = -pr.second;
      scol.push_back(e);
      cost.push_back(-P->c0[j]);
    } else {
      P->cols.push_back({j, 2, 0.0});
      scol.push_back(e);
      for (auto& pr : e) pr.second = -pr.second;
      scol.push_back(e);
      cost.push_back(P->c0[j]);
      cost.push_back(-P->c0[j]);
      I.free_split++;
    }
  }
  const int ns = (int)scol.size(), nu = (int)up.size();
  const int m = mk + nu, n = ns + nu;
  P->m = m;
  P->n = n;
  // rows of the standard form: equality rows from the structural columns, then the bound rows
  std::vector<std::vector<std::pair<int, double>>> srow(m);
  for (int jj = 0; jj < ns; ++jj)
    for (auto& [r, a] : scol[jj]) srow[r].emplace_back(jj, a);
  for (int u = 0; u < nu; ++u) {
    srow[mk + u].emplace_back(up[u].first, 1.0);
    srow[mk + u].emplace_back(ns + u, 1.0);
  }
  P->b = bs;
  for (int u = 0; u < nu; ++u) P->b.push_back(up[u].second);
  P->c = cost;
  P->c.resize(n, 0.0);
  P->rp.assign(m + 1, 0);
  for (int i = 0; i < m; ++i) {
    for (auto& [jj, a] : srow[i]) { P->ci.push_back(jj); P->v.push_back(a); }
    P->rp[i + 1] = (int64_t)P->ci.size();
  }
  I.upper_rows = nu;

  // Ruiz equilibration
  P->D.assign(m, 1.0);
  P->E.assign(n, 1.0);
  std::vector<double> S(P->v);
  std::vector<double> ra(m), ca(n), dr(m), dc(n);
  for (int pass = 0; pass < ruiz; ++pass) {
    std::fill(ra.begin(), ra.end(), 0.0);
    std::fill(ca.begin(), ca.end(), 0.0);
    for (int i = 0; i < m; ++i)
      for (int64_t k = P->rp[i]; k < P->rp[i + 1]; ++k) {
        const double a = std::fabs(S[k]);
        ra[i] = std::max(ra[i], a);
        ca[P->ci[k]] = std::max(ca[P->ci[k]], a);
      }
    for (int i = 0; i < m; ++i) dr[i] = ra[i] > 0 ? 1.0 / std::sqrt(ra[i]) : 1.0;
    for (int j = 0; j < n; ++j) dc[j] = ca[j] > 0 ? 1.0 / std::sqrt(ca[j]) : 1.0;
    for (int i = 0; i < m; ++i) P->D[i] *= dr[i];
    for (int j = 0; j < n; ++j) P->E[j] *= dc[j];
    for (int i = 0; i < m; ++i)
      for (int64_t k = P->rp[i]; k < P->rp[i + 1]; ++k) S[k] = (dr[i] * S[k]) * dc[P->ci[k]];
  }
  for (int i = 0; i < m; ++i)
    for (int64_t k = P->rp[i]; k < P->rp[i + 1]; ++k) P->v[k] = (P->D[i] * P->v[k]) * P->E[P->ci[k]];
  for (int i = 0; i < m; ++i) P->b[i] *= P->D[i];
  for (int j = 0; j < n; ++j) P->c[j] *= P->E[j];
  P->rows = rows;
  P->offset = offset;
  I.m = m;
  I.n = n;
  I.nnz = (int64_t)P->ci.size();
  I.obj_offset = offset;
  // every row went in the reductions (and so every column): the reductions alone solved
  // the LP, and postsolve takes empty x, y
  I.status = m == 0 ? ABIP_OPTIMAL : 0;
  P->status = I.status;
  if (info) *info = I;
  *out = P;
  return ABIP_OK;
}

int abip_presolved_lp(const abip_presolved* P, int64_t* row_ptr, int32_t* col_idx, double* val, double* b,
                      double* c) {
  if (!P) { abip::set_global_error("NULL argument"); return ABIP_E_INVALID_ARG; }
  if (P->status != 0) { abip::set_global_error("presolve decided the status: no reduced LP"); return ABIP_E_INVALID_ARG; }
  if (row_ptr) std::memcpy(row_ptr, P->rp.data(), P->rp.size() * sizeof(int64_t));
  if (col_idx && !P->ci.empty()) std::memcpy(col_idx, P->ci.data(), P->ci.size() * sizeof(int32_t));
  if (val && !P->v.empty()) std::memcpy(val, P->v.data(), P->v.size() * sizeof(double));
  if (b && P->m > 0) std::memcpy(b, P->b.data(), P->m * sizeof(double));
  if (c && P->n > 0) std::memcpy(c, P->c.data(), P->n * sizeof(double));
  return ABIP_OK;
}

int abip_postsolve(const abip_presolved* P, const double* x, const double* y, const double* s, double* x_out,
                   double* y_out, double* z_out, double* obj) {
  (void)s;
  if (!P || !x_out || (P->n > 0 && !x) || (P->m > 0 && !y)) {
    abip::set_global_error("NULL argument");
    return ABIP_E_INVALID_ARG;
  }
  if (P->status != 0 && !(P->status == ABIP_OPTIMAL && P->m == 0)) {
    abip::set_global_error("presolve decided the status: nothing to postsolve");
    return ABIP_E_INVALID_ARG;
  }
  const int n0 = P->n0, m0 = P->m0;
  std::vector<double> xo(n0, 0.0), yo(m0, 0.0);
  for (int j = 0; j < n0; ++j) if (P->fixed_flag[j]) xo[j] = P->fixed_val[j];
  int t = 0;
  for (const auto& col : P->cols) {
    if (col.kind == 0) { xo[col.j] = col.bound + P->E[t] * x[t]; t += 1; }
    else if (col.kind == 1) { xo[col.j] = col.bound - P->E[t] * x[t]; t += 1; }
    else { xo[col.j] = P->E[t] * x[t] - P->E[t + 1] * x[t + 1]; t += 2; }
  }
  for (size_t u = 0; u < P->rows.size(); ++u) yo[P->rows[u]] = P->D[u] * y[u];
  for (size_t q = P->singleton.size(); q-- > 0;) {
    const int i = P->singleton[q].first, k = P->singleton[q].second;
    double acc = P->c0[k], aik = 0.0;
    for (int64_t e = P->cp[k]; e < P->cp[k + 1]; ++e) {
      if (P->ri[e] == i) aik = P->cv[e];
      else acc -= P->cv[e] * yo[P->ri[e]];
    }
    yo[i] = acc / aik;
  }
  if (z_out) {
    for (int j = 0; j < n0; ++j) {
      double zj = P->c0[j];
      for (int64_t e = P->cp[j]; e < P->cp[j + 1]; ++e) zj -= P->cv[e] * yo[P->ri[e]];
      z_out[j] = zj;
    }
  }
  if (obj) {
    double o = 0.0;
    for (int j = 0; j < n0; ++j) o += P->c0[j] * xo[j];
    *obj = o;
  }
  std::memcpy(x_out, xo.data(), n0 * sizeof(double));
  if (y_out && m0 > 0) std::memcpy(y_out, yo.data(), m0 * sizeof(double));
  return ABIP_OK;
}

void abip_presolve_free(abip_presolved* P) { delete P; }

}  // extern "C"
