// C ABI of libabip (declared in include/abip.h): validation, device memory,
// launches of the persistent kernels, and result marshalling.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <type_traits>
#include <vector>

#include "abip_device.cuh"
#include "abip_internal.h"
#include "ldl_host.h"
#include "sell_host.h"

using abip::BackwardInst;
using abip::DenseInst;
using abip::DenseParams;
using abip::GridData;
using abip::SellMat;
using abip::SolveCtl;
using abip::sell_host::HostCSR;
using abip::sell_host::HostSell;
using abip::sell_host::sell_lanes;
using abip::sell_host::to_sell;
using abip::sell_host::transpose;
using abip::sell_host::warp_partition;

namespace {

thread_local std::string g_err = "";

int fail(abip_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_err = msg;
  return code;
}

}  // namespace

namespace abip {
void set_global_error(const std::string& msg) { g_err = msg; }
}  // namespace abip

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// copy n elements of T from host or device memory to a host vector
template <typename T>
cudaError_t fetch(const T* src, size_t n, bool dev, std::vector<T>& out) {
  out.resize(n);
  if (n == 0) return cudaSuccess;
  if (dev) return cudaMemcpy(out.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost);
  std::memcpy(out.data(), src, n * sizeof(T));
  return cudaSuccess;
}

// bump allocator over one cudaMalloc; every block aligned to 256 bytes
struct Arena {
  size_t off = 0;
  char* base = nullptr;
  template <typename T>
  T* take(size_t n) {
    const size_t at = off;
    off += ((n * sizeof(T) + 255) / 256) * 256;
    return base ? reinterpret_cast<T*>(base + at) : nullptr;
  }
};

template <typename T>
__global__ void fill_kernel(T* p, int64_t n, T v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

template <typename T>
__global__ void convert_kernel(const double* src, T* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = static_cast<T>(src[i]);
}

// user outputs from the raw state: scaled candidate or certificate (Sec. 4.1)
template <typename T>
__global__ void output_kernel(const T* v, int64_t n, double scale, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = static_cast<double>(v[i]) * scale;
}

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

int device_error_code(int err) {
  switch (err) {
    case abip::DEV_ERR_BARRIER_TIMEOUT: return ABIP_E_TIMEOUT;
    default: return ABIP_E_NUMERICAL;
  }
}

const char* device_error_str(int err) {
  switch (err) {
    case abip::DEV_ERR_BARRIER_TIMEOUT: return "grid barrier wait timed out";
    case abip::DEV_ERR_PCG: return "PCG exceeded cg_max_iter";
    case abip::DEV_ERR_NONFINITE: return "non-finite value in a reduction";
    case abip::DEV_ERR_CHOLESKY: return "Cholesky factorisation of I + A A^T broke down";
    case abip::DEV_ERR_LDL: return "sparse LDL^T factorisation of the quasi-definite system broke down";
    default: return "device error";
  }
}

int check_params(const abip_params& p, std::string& why) {
  if (!(p.beta > 0) || !std::isfinite(p.beta)) { why = "beta must be > 0"; return 0; }
  if (!(p.gamma > 0 && p.gamma < 1)) { why = "gamma must be in (0, 1)"; return 0; }
  if (!(p.alpha > 0 && p.alpha < 2)) { why = "alpha must be in (0, 2)"; return 0; }
  if (!(p.eps > 0)) { why = "eps must be > 0"; return 0; }
  if (p.max_admm_iters < 1) { why = "max_admm_iters must be >= 1"; return 0; }
  if (!(p.cg_tol > 0)) { why = "cg_tol must be > 0"; return 0; }
  if (!(p.cg_rel >= 0)) { why = "cg_rel must be >= 0"; return 0; }
  if (p.cg_max_iter < 1) { why = "cg_max_iter must be >= 1"; return 0; }
  if (p.precision != ABIP_PREC_F64 && p.precision != ABIP_PREC_MIXED && p.precision != ABIP_PREC_MIXED_BF16) {
    why = "unknown precision";
    return 0;
  }
  if (p.linsys != ABIP_LINSYS_DENSE_CHOL && p.linsys != ABIP_LINSYS_PCG && p.linsys != ABIP_LINSYS_SPARSE_LDL &&
      p.linsys != -1) {
    why = "unknown linsys";
    return 0;
  }
  if (p.linsys == ABIP_LINSYS_SPARSE_LDL && p.precision != ABIP_PREC_F64) {
    why = "the sparse direct projection (linsys = SPARSE_LDL) runs in FP64 (precision = F64)";
    return 0;
  }
  if (p.warmstart != 0 && p.warmstart != 1) { why = "warmstart must be 0 or 1"; return 0; }
  if (p.cg_warm < 0 || p.cg_warm > 2) { why = "cg_warm must be 0, 1 or 2"; return 0; }
  if (p.stop_rule != 0 && p.stop_rule != 1) { why = "stop_rule must be 0 or 1"; return 0; }
  if (p.barrier_limit_ns < 0) { why = "barrier_limit_ns must be >= 0"; return 0; }
  if (p.bb_beta != 0 && p.bb_beta != 1) { why = "bb_beta must be 0 or 1"; return 0; }
  if (!(p.gamma_max == 0.0 || (p.gamma_max >= p.gamma && p.gamma_max < 1.0))) {
    why = "gamma_max must be 0 (off) or in [gamma, 1)";
    return 0;
  }
  if (p.autotune != 0 && p.autotune != 1) { why = "autotune must be 0 or 1"; return 0; }
  if (p.batch_order != 0 && p.batch_order != 1) { why = "batch_order must be 0 or 1"; return 0; }
  if (p.bb_beta && (p.bb_max_redo < 0 || !(p.eps_cor >= 0) || !(p.eps_penalty >= 0))) {
    why = "bb_max_redo, eps_cor and eps_penalty must be >= 0";
    return 0;
  }
  return 1;
}

// ---------------------------------------------------------------------------
// CSR grid path
// ---------------------------------------------------------------------------

void assign_vectors(GridData<double>& g, Arena& ar, int m, int n) {
  using T = double;
  g.b = ar.take<T>(m);
  g.c = ar.take<T>(n);
  g.bbar = ar.take<T>(m); g.cbar = ar.take<T>(n); g.dinv = ar.take<T>(m);
  g.g1y = ar.take<T>(m); g.g1x = ar.take<T>(n); g.g2y = ar.take<T>(m); g.g2x = ar.take<T>(n);
  g.y = ar.take<T>(m); g.x = ar.take<T>(n); g.s = ar.take<T>(n);
  g.Ax = ar.take<T>(m); g.As = ar.take<T>(m); g.ATy = ar.take<T>(n);
  g.zy = ar.take<T>(m); g.zx = ar.take<T>(n); g.zp2 = ar.take<T>(m); g.zp3 = ar.take<T>(m);
  g.r = ar.take<T>(m); g.p = ar.take<T>(m); g.Gp = ar.take<T>(m);
  g.ut = ar.take<double2>(n); g.zd = ar.take<double2>(m); g.zd2 = ar.take<double2>(m);
}

void assign_vectors(abip::GridDelta& g, Arena& ar, int m, int n) {
  g.b = ar.take<double>(m);
  g.c = ar.take<double>(n);
  g.bbar = ar.take<double>(m); g.cbar = ar.take<double>(n);
  g.g1y = ar.take<double>(m); g.g1x = ar.take<double>(n); g.g2y = ar.take<double>(m); g.g2x = ar.take<double>(n);
  g.y = ar.take<double>(m); g.x = ar.take<double>(n); g.s = ar.take<double>(n);
  g.Ax = ar.take<double>(m); g.As = ar.take<double>(m); g.ATy = ar.take<double>(n);
  g.zy = ar.take<double>(m); g.ATz = ar.take<double>(n);
  g.dinv = ar.take<float>(m); g.dz = ar.take<float>(m); g.d1 = ar.take<float>(m); g.d2 = ar.take<float>(m);
  g.r = ar.take<float>(m); g.p = ar.take<float>(m); g.Gp = ar.take<float>(m);
  g.ut = ar.take<float2>(n); g.zd = ar.take<float2>(m); g.zd2 = ar.take<float2>(m);
  g.wdel = ar.take<float>(n); g.xsw = ar.take<abip::XSW>(n); g.dy = ar.take<float>(m);
}

// Arrays of the sparse direct projection (FP64 path only): the factor's pattern, K's
// values on it (factored in place by the setup launch), pivots, sweep values, flags and
// the LdlView the device routines read.  `view` receives the host copy of that view.
void layout_ldl(Arena& ar, GridData<double>& g, const abip::ldl_host::Symbolic* sym, abip::LdlView& view) {
  g.ldl_N = 0;
  g.ldlv = nullptr;
  view = abip::LdlView{};
  if (!sym) return;
  const int N = sym->N;
  const size_t nz = sym->Li.size();
  abip::LdlDev& L = view.F;
  L.N = N;
  L.perm = ar.take<int32_t>(N);
  L.Lp = ar.take<int64_t>((size_t)N + 1);
  L.Li = ar.take<int32_t>(nz);
  L.Lx = ar.take<double>(nz);
  L.Rp = ar.take<int64_t>((size_t)N + 1);
  L.Rk = ar.take<int32_t>(nz);
  L.Rpos = ar.take<int32_t>(nz);
  L.Dd = ar.take<double>(N);
  L.zf = ar.take<double>(2 * (size_t)N);
  L.wb = ar.take<double>(2 * (size_t)N);
  L.flag = ar.take<unsigned long long>(N);
  view.m = g.m; view.n = g.n;
  view.b = g.b; view.c = g.c; view.bbar = g.bbar; view.cbar = g.cbar;
  view.y = g.y; view.x = g.x; view.s = g.s; view.zy = g.zy; view.zx = g.zx;
  view.g1y = g.g1y; view.g1x = g.g1x; view.g2y = g.g2y; view.g2x = g.g2x;
  view.partials = g.partials;
  view.ctl = g.ctl;
  g.ldlv = ar.take<abip::LdlView>(1);
  g.ldl_N = N;
}
void layout_ldl(Arena&, abip::GridDelta&, const abip::ldl_host::Symbolic*, abip::LdlView&) {}

void upload_ldl(const GridData<double>& g, const abip::ldl_host::Symbolic* sym, const std::vector<double>* lx0,
                const abip::LdlView& view) {
  if (!sym) return;
  const abip::LdlDev& L = view.F;
  const size_t nz = sym->Li.size();
  cudaMemcpy((void*)L.perm, sym->perm.data(), sym->perm.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy((void*)L.Lp, sym->Lp.data(), sym->Lp.size() * 8, cudaMemcpyHostToDevice);
  cudaMemcpy((void*)L.Rp, sym->Rp.data(), sym->Rp.size() * 8, cudaMemcpyHostToDevice);
  if (nz > 0) {
    cudaMemcpy((void*)L.Li, sym->Li.data(), nz * 4, cudaMemcpyHostToDevice);
    cudaMemcpy((void*)L.Lx, lx0->data(), nz * 8, cudaMemcpyHostToDevice);
    cudaMemcpy((void*)L.Rk, sym->Rk.data(), nz * 4, cudaMemcpyHostToDevice);
    cudaMemcpy((void*)L.Rpos, sym->Rpos.data(), nz * 4, cudaMemcpyHostToDevice);
  }
  const std::vector<unsigned long long> empty(2 * (size_t)L.N, abip::kLdlEmpty);
  cudaMemcpy((void*)L.zf, empty.data(), empty.size() * 8, cudaMemcpyHostToDevice);
  cudaMemcpy((void*)L.wb, empty.data(), empty.size() * 8, cudaMemcpyHostToDevice);
  cudaMemcpy((void*)g.ldlv, &view, sizeof(view), cudaMemcpyHostToDevice);
}
void upload_ldl(const abip::GridDelta&, const abip::ldl_host::Symbolic*, const std::vector<double>*,
                const abip::LdlView&) {}

cudaError_t launch_persistent(abip_handle* h, cudaStream_t st) {
  if (h->mixed) return abip::launch_grid_delta(h->gdd, h->grid, st);
  return abip::launch_grid_solver_f64(h->gd64, h->val_f64 != 0, h->grid, st);
}

// Setup of the sparse path for one LP: SELL copies of A and A^T, the device arena of G
// (GridData<double> for FP64, GridDelta for mixed precision) and one launch of the
// persistent kernel in MODE_SETUP.  vf64: store A's values as double.  sym / lx0 (FP64
// only): the symbolic factor of the direct projection and K's values on its pattern; the
// setup launch factors it.  Null: the projection runs Jacobi-PCG.
template <typename G>
int setup_grid_path(abip_handle* h, G& g, const HostCSR& A, const std::vector<double>& b,
                    const std::vector<double>& c, bool vf64, int maxc,
                    const abip::ldl_host::Symbolic* sym = nullptr, const std::vector<double>* lx0 = nullptr) {
  const int m = A.m, n = A.n;
  HostCSR AT = transpose(A);
  h->val_f64 = vf64 ? 1 : 0;
  const size_t vb = vf64 ? 8 : 4;
  if (maxc <= 0) return fail(h, ABIP_E_CUDA, "grid kernel cannot be made resident");
  // grid_total reads at most kGridTotalPer partials per thread
  const int cap = std::min(maxc, abip::kGridTotalPer * 32);
  int grid = h->prm.grid_ctas > 0 ? std::min(h->prm.grid_ctas, cap) : cap;
  h->grid = grid;

  constexpr bool delta = std::is_same<G, abip::GridDelta>::value;
  const double per_lane = delta ? 32.0 : 16.0;
  const HostSell SA = to_sell(A, sell_lanes(A, per_lane)), ST = to_sell(AT, sell_lanes(AT, per_lane));
  const int wpc = abip::kGridThreads / 32;
  const std::vector<int32_t> wpA = warp_partition(SA, grid * wpc), wpT = warp_partition(ST, grid * wpc);

  auto layout_sell = [&](Arena& ar, SellMat& M, const HostSell& H) {
    M.rows = H.rows;
    M.nslices = H.nslices;
    M.lanes = H.lanes;
    M.sp = ar.take<int64_t>(H.nslices + 1);
    M.ci = ar.take<int32_t>(H.ci.size());
    M.val = ar.take<char>(H.ci.size() * vb);
    M.perm = ar.take<int32_t>(H.perm.size());
    M.wsl = ar.take<int32_t>((size_t)grid * (abip::kGridThreads / 32) + 1);
  };
  abip::LdlView ldl_view;   // direct projection: host copy of the device view
  auto layout = [&](Arena& ar, G& gg) {
    h->ctl = ar.take<SolveCtl>(1);
    layout_sell(ar, gg.A, SA);
    layout_sell(ar, gg.AT, ST);
    assign_vectors(gg, ar, m, n);
    gg.partials = ar.take<double>((size_t)abip::kNumSlots * grid);
    gg.bar = ar.take<unsigned long long>(1);
    h->stage = ar.take<double>((size_t)m + 2 * (size_t)n);
    gg.m = m; gg.n = n;
    gg.ctl = h->ctl;
    layout_ldl(ar, gg, sym, ldl_view);
  };
  Arena probe;
  G tmp{};
  layout(probe, tmp);
  void* mem = nullptr;
  if (cudaMalloc(&mem, probe.off) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, ABIP_E_OOM, "device allocation of " + std::to_string(probe.off) + " bytes failed");
  }
  h->arena = mem;
  h->arena_bytes = probe.off;
  Arena ar;
  ar.base = static_cast<char*>(mem);
  g = G{};
  layout(ar, g);
  g.m = m; g.n = n;
  g.ctl = h->ctl;
  h->padded_nnz_a = (int64_t)SA.ci.size();
  h->padded_nnz_at = (int64_t)ST.ci.size();
  cudaMemset(mem, 0, probe.off);
  auto upload_sell = [&](const SellMat& M, const HostSell& H, const std::vector<int32_t>& wp) {
    cudaMemcpy((void*)M.sp, H.sp.data(), H.sp.size() * 8, cudaMemcpyHostToDevice);
    cudaMemcpy((void*)M.ci, H.ci.data(), H.ci.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy((void*)M.perm, H.perm.data(), H.perm.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy((void*)M.wsl, wp.data(), wp.size() * 4, cudaMemcpyHostToDevice);
    if (vf64) {
      cudaMemcpy((void*)M.val, H.v.data(), H.v.size() * 8, cudaMemcpyHostToDevice);
    } else {
      std::vector<float> f(H.v.begin(), H.v.end());
      cudaMemcpy((void*)M.val, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
    }
  };
  upload_sell(g.A, SA, wpA);
  upload_sell(g.AT, ST, wpT);
  upload_ldl(g, sym, lx0, ldl_view);
  cudaMemcpy((void*)g.b, b.data(), m * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy((void*)g.c, c.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  SolveCtl hc{};
  hc.beta = h->prm.beta; hc.gamma = h->prm.gamma; hc.alpha = h->prm.alpha; hc.eps = h->prm.eps;
  hc.gamma_max = h->prm.gamma_max;
  hc.cg_tol = h->prm.cg_tol; hc.cg_rel = h->prm.cg_rel; hc.cg_max = h->prm.cg_max_iter; hc.max_admm = h->prm.max_admm_iters;
  hc.warmstart = h->prm.warmstart; hc.stop_rule = h->prm.stop_rule; hc.check_every = std::max(1, h->prm.check_every);
  hc.cg_warm = h->prm.cg_warm;
  hc.bar_limit_ns = (unsigned long long)h->prm.barrier_limit_ns;
  hc.mode = abip::MODE_SETUP;
  cudaMemcpy(h->ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, ABIP_E_CUDA, std::string("setup copies: ") + cudaGetErrorString(e));
  e = launch_persistent(h, 0);
  if (e != cudaSuccess) return fail(h, ABIP_E_CUDA, std::string("setup launch: ") + cudaGetErrorString(e));
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(h, ABIP_E_CUDA, std::string("setup kernel: ") + cudaGetErrorString(e));
  cudaMemcpy(&hc, h->ctl, sizeof(hc), cudaMemcpyDeviceToHost);
  if (hc.err != 0) return fail(h, device_error_code(hc.err), std::string("setup: ") + device_error_str(hc.err));
  const double det = hc.K[0] * hc.K[3] - hc.K[1] * hc.K[2];
  if (!std::isfinite(det) || det == 0.0) return fail(h, ABIP_E_NUMERICAL, "singular Schur complement");
  hc.Kinv[0] = hc.K[3] / det; hc.Kinv[1] = -hc.K[1] / det; hc.Kinv[2] = -hc.K[2] / det; hc.Kinv[3] = hc.K[0] / det;
  hc.zbar = hc.sum_c + 1.0;
  hc.xi = -(double)n - 1.0;
  hc.nb = std::sqrt(hc.sum_b2);
  hc.nc = std::sqrt(hc.sum_c2);
  h->nb = hc.nb;
  h->nc = hc.nc;
  cudaMemcpy(h->ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice);
  return ABIP_OK;
}

// Start vectors of a solve on the sparse path: Algorithm 2's start (or the state set
// by abip_set_state) and a cold projection (z_y = 0, no previous solutions).
void init_grid_state(abip_handle* h, cudaStream_t st) {
  const int m = h->m, n = h->n;
  double* y = h->mixed ? h->gdd.y : h->gd64.y;
  double* x = h->mixed ? h->gdd.x : h->gd64.x;
  double* s = h->mixed ? h->gdd.s : h->gd64.s;
  if (h->resume) {
    const std::vector<double>& rs = h->resume_state;
    cudaMemcpyAsync(y, rs.data(), m * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(x, rs.data() + m, n * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s, rs.data() + m + n + 2, n * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
  } else {
    fill_kernel<double><<<64, 256, 0, st>>>(y, m, 0.0);
    fill_kernel<double><<<256, 256, 0, st>>>(x, n, 1.0);
    fill_kernel<double><<<256, 256, 0, st>>>(s, n, 1.0);
  }
  if (h->mixed) {
    abip::GridDelta& g = h->gdd;
    fill_kernel<double><<<64, 256, 0, st>>>(g.zy, m, 0.0);
    fill_kernel<float><<<64, 256, 0, st>>>(g.d1, m, 0.f);
    fill_kernel<float><<<64, 256, 0, st>>>(g.d2, m, 0.f);
    fill_kernel<float><<<64, 256, 0, st>>>(g.dz, m, 0.f);
  } else {
    GridData<double>& g = h->gd64;
    fill_kernel<double><<<64, 256, 0, st>>>(g.zy, m, 0.0);
    fill_kernel<double><<<64, 256, 0, st>>>(g.zp2, m, 0.0);
    fill_kernel<double><<<64, 256, 0, st>>>(g.zp3, m, 0.0);
  }
}

int solve_grid_path(abip_handle* h, cudaStream_t st) {
  const int m = h->m, n = h->n;
  const bool resume = h->resume;
  init_grid_state(h, st);
  SolveCtl hc;
  cudaMemcpyAsync(&hc, h->ctl, sizeof(hc), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  hc.mode = abip::MODE_SOLVE;
  hc.tau = hc.kappa = hc.theta = 1.0;
  hc.mu = h->prm.beta;
  if (resume) {
    const std::vector<double>& rs = h->resume_state;
    hc.tau = rs[m + n]; hc.theta = rs[m + n + 1]; hc.kappa = rs[m + 2 * n + 2]; hc.mu = rs[m + 2 * n + 3];
    h->resume = false;
  }
  hc.admm_iters = 0; hc.cg_iters = 0; hc.outer_iters = 0; hc.status = 0; hc.err = 0; hc.refreshes = 0;
  hc.max_admm = h->prm.max_admm_iters;
  // ABIP_PROFILE=1: phase timers of CTA 0, printed to stderr after the solve
  const char* prof_env = std::getenv("ABIP_PROFILE");
  unsigned long long* prof = nullptr;
  if (prof_env && prof_env[0] == '1') {
    if (cudaMalloc(&prof, abip::kProfBuckets * sizeof(unsigned long long)) == cudaSuccess)
      cudaMemsetAsync(prof, 0, abip::kProfBuckets * sizeof(unsigned long long), st);
    else { cudaGetLastError(); prof = nullptr; }
  }
  hc.prof = prof;
  unsigned long long* bar = h->mixed ? h->gdd.bar : h->gd64.bar;
  cudaMemcpyAsync(h->ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(bar, 0, sizeof(unsigned long long), st);
  cudaEventRecord(h->ev0, st);
  cudaError_t e = launch_persistent(h, st);
  if (e != cudaSuccess) return fail(h, ABIP_E_CUDA, std::string("solve launch: ") + cudaGetErrorString(e));
  cudaEventRecord(h->ev1, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(h, ABIP_E_CUDA, std::string("solve kernel: ") + cudaGetErrorString(e));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->kernel_s = ms * 1e-3;
  h->launches = (resume ? 0 : 3) + (h->mixed ? 4 : 3) + 1;   // fills and the persistent solve kernel
  if (prof) {
    unsigned long long pv[abip::kProfBuckets];
    cudaMemcpy(pv, prof, sizeof(pv), cudaMemcpyDeviceToHost);
    cudaFree(prof);
    const char* names[abip::kProfBuckets] = {"pcg_init", "cg_AT", "cg_A", "cg_upd", "zx", "upd", "res",
                                             "warm", "barrier", "totals", "setup"};
    std::fprintf(stderr, "[abip profile] kernel %.3f ms:", ms);
    for (int b = 0; b < abip::kProfBuckets; ++b) std::fprintf(stderr, " %s=%.3f", names[b], pv[b] * 1e-6);
    std::fprintf(stderr, " (ms, CTA 0)\n");
    unsigned long long* none = nullptr;
    cudaMemcpy(&h->ctl->prof, &none, sizeof(none), cudaMemcpyHostToDevice);
  }
  return ABIP_OK;
}

// ---------------------------------------------------------------------------
// dense CTA path (single instance and batches)
// ---------------------------------------------------------------------------

struct DenseHostInst {
  int m, n;
  std::vector<double> A, b, c;   // A row-major m x n
};

constexpr size_t kDenseSmemLimit = 200 * 1024;

// shared memory of the dense solve: 5m + 3n elements; the mixed path also needs the
// FP64 size because an instance may finish in FP64 after escalation
size_t dense_solve_smem(int m, int n, bool mixed = false) {
  // FP64: y, zy, w, Ax, As (m) and x, s, zx (n) doubles.  Mixed (FP64 state, FP32
  // changes): y, Ax, As, zy, q_prev (m) and x, s, A^T y, A^T zy (n) doubles, plus
  // dy, dq, dz (m, padded to 4) and dx, ds (n, padded to 4) floats, 16-byte aligned.
  if (mixed) {
    const size_t mp = (m + 3) / 4 * 4, np = (n + 3) / 4 * 4;
    return (size_t)(5 * m + 4 * n + 2) * sizeof(double) + (3 * mp + 2 * np) * sizeof(float);
  }
  return (size_t)(5 * m + 3 * n) * sizeof(double);
}
size_t dense_setup_smem(int m, int n) {
  return std::max((size_t)(2 * 32 * 33), (size_t)(2 * m + n)) * sizeof(double);
}

// Allocate and fill the device descriptors of a set of dense instances.
int dense_alloc(abip_handle* h, const std::vector<DenseHostInst>& hi, void** arena_out, DenseInst** dinst,
                int** queue, std::vector<DenseInst>& hdesc, bool mixed = false, bool bb = false) {
  const int count = (int)hi.size();
  auto layout = [&](Arena& ar, std::vector<DenseInst>& d) {
    DenseInst* di = ar.take<DenseInst>(count);
    int* q = ar.take<int>(2);
    if (ar.base) { *dinst = di; *queue = q; }
    d.assign(count, DenseInst{});
    for (int k = 0; k < count; ++k) {
      const int m = hi[k].m, n = hi[k].n;
      DenseInst& I = d[k];
      I.m = m; I.n = n; I.ld = n;
      I.A = ar.take<double>((size_t)m * n);
      I.b = ar.take<double>(m); I.c = ar.take<double>(n);
      I.L = ar.take<double>((size_t)m * m);
      I.bbar = ar.take<double>(m); I.cbar = ar.take<double>(n);
      I.g1 = ar.take<double>(m + n); I.g2 = ar.take<double>(m + n);
      I.y = ar.take<double>(m); I.x = ar.take<double>(n); I.s = ar.take<double>(n);
      I.out_y = ar.take<double>(m); I.out_x = ar.take<double>(n); I.out_s = ar.take<double>(n);
      I.work = bb ? ar.take<double>(abip::bb_work_doubles(m, n)) : nullptr;
      I.ldf = (n + 3) / 4 * 4;
      I.ldtf = (m + 3) / 4 * 4;
      if (mixed) {
        I.Af = ar.take<float>((size_t)m * I.ldf);
        I.ATf = ar.take<float>((size_t)n * I.ldtf);
        I.Ginvf = ar.take<float>((size_t)m * I.ldtf);
      } else {
        I.Af = nullptr; I.ATf = nullptr; I.Ginvf = nullptr;
      }
    }
  };
  Arena probe;
  std::vector<DenseInst> tmp;
  layout(probe, tmp);
  void* mem = nullptr;
  if (cudaMalloc(&mem, probe.off) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, ABIP_E_OOM, "device allocation of " + std::to_string(probe.off) + " bytes failed");
  }
  Arena ar;
  ar.base = static_cast<char*>(mem);
  layout(ar, hdesc);
  cudaMemset(mem, 0, probe.off);
  for (int k = 0; k < count; ++k) {
    const DenseInst& I = hdesc[k];
    cudaMemcpy((void*)I.A, hi[k].A.data(), hi[k].A.size() * 8, cudaMemcpyHostToDevice);
    cudaMemcpy((void*)I.b, hi[k].b.data(), hi[k].m * 8, cudaMemcpyHostToDevice);
    cudaMemcpy((void*)I.c, hi[k].c.data(), hi[k].n * 8, cudaMemcpyHostToDevice);
    if (mixed) {   // padded FP32 copies of A and A^T (padding stays 0 from the memset)
      const int m = hi[k].m, n = hi[k].n;
      std::vector<float> f((size_t)m * I.ldf, 0.f), ft((size_t)n * I.ldtf, 0.f);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
          const float v = (float)hi[k].A[(size_t)i * n + j];
          f[(size_t)i * I.ldf + j] = v;
          ft[(size_t)j * I.ldtf + i] = v;
        }
      cudaMemcpy((void*)I.Af, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
      cudaMemcpy((void*)I.ATf, ft.data(), ft.size() * 4, cudaMemcpyHostToDevice);
    }
  }
  cudaMemcpy(*dinst, hdesc.data(), sizeof(DenseInst) * count, cudaMemcpyHostToDevice);
  *arena_out = mem;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, ABIP_E_CUDA, std::string("dense copies: ") + cudaGetErrorString(e));
  return ABIP_OK;
}

int dense_run_setup(abip_handle* h, DenseInst* dinst, int* queue, int count, int grid, size_t smem, cudaStream_t st) {
  cudaMemsetAsync(queue, 0, 8, st);
  cudaError_t e = abip::launch_dense_setup(dinst, count, queue, grid, smem, st);
  if (e != cudaSuccess) return fail(h, ABIP_E_CUDA, std::string("dense setup launch: ") + cudaGetErrorString(e));
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(h, ABIP_E_CUDA, std::string("dense setup: ") + cudaGetErrorString(e));
  return ABIP_OK;
}

DenseParams dense_params(const abip_params& p) {
  return DenseParams{p.beta, p.gamma, p.alpha, p.eps, p.max_admm_iters, p.warmstart, p.stop_rule,
                     p.precision != ABIP_PREC_F64 ? 1 : 0, std::max(1, p.check_every), p.bb_beta ? 1 : 0,
                     p.bb_max_redo, p.eps_cor, p.eps_penalty, p.gamma_max};
}

int dense_run_solve(abip_handle* h, DenseInst* dinst, int* queue, int count, int grid, size_t smem,
                    const DenseParams& dp, cudaStream_t st, const int* order = nullptr, int variant = 0) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaMemsetAsync(queue, 0, 8, st);
  cudaEventRecord(e0, st);
  cudaError_t e = abip::launch_dense_solve(dinst, count, dp, queue, order, grid, smem, variant, st);
  cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(h, ABIP_E_CUDA, std::string("dense solve: ") + cudaGetErrorString(e));
  h->kernel_s = ms * 1e-3;
  h->launches = 1;
  return ABIP_OK;
}

// ---------------------------------------------------------------------------
// Batch autotuner: the occupancy variant of the dense solve kernel, chosen by timing a
// short capped run of the batch itself, cached per (GPU, precision, batch shape)
// ---------------------------------------------------------------------------
struct TuneCache {
  std::mutex mu;
  bool loaded = false;
  std::map<std::string, int> best;
};

TuneCache& tune_cache() {
  static TuneCache c;
  return c;
}

std::string tune_key(int device, bool mixed, const std::vector<DenseHostInst>& hi) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    std::strcpy(prop.name, "unknown");
  }
  double mn = 0.0;
  int mmax = 0;
  for (const DenseHostInst& x : hi) {
    mn += (double)x.m * x.n;
    mmax = std::max(mmax, x.m);
  }
  char buf[384];
  std::snprintf(buf, sizeof buf, "%s|%s|count=%d|mmax=%d|mn=%.1e", prop.name, mixed ? "mixed" : "f64",
                (int)hi.size(), mmax, mn);
  std::string k(buf);
  for (char& ch : k)
    if (ch == '"' || ch == ':' || ch == '\\') ch = '_';
  return k;
}

// the file the environment names in ABIP_TUNE_CACHE: one JSON object {"key": variant, ...}
void tune_load(TuneCache& c) {
  c.loaded = true;
  const char* path = std::getenv("ABIP_TUNE_CACHE");
  if (!path || !path[0]) return;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t q0 = line.find('"'), q1 = line.find('"', q0 + 1), colon = line.rfind(':');
    if (q0 == std::string::npos || q1 == std::string::npos || colon == std::string::npos || colon < q1) continue;
    c.best[line.substr(q0 + 1, q1 - q0 - 1)] = std::atoi(line.c_str() + colon + 1);
  }
}

void tune_store(const TuneCache& c) {
  const char* path = std::getenv("ABIP_TUNE_CACHE");
  if (!path || !path[0]) return;
  std::ofstream f(path);
  f << "{\n";
  size_t k = 0;
  for (const auto& kv : c.best) f << "  \"" << kv.first << "\": " << kv.second << (++k < c.best.size() ? ",\n" : "\n");
  f << "}\n";
}

int read_matrix_dense(abip_handle* h, const abip_matrix* A, std::vector<double>& out) {
  const int m = A->m, n = A->n;
  out.assign((size_t)m * n, 0.0);
  const bool dev = A->on_device != 0;
  if (A->fmt == ABIP_DENSE_ROWMAJOR) {
    if (A->ld < n) return fail(h, ABIP_E_DIM, "ld < n");
    const size_t tot = (size_t)(m - 1) * A->ld + n;
    if (A->dtype == ABIP_F64) {
      std::vector<double> raw;
      if (fetch((const double*)A->val, tot, dev, raw) != cudaSuccess) return fail(h, ABIP_E_CUDA, "reading A");
      for (int i = 0; i < m; ++i) std::memcpy(&out[(size_t)i * n], &raw[(size_t)i * A->ld], n * 8);
    } else {
      std::vector<float> raw;
      if (fetch((const float*)A->val, tot, dev, raw) != cudaSuccess) return fail(h, ABIP_E_CUDA, "reading A");
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) out[(size_t)i * n + j] = raw[(size_t)i * A->ld + j];
    }
  } else {
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    if (fetch(A->row_ptr, m + 1, dev, rp) != cudaSuccess) return fail(h, ABIP_E_CUDA, "reading row_ptr");
    const int64_t nnz = rp[m];
    if (fetch(A->col_idx, nnz, dev, ci) != cudaSuccess) return fail(h, ABIP_E_CUDA, "reading col_idx");
    std::vector<double> v(nnz);
    if (A->dtype == ABIP_F64) {
      if (fetch((const double*)A->val, nnz, dev, v) != cudaSuccess) return fail(h, ABIP_E_CUDA, "reading val");
    } else {
      std::vector<float> f;
      if (fetch((const float*)A->val, nnz, dev, f) != cudaSuccess) return fail(h, ABIP_E_CUDA, "reading val");
      for (int64_t k = 0; k < nnz; ++k) v[k] = f[k];
    }
    for (int i = 0; i < m; ++i)
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) out[(size_t)i * n + ci[k]] += v[k];
  }
  if (!finite_all(out.data(), out.size())) return fail(h, ABIP_E_INVALID_ARG, "A has non-finite entries");
  return ABIP_OK;
}

int read_matrix_csr(abip_handle* h, const abip_matrix* A, HostCSR& out, bool& f32) {
  const int m = A->m, n = A->n;
  const bool dev = A->on_device != 0;
  out.m = m;
  out.n = n;
  f32 = A->dtype == ABIP_F32;
  if (A->fmt == ABIP_CSR) {
    if (!A->row_ptr || !A->col_idx || (!A->val && A->nnz > 0)) return fail(h, ABIP_E_INVALID_ARG, "null CSR array");
    if (fetch(A->row_ptr, m + 1, dev, out.rp) != cudaSuccess) return fail(h, ABIP_E_CUDA, "reading row_ptr");
    if (out.rp[0] != 0 || out.rp[m] != A->nnz) return fail(h, ABIP_E_DIM, "row_ptr[0] != 0 or row_ptr[m] != nnz");
    for (int i = 0; i < m; ++i)
      if (out.rp[i + 1] < out.rp[i]) return fail(h, ABIP_E_DIM, "row_ptr not monotone");
    const int64_t nnz = A->nnz;
    if (fetch(A->col_idx, nnz, dev, out.ci) != cudaSuccess) return fail(h, ABIP_E_CUDA, "reading col_idx");
    for (int64_t k = 0; k < nnz; ++k)
      if (out.ci[k] < 0 || out.ci[k] >= n) return fail(h, ABIP_E_DIM, "column index out of range");
    if (A->dtype == ABIP_F64) {
      if (fetch((const double*)A->val, nnz, dev, out.v) != cudaSuccess) return fail(h, ABIP_E_CUDA, "reading val");
    } else {
      std::vector<float> f;
      if (fetch((const float*)A->val, nnz, dev, f) != cudaSuccess) return fail(h, ABIP_E_CUDA, "reading val");
      out.v.assign(f.begin(), f.end());
    }
    if (!finite_all(out.v.data(), out.v.size())) return fail(h, ABIP_E_INVALID_ARG, "A has non-finite entries");
  } else {
    std::vector<double> d;
    int rc = read_matrix_dense(h, A, d);
    if (rc) return rc;
    out.rp.assign(m + 1, 0);
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < n; ++j)
        if (d[(size_t)i * n + j] != 0.0) {
          out.ci.push_back(j);
          out.v.push_back(d[(size_t)i * n + j]);
        }
      out.rp[i + 1] = (int64_t)out.ci.size();
    }
  }
  return ABIP_OK;
}

int validate_matrix(abip_handle* h, const abip_matrix* A) {
  if (!A) return fail(h, ABIP_E_INVALID_ARG, "A is NULL");
  if (A->m < 1 || A->n < A->m) return fail(h, ABIP_E_DIM, "need 1 <= m <= n");
  if (A->fmt != ABIP_DENSE_ROWMAJOR && A->fmt != ABIP_CSR) return fail(h, ABIP_E_INVALID_ARG, "unknown matrix format");
  if (A->dtype != ABIP_F32 && A->dtype != ABIP_F64) return fail(h, ABIP_E_INVALID_ARG, "unknown dtype");
  if (A->fmt == ABIP_DENSE_ROWMAJOR && !A->val) return fail(h, ABIP_E_INVALID_ARG, "A.val is NULL");
  if (A->fmt == ABIP_CSR && A->nnz < 0) return fail(h, ABIP_E_DIM, "nnz < 0");
  return ABIP_OK;
}

// ---------------------------------------------------------------------------
// Differentiation at the central point: host staging shared by the single-handle and
// batch entry points.  Each item carries its data on the host (A only when not already
// on the device), the raw final iterate and the caller's output pointers.
// ---------------------------------------------------------------------------
constexpr int kNewtonMax = 40;
constexpr double kNewtonTol = 1e-15;   // relative to 1 + tau + kappa; the floor test usually ends it first

struct BwdItem {
  int m = 0, n = 0;
  int64_t ld = 0;
  const double* A_dev = nullptr;          // device A (ld) when resident, else A_host (ld = n)
  const double* b_dev = nullptr;
  const double* c_dev = nullptr;
  std::vector<double> A_host, b_host, c_host;
  std::vector<double> y, x, s, g;         // raw iterate and dL/dx*
  double tau = 0, theta = 0, kappa = 0, cmu = 0;
  double* out_dA = nullptr;
  double* out_db = nullptr;
  double* out_dc = nullptr;
};

int run_backward(abip_handle* h, std::vector<BwdItem>& items, cudaStream_t st) {
  const int count = (int)items.size();
  Arena ar;
  auto plan = [&](std::vector<BackwardInst>* hb) {
    ar.take<BackwardInst>(count);
    for (int k = 0; k < count; ++k) {
      BwdItem& it = items[k];
      const size_t m = it.m, n = it.n;
      BackwardInst q{};
      q.m = it.m; q.n = it.n; q.ld = it.ld;
      q.A = it.A_dev ? it.A_dev : ar.take<double>(m * n);
      q.b = it.b_dev ? it.b_dev : ar.take<double>(m);
      q.c = it.c_dev ? it.c_dev : ar.take<double>(n);
      q.y = ar.take<double>(m); q.x = ar.take<double>(n); q.s = ar.take<double>(n);
      q.dl_dx = ar.take<double>(n);
      q.dA = it.out_dA ? ar.take<double>(m * n) : nullptr;
      q.db = it.out_db ? ar.take<double>(m) : nullptr;
      q.dc = it.out_dc ? ar.take<double>(n) : nullptr;
      q.K = ar.take<double>((m + n + 2) * (m + n + 2));
      q.work = ar.take<double>(abip::backward_work_doubles(it.m, it.n));
      q.tau = it.tau; q.theta = it.theta; q.kappa = it.kappa; q.cmu = it.cmu;
      q.newton_max = kNewtonMax;
      q.newton_tol = kNewtonTol;
      if (hb) (*hb)[k] = q;
    }
  };
  plan(nullptr);
  const size_t bytes = ar.off;
  void* arena = nullptr;
  if (cudaMalloc(&arena, bytes) != cudaSuccess) return fail(h, ABIP_E_OOM, "backward scratch: " + std::to_string(bytes) + " bytes");
  ar.off = 0;
  ar.base = static_cast<char*>(arena);
  BackwardInst* dinsts = reinterpret_cast<BackwardInst*>(arena);   // first block of the plan
  std::vector<BackwardInst> hb(count);
  plan(&hb);
  int rc = ABIP_OK;
  auto up = [&](const double* dst, const std::vector<double>& v) {
    if (rc == ABIP_OK && !v.empty() &&
        cudaMemcpyAsync(const_cast<double*>(dst), v.data(), v.size() * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
      rc = fail(h, ABIP_E_CUDA, "backward upload");
  };
  for (int k = 0; k < count; ++k) {
    BwdItem& it = items[k];
    if (!it.A_dev) up(hb[k].A, it.A_host);
    if (!it.b_dev) up(hb[k].b, it.b_host);
    if (!it.c_dev) up(hb[k].c, it.c_host);
    up(hb[k].y, it.y); up(hb[k].x, it.x); up(hb[k].s, it.s); up(hb[k].dl_dx, it.g);
  }
  if (rc == ABIP_OK && cudaMemcpyAsync(dinsts, hb.data(), sizeof(BackwardInst) * count, cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = fail(h, ABIP_E_CUDA, "backward descriptors");
  if (rc == ABIP_OK) {
    const int grid = std::min(count, abip::dense_max_ctas(h ? h->device : 0));
    cudaError_t e = abip::launch_dense_backward(dinsts, count, std::max(grid, 1), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = fail(h, ABIP_E_CUDA, std::string("backward kernel: ") + cudaGetErrorString(e));
    if (h) h->launches = 1;
  }
  std::vector<BackwardInst> res(count);
  if (rc == ABIP_OK && cudaMemcpy(res.data(), dinsts, sizeof(BackwardInst) * count, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = fail(h, ABIP_E_CUDA, "backward results");
  for (int k = 0; k < count && rc == ABIP_OK; ++k) {
    if (res[k].err) {
      rc = fail(h, ABIP_E_NUMERICAL, "instance " + std::to_string(k) + ": the KKT matrix at the central point is singular");
      break;
    }
    const BwdItem& it = items[k];
    const size_t m = it.m, n = it.n;
    auto down = [&](double* dst, const double* src, size_t len) {
      if (rc == ABIP_OK && dst && cudaMemcpy(dst, src, len * 8, cudaMemcpyDefault) != cudaSuccess)
        rc = fail(h, ABIP_E_CUDA, "backward output copy");
    };
    down(it.out_dA, res[k].dA, m * n);
    down(it.out_db, res[k].db, m);
    down(it.out_dc, res[k].dc, n);
  }
  cudaFree(arena);
  return rc;
}

}  // namespace

namespace abip {
int check_params_internal(const abip_params& p, std::string& why) { return check_params(p, why); }
int noalloc_fail(int code, const std::string& msg) { return fail(nullptr, code, msg); }
}  // namespace abip

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

int abip_default_params(abip_params* p) {
  if (!p) return ABIP_E_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->beta = 1.0;
  p->gamma = 0.1;
  p->alpha = 1.8;
  p->eps = 1e-6;
  p->max_admm_iters = 1000000;
  p->linsys = -1;   // automatic
  p->cg_tol = 1e-10;
  p->cg_rel = 0.0;
  p->cg_warm = 2;
  p->cg_max_iter = 1000;
  p->precision = ABIP_PREC_F64;
  p->warmstart = 0;
  p->stop_rule = 0;
  p->check_every = 1;
  p->grid_ctas = 0;
  p->bb_beta = 0;
  p->bb_max_redo = 5;
  p->eps_cor = 0.2;
  p->eps_penalty = 0.1;
  p->autotune = 0;
  p->batch_order = 1;
  return ABIP_OK;
}

int abip_setup(const abip_matrix* A, const double* b, const double* c, const abip_params* p, abip_handle** out) {
  const double t0 = now_s();
  if (!out) return fail(nullptr, ABIP_E_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate_matrix(nullptr, A);
  if (rc) return rc;
  if (!b || !c) return fail(nullptr, ABIP_E_INVALID_ARG, "b or c is NULL");
  abip_params prm;
  if (p) prm = *p;
  else abip_default_params(&prm);
  std::string why;
  if (!check_params(prm, why)) return fail(nullptr, ABIP_E_INVALID_ARG, why);
  abip_handle* h = new abip_handle();
  cudaGetDevice(&h->device);
  h->m = A->m;
  h->n = A->n;
  h->prm = prm;
  const int m = A->m, n = A->n;
  std::vector<double> hb, hc;
  const bool dev = A->on_device != 0;
  if (fetch(b, m, dev, hb) != cudaSuccess || fetch(c, n, dev, hc) != cudaSuccess) {
    rc = fail(h, ABIP_E_CUDA, "reading b, c");
    g_err = h->err; delete h; return rc;
  }
  if (!finite_all(hb.data(), m) || !finite_all(hc.data(), n)) {
    g_err = "b or c has non-finite entries"; delete h; return ABIP_E_INVALID_ARG;
  }
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
    cudaGetLastError();
    g_err = "cudaEventCreate failed (no usable CUDA device?)";
    abip_free(h);
    return ABIP_E_CUDA;
  }
  int linsys = prm.linsys;
  if (linsys < 0) linsys = A->fmt == ABIP_CSR ? ABIP_LINSYS_PCG : ABIP_LINSYS_DENSE_CHOL;
  if (prm.bb_beta && (linsys != ABIP_LINSYS_DENSE_CHOL || prm.precision != ABIP_PREC_F64)) {
    g_err = "bb_beta needs the dense Cholesky path in FP64";
    abip_free(h);
    return ABIP_E_UNSUPPORTED;
  }
  h->prm.linsys = linsys;
  h->mixed = prm.precision != ABIP_PREC_F64;
  if (linsys == ABIP_LINSYS_PCG || linsys == ABIP_LINSYS_SPARSE_LDL) {
    h->path = 0;
    HostCSR hA;
    bool f32 = false;
    rc = read_matrix_csr(h, A, hA, f32);
    if (rc == ABIP_OK && linsys == ABIP_LINSYS_SPARSE_LDL) {
      abip::ldl_host::Symbolic sym;
      std::string why;
      if (!abip::ldl_host::analyze(hA, sym, why)) {
        rc = fail(h, ABIP_E_UNSUPPORTED, "sparse direct projection: " + why + "; use linsys = PCG");
      } else {
        const std::vector<double> lx0 = abip::ldl_host::initial_values(hA, sym);
        rc = setup_grid_path(h, h->gd64, hA, hb, hc, !f32, abip::grid_solver_max_ctas(!f32, h->device), &sym, &lx0);
      }
    } else if (rc == ABIP_OK) {
      if (h->mixed)   // FP32 values: exact for float input, rounded for double input (FP64 refreshes see them)
        rc = setup_grid_path(h, h->gdd, hA, hb, hc, false, abip::grid_delta_max_ctas(h->device));
      else
        rc = setup_grid_path(h, h->gd64, hA, hb, hc, !f32, abip::grid_solver_max_ctas(!f32, h->device));
    }
  } else {
    h->path = 1;
    if (dense_solve_smem(m, n, h->mixed) > kDenseSmemLimit)
      rc = fail(h, ABIP_E_UNSUPPORTED, "dense Cholesky path needs 40m + 24n bytes (FP64) or 48m + 40n bytes (mixed) of shared memory, at most 200 KB; use linsys = PCG");
    else {
      std::vector<DenseHostInst> hi(1);
      hi[0].m = m; hi[0].n = n; hi[0].b = hb; hi[0].c = hc;
      rc = read_matrix_dense(h, A, hi[0].A);
      std::vector<DenseInst> hd;
      if (rc == ABIP_OK) rc = dense_alloc(h, hi, &h->arena, &h->dinst, &h->queue, hd, h->mixed != 0, prm.bb_beta != 0);
      if (rc == ABIP_OK) {
        h->hinst = hd[0];
        rc = dense_run_setup(h, h->dinst, h->queue, 1, 1, dense_setup_smem(m, n), 0);
      }
      if (rc == ABIP_OK) {
        cudaMemcpy(&h->hinst, h->dinst, sizeof(DenseInst), cudaMemcpyDeviceToHost);
        if (h->hinst.err != 0) rc = fail(h, device_error_code(h->hinst.err), std::string("setup: ") + device_error_str(h->hinst.err));
      }
    }
  }
  if (rc != ABIP_OK) {
    g_err = h->err;
    abip_free(h);
    return rc;
  }
  h->setup_s = now_s() - t0;
  *out = h;
  return ABIP_OK;
}

static int copy_out(abip_handle* h, double* dst, const double* dev_src, int64_t n, cudaStream_t st) {
  if (!dst) return ABIP_OK;
  cudaError_t e = cudaMemcpyAsync(dst, dev_src, n * 8, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return fail(h, ABIP_E_CUDA, std::string("output copy: ") + cudaGetErrorString(e));
  return ABIP_OK;
}

int abip_solve(abip_handle* h, double* x, double* y, double* s, abip_info* info, void* stream) {
  if (!h) return fail(nullptr, ABIP_E_INVALID_ARG, "handle is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double t0 = now_s();
  const int m = h->m, n = h->n;
  int rc;
  abip_info inf{};
  if (h->path == 0) {
    rc = solve_grid_path(h, st);
    if (rc) return rc;
    SolveCtl hc;
    cudaMemcpy(&hc, h->ctl, sizeof(hc), cudaMemcpyDeviceToHost);
    if (hc.err != 0) return fail(h, device_error_code(hc.err), std::string("solve: ") + device_error_str(hc.err));
    inf.status = hc.status; inf.outer_iters = hc.outer_iters; inf.admm_iters = hc.admm_iters; inf.cg_iters = hc.cg_iters;
    inf.tau = hc.tau; inf.kappa = hc.kappa; inf.theta = hc.theta; inf.mu = hc.mu;
    inf.obj = hc.ctx / hc.tau; inf.pres = hc.pres; inf.dres = hc.dres; inf.dgap = hc.dgap;
    inf.beta = h->prm.beta;
    inf.fp32_iters = h->mixed ? hc.admm_iters : 0;
    double sx = 1.0 / hc.tau, sy = 1.0 / hc.tau;
    if (hc.status == ABIP_PRIMAL_INFEASIBLE) { sx = 1.0; sy = 1.0 / hc.bty; }
    if (hc.status == ABIP_DUAL_INFEASIBLE) { sx = -1.0 / hc.ctx; sy = 1.0; }
    double* stage = h->stage;
    const double* gx = h->mixed ? h->gdd.x : h->gd64.x;
    const double* gy = h->mixed ? h->gdd.y : h->gd64.y;
    const double* gs = h->mixed ? h->gdd.s : h->gd64.s;
    output_kernel<double><<<128, 256, 0, st>>>(gx, n, sx, stage);
    output_kernel<double><<<128, 256, 0, st>>>(gy, m, sy, stage + n);
    output_kernel<double><<<128, 256, 0, st>>>(gs, n, sy, stage + n + m);
    h->launches += 3;
    rc = copy_out(h, x, stage, n, st);
    if (!rc) rc = copy_out(h, y, stage + n, m, st);
    if (!rc) rc = copy_out(h, s, stage + n + m, n, st);
    cudaStreamSynchronize(st);
    if (rc) return rc;
  } else {
    if (h->resume) {
      const std::vector<double>& rs = h->resume_state;
      DenseInst I = h->hinst;
      cudaMemcpy(I.y, rs.data(), m * 8, cudaMemcpyHostToDevice);
      cudaMemcpy(I.x, rs.data() + m, n * 8, cudaMemcpyHostToDevice);
      cudaMemcpy(I.s, rs.data() + m + n + 2, n * 8, cudaMemcpyHostToDevice);
      I.resume = 1;
      I.r_tau = rs[m + n]; I.r_theta = rs[m + n + 1]; I.r_kappa = rs[m + 2 * n + 2]; I.r_mu = rs[m + 2 * n + 3];
      cudaMemcpy(h->dinst, &I, sizeof(DenseInst), cudaMemcpyHostToDevice);
      h->resume = false;
    }
    rc = dense_run_solve(h, h->dinst, h->queue, 1, 1, dense_solve_smem(m, n, h->mixed != 0), dense_params(h->prm), st);
    if (rc) return rc;
    cudaMemcpy(&h->hinst, h->dinst, sizeof(DenseInst), cudaMemcpyDeviceToHost);
    const DenseInst& I = h->hinst;
    if (I.err != 0) return fail(h, device_error_code(I.err), std::string("solve: ") + device_error_str(I.err));
    inf.status = I.status; inf.outer_iters = I.outer_iters; inf.admm_iters = I.admm_iters; inf.cg_iters = 0;
    inf.fp32_iters = h->mixed ? (((int64_t)I.fp32_iters_hi << 31) | I.fp32_iters_lo) : 0;
    if (h->mixed && !I.fp32_iters_lo && !I.fp32_iters_hi) inf.fp32_iters = I.admm_iters;
    inf.tau = I.tau; inf.kappa = I.kappa; inf.theta = I.theta; inf.mu = I.mu;
    inf.obj = I.obj; inf.pres = I.pres; inf.dres = I.dres; inf.dgap = I.dgap;
    inf.beta = I.beta_last;
    rc = copy_out(h, x, I.out_x, n, st);
    if (!rc) rc = copy_out(h, y, I.out_y, m, st);
    if (!rc) rc = copy_out(h, s, I.out_s, n, st);
    cudaStreamSynchronize(st);
    if (rc) return rc;
  }
  h->solved = true;
  h->solve_s = now_s() - t0;
  inf.setup_s = h->setup_s;
  inf.solve_s = h->solve_s;
  inf.kernel_s = h->kernel_s;
  inf.launches = h->launches;
  if (info) *info = inf;
  return ABIP_OK;
}

int abip_solve_batch(int32_t count, const abip_matrix* A, const double* const* b, const double* const* c,
                     const abip_params* p, double* const* x, double* const* y, double* const* s,
                     abip_info* infos, void* stream) {
  const double t0 = now_s();
  if (count < 0) return fail(nullptr, ABIP_E_INVALID_ARG, "count < 0");
  if (count == 0) return ABIP_OK;
  if (!A || !b || !c) return fail(nullptr, ABIP_E_INVALID_ARG, "A, b or c is NULL");
  abip_params prm;
  if (p) prm = *p;
  else abip_default_params(&prm);
  std::string why;
  if (!check_params(prm, why)) return fail(nullptr, ABIP_E_INVALID_ARG, why);
  const bool mixed = prm.precision != ABIP_PREC_F64;
  if (prm.bb_beta && mixed) return fail(nullptr, ABIP_E_UNSUPPORTED, "bb_beta needs FP64 (precision = ABIP_PREC_F64)");
  abip_handle tmp;
  cudaGetDevice(&tmp.device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<DenseHostInst> hi(count);
  size_t smem_solve = 0, smem_setup = 0;
  for (int k = 0; k < count; ++k) {
    int rc = validate_matrix(&tmp, &A[k]);
    if (rc) return fail(nullptr, rc, "instance " + std::to_string(k) + ": " + tmp.err);
    if (!b[k] || !c[k]) return fail(nullptr, ABIP_E_INVALID_ARG, "instance " + std::to_string(k) + ": b or c is NULL");
    const int m = A[k].m, n = A[k].n;
    if (dense_solve_smem(m, n, mixed) > kDenseSmemLimit)
      return fail(nullptr, ABIP_E_UNSUPPORTED, "instance " + std::to_string(k) + ": needs 40m + 24n bytes (FP64) or "
                                                  "48m + 40n bytes (mixed) of shared memory, at most 200 KB");
    hi[k].m = m; hi[k].n = n;
    rc = read_matrix_dense(&tmp, &A[k], hi[k].A);
    if (rc) return fail(nullptr, rc, "instance " + std::to_string(k) + ": " + tmp.err);
    const bool dev = A[k].on_device != 0;
    if (fetch(b[k], m, dev, hi[k].b) != cudaSuccess || fetch(c[k], n, dev, hi[k].c) != cudaSuccess)
      return fail(nullptr, ABIP_E_CUDA, "reading b, c");
    if (!finite_all(hi[k].b.data(), m) || !finite_all(hi[k].c.data(), n))
      return fail(nullptr, ABIP_E_INVALID_ARG, "instance " + std::to_string(k) + ": non-finite b or c");
    smem_solve = std::max(smem_solve, dense_solve_smem(m, n, mixed));
    smem_setup = std::max(smem_setup, dense_setup_smem(m, n));
  }
  void* arena = nullptr;
  DenseInst* dinst = nullptr;
  int* queue = nullptr;
  std::vector<DenseInst> hd;
  int rc = dense_alloc(&tmp, hi, &arena, &dinst, &queue, hd, mixed, prm.bb_beta != 0);
  if (rc) return fail(nullptr, rc, tmp.err);
  // hand-out order: largest first (the batch's wall time is its slowest instance)
  int* order = nullptr;
  if (prm.batch_order == 1 && count > 1) {
    std::vector<int> ord(count);
    for (int k = 0; k < count; ++k) ord[k] = k;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      const double ca = (double)hi[a].m * hi[a].n + (double)hi[a].m * hi[a].m;
      const double cb = (double)hi[b].m * hi[b].n + (double)hi[b].m * hi[b].m;
      return ca > cb;
    });
    if (cudaMalloc(&order, count * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(arena);
      return fail(nullptr, ABIP_E_OOM, "batch order: device allocation failed");
    }
    cudaMemcpy(order, ord.data(), count * sizeof(int), cudaMemcpyHostToDevice);
  }
  const int sms = abip::dense_max_ctas(tmp.device);
  const DenseParams dp = dense_params(prm);
  rc = dense_run_setup(&tmp, dinst, queue, count, std::min(count, sms * 4), smem_setup, st);
  // occupancy variant: 0, or the autotuner's (cached, or timed on this batch)
  int variant = 0, tuned = 0;
  if (!rc && prm.autotune) {
    TuneCache& tc = tune_cache();
    const std::string key = tune_key(tmp.device, mixed, hi);
    {
      std::lock_guard<std::mutex> lock(tc.mu);
      if (!tc.loaded) tune_load(tc);
      auto it = tc.best.find(key);
      if (it != tc.best.end() && it->second >= 0 && it->second < abip::kDenseVariants) { variant = it->second; tuned = 2; }
    }
    if (!tuned) {
      DenseParams probe = dp;   // 30 updates of every instance, no test can stop them
      probe.max_admm = 30;
      probe.eps = 0.0;
      probe.bb = 0;
      double best_s = 1e300;
      for (int v = 0; v < abip::kDenseVariants && !rc; ++v) {
        const int per_v = abip::dense_solve_ctas_per_sm(mixed, smem_solve, v);
        if (per_v < 1) continue;
        rc = dense_run_solve(&tmp, dinst, queue, count, std::min(count, sms * per_v), smem_solve, probe, st, order, v);
        if (!rc && tmp.kernel_s < best_s) { best_s = tmp.kernel_s; variant = v; }
      }
      tuned = 1;
      std::lock_guard<std::mutex> lock(tc.mu);
      tc.best[key] = variant;
      tune_store(tc);
    }
  }
  const int per = std::max(1, abip::dense_solve_ctas_per_sm(mixed, smem_solve, variant));
  const int grid = std::min(count, sms * per);
  if (!rc) rc = dense_run_solve(&tmp, dinst, queue, count, grid, smem_solve, dp, st, order, variant);
  if (!rc) {
    std::vector<DenseInst> res(count);
    cudaMemcpy(res.data(), dinst, sizeof(DenseInst) * count, cudaMemcpyDeviceToHost);
    const double el = now_s() - t0;
    for (int k = 0; k < count && !rc; ++k) {
      const DenseInst& I = res[k];
      if (I.err != 0) { rc = fail(nullptr, device_error_code(I.err), "instance " + std::to_string(k) + ": " + device_error_str(I.err)); break; }
      if (infos) {
        abip_info& f = infos[k];
        std::memset(&f, 0, sizeof(f));
        f.status = I.status; f.outer_iters = I.outer_iters; f.admm_iters = I.admm_iters;
        f.fp32_iters = mixed ? (((int64_t)I.fp32_iters_hi << 31) | I.fp32_iters_lo) : 0;
        if (mixed && !I.fp32_iters_lo && !I.fp32_iters_hi) f.fp32_iters = I.admm_iters;
        f.tau = I.tau; f.kappa = I.kappa; f.theta = I.theta; f.mu = I.mu;
        f.obj = I.obj; f.pres = I.pres; f.dres = I.dres; f.dgap = I.dgap;
        f.beta = I.beta_last;
        f.ctas_per_sm = per;
        f.tuned = tuned;
        f.solve_s = el;
        f.kernel_s = tmp.kernel_s;
        f.launches = tmp.launches;
      }
      if (x && x[k]) rc = copy_out(&tmp, x[k], I.out_x, I.n, st);
      if (!rc && y && y[k]) rc = copy_out(&tmp, y[k], I.out_y, I.m, st);
      if (!rc && s && s[k]) rc = copy_out(&tmp, s[k], I.out_s, I.n, st);
    }
    cudaStreamSynchronize(st);
    if (rc) g_err = tmp.err.empty() ? g_err : tmp.err;
  } else {
    g_err = tmp.err;
  }
  if (order) cudaFree(order);
  cudaFree(arena);
  return rc;
}

int abip_solve_batch_shared(int32_t count, const abip_matrix* A, const double* const* b, const double* const* c,
                            const abip_params* p, double* const* x, double* const* y, double* const* s,
                            abip_info* infos, void* stream) {
  const double t0 = now_s();
  if (count < 0) return fail(nullptr, ABIP_E_INVALID_ARG, "count < 0");
  if (count == 0) return ABIP_OK;
  if (!A || !b || !c) return fail(nullptr, ABIP_E_INVALID_ARG, "A, b or c is NULL");
  if (A->fmt != ABIP_DENSE_ROWMAJOR) return fail(nullptr, ABIP_E_UNSUPPORTED, "the shared-A batch takes a dense A");
  if (p && p->bb_beta) return fail(nullptr, ABIP_E_UNSUPPORTED, "bb_beta is not provided on the shared-A batch");
  abip_params prm;
  if (p) prm = *p;
  else abip_default_params(&prm);
  std::string why;
  if (!check_params(prm, why)) return fail(nullptr, ABIP_E_INVALID_ARG, why);
  abip_handle tmp;
  cudaGetDevice(&tmp.device);
  int rc = validate_matrix(&tmp, A);
  if (rc) return fail(nullptr, rc, tmp.err);
  const int m = A->m, n = A->n;
  std::vector<double> Ah;
  rc = read_matrix_dense(&tmp, A, Ah);
  if (rc) return fail(nullptr, rc, tmp.err);
  std::vector<std::vector<double>> hb(count), hc(count);
  for (int k = 0; k < count; ++k) {
    if (!b[k] || !c[k]) return fail(nullptr, ABIP_E_INVALID_ARG, "instance " + std::to_string(k) + ": b or c is NULL");
    if (fetch(b[k], m, is_device_ptr(b[k]), hb[k]) != cudaSuccess || fetch(c[k], n, is_device_ptr(c[k]), hc[k]) != cudaSuccess)
      return fail(nullptr, ABIP_E_CUDA, "reading b, c");
    if (!finite_all(hb[k].data(), m) || !finite_all(hc[k].data(), n))
      return fail(nullptr, ABIP_E_INVALID_ARG, "instance " + std::to_string(k) + ": non-finite b or c");
  }
  abip::ShParams sp{};
  sp.beta = prm.beta; sp.gamma = prm.gamma; sp.alpha = prm.alpha; sp.eps = prm.eps;
  sp.gamma_max = prm.gamma_max;
  sp.max_admm = prm.max_admm_iters; sp.warmstart = prm.warmstart; sp.stop_rule = prm.stop_rule;
  sp.mixed = prm.precision != ABIP_PREC_F64 ? 1 : 0;
  sp.tc = 0;
  if (prm.precision == ABIP_PREC_MIXED_BF16) {
    // the tensor-core products take A as bfloat16 terms: one when A is exact in bfloat16,
    // three otherwise (they hold A's FP32 value exactly); A must lie in the FP32 range
    sp.tc = 1;
    for (const double v : Ah) {
      const float f = (float)v;
      if (!std::isfinite(f))
        return fail(nullptr, ABIP_E_INVALID_ARG, "ABIP_PREC_MIXED_BF16 needs A within the FP32 range");
      uint32_t u;
      std::memcpy(&u, &f, 4);
      if ((double)f != v || (u & 0xFFFFu) != 0) sp.tc = 3;
    }
  }
  sp.n = n;
  sp.confirm_gap = std::max<int64_t>(prm.check_every, 20);
  sp.refresh = 192;   // a multiple of the 16-cycle groups of the shared-A solve loop
  for (int k0 = 0; k0 < count; k0 += 64) {
    const int cnt = std::min(64, count - k0);
    std::vector<const double*> bp(cnt), cp(cnt);
    for (int k = 0; k < cnt; ++k) { bp[k] = hb[k0 + k].data(); cp[k] = hc[k0 + k].data(); }
    abip::SharedBatchArgs args{m, n, cnt, Ah.data(), bp.data(), cp.data(), sp, static_cast<cudaStream_t>(stream)};
    std::vector<abip::SharedBatchResult> res;
    std::string err;
    rc = abip::shared_batch_run(args, res, err);
    if (rc) return fail(nullptr, rc, err);
    const double el = now_s() - t0;
    for (int k = 0; k < cnt; ++k) {
      const abip::ShInst& I = res[k].inst;
      const int id = k0 + k;
      if (infos) {
        abip_info& f = infos[id];
        std::memset(&f, 0, sizeof(f));
        f.status = I.status; f.outer_iters = I.outer; f.admm_iters = I.total;
        f.fp32_iters = sp.mixed ? I.total : 0;
        f.tau = I.tau; f.kappa = I.kappa; f.theta = I.theta; f.mu = I.mu;
        f.obj = I.ctx / I.tau; f.pres = I.pres; f.dres = I.dres; f.dgap = I.dgap;
        f.beta = prm.beta;
        f.setup_s = res[k].setup_s; f.solve_s = el; f.kernel_s = res[k].kernel_s; f.launches = res[k].launches;
      }
      auto put = [&](double* dst, const std::vector<double>& v) {
        if (rc == ABIP_OK && dst && cudaMemcpy(dst, v.data(), v.size() * 8, cudaMemcpyDefault) != cudaSuccess)
          rc = fail(nullptr, ABIP_E_CUDA, "output copy");
      };
      if (x) put(x[id], res[k].x);
      if (y) put(y[id], res[k].y);
      if (s) put(s[id], res[k].s);
    }
    if (rc) return rc;
  }
  return ABIP_OK;
}

int abip_backward(abip_handle* h, const double* dl_dx, double* dl_dc, double* dl_db, double* dl_dA) {
  if (!h || !dl_dx) return fail(h, ABIP_E_INVALID_ARG, "NULL argument");
  if (!h->solved) return fail(h, ABIP_E_NOT_SOLVED, "no solve has run on this handle");
  if (h->path != 1)
    return fail(h, ABIP_E_UNSUPPORTED, "abip_backward needs a dense handle (linsys = dense): the adjoint factors the dense reduced KKT matrix of order m + n + 2");
  const DenseInst& I = h->hinst;
  if (I.status != ABIP_OPTIMAL && I.status != ABIP_MAX_ITER)
    return fail(h, ABIP_E_INVALID_ARG, std::string("no gradient at a ") + abip_status_str(I.status) + " result (needs tau > 0)");
  const int m = h->m, n = h->n;
  std::vector<BwdItem> items(1);
  BwdItem& it = items[0];
  it.m = m; it.n = n; it.ld = I.ld;
  it.A_dev = I.A; it.b_dev = I.b; it.c_dev = I.c;
  if (fetch(I.y, m, true, it.y) != cudaSuccess || fetch(I.x, n, true, it.x) != cudaSuccess ||
      fetch(I.s, n, true, it.s) != cudaSuccess || fetch(dl_dx, n, is_device_ptr(dl_dx), it.g) != cudaSuccess)
    return fail(h, ABIP_E_CUDA, "reading the state or dl_dx");
  if (!finite_all(it.g.data(), n)) return fail(h, ABIP_E_INVALID_ARG, "dl_dx has non-finite entries");
  it.tau = I.tau; it.theta = I.theta; it.kappa = I.kappa; it.cmu = I.mu / (h->prm.bb_beta ? I.beta_last : h->prm.beta);
  it.out_dA = dl_dA; it.out_db = dl_db; it.out_dc = dl_dc;
  return run_backward(h, items, nullptr);
}

int abip_backward_batch(int32_t count, const abip_matrix* A, const double* const* b, const double* const* c,
                        const abip_params* p, const double* const* x, const double* const* y,
                        const double* const* s, const abip_info* infos, const double* const* dl_dx,
                        double* const* dl_dc, double* const* dl_db, double* const* dl_dA, void* stream) {
  if (count < 0) return fail(nullptr, ABIP_E_INVALID_ARG, "count < 0");
  if (count == 0) return ABIP_OK;
  if (!A || !b || !c || !x || !y || !s || !infos || !dl_dx)
    return fail(nullptr, ABIP_E_INVALID_ARG, "A, b, c, x, y, s, infos or dl_dx is NULL");
  abip_params prm;
  if (p) prm = *p;
  else abip_default_params(&prm);
  std::string why;
  if (!check_params(prm, why)) return fail(nullptr, ABIP_E_INVALID_ARG, why);
  abip_handle tmp;
  cudaGetDevice(&tmp.device);
  std::vector<BwdItem> items(count);
  for (int k = 0; k < count; ++k) {
    const std::string at = "instance " + std::to_string(k) + ": ";
    int rc = validate_matrix(&tmp, &A[k]);
    if (rc) return fail(nullptr, rc, at + tmp.err);
    if (!b[k] || !c[k] || !x[k] || !y[k] || !s[k] || !dl_dx[k]) return fail(nullptr, ABIP_E_INVALID_ARG, at + "NULL vector");
    const abip_info& f = infos[k];
    if (f.status != ABIP_OPTIMAL && f.status != ABIP_MAX_ITER)
      return fail(nullptr, ABIP_E_INVALID_ARG, at + "no gradient at a " + abip_status_str(f.status) + " result (needs tau > 0)");
    if (!(f.tau > 0) || !(f.kappa > 0) || !(f.mu > 0)) return fail(nullptr, ABIP_E_INVALID_ARG, at + "tau, kappa and mu must be > 0");
    BwdItem& it = items[k];
    const int m = A[k].m, n = A[k].n;
    it.m = m; it.n = n; it.ld = n;
    rc = read_matrix_dense(&tmp, &A[k], it.A_host);
    if (rc) return fail(nullptr, rc, at + tmp.err);
    if (fetch(b[k], m, is_device_ptr(b[k]), it.b_host) != cudaSuccess ||
        fetch(c[k], n, is_device_ptr(c[k]), it.c_host) != cudaSuccess ||
        fetch(y[k], m, is_device_ptr(y[k]), it.y) != cudaSuccess ||
        fetch(x[k], n, is_device_ptr(x[k]), it.x) != cudaSuccess ||
        fetch(s[k], n, is_device_ptr(s[k]), it.s) != cudaSuccess ||
        fetch(dl_dx[k], n, is_device_ptr(dl_dx[k]), it.g) != cudaSuccess)
      return fail(nullptr, ABIP_E_CUDA, at + "reading the inputs");
    // the solve returned (y, x, s) / tau: undo the scaling to get the raw iterate
    for (auto* v : {&it.y, &it.x, &it.s})
      for (double& e : *v) e *= f.tau;
    for (int j = 0; j < n; ++j)
      if (!(it.x[j] > 0) || !(it.s[j] > 0)) return fail(nullptr, ABIP_E_INVALID_ARG, at + "x and s must be > 0");
    if (!finite_all(it.b_host.data(), m) || !finite_all(it.c_host.data(), n) || !finite_all(it.y.data(), m) ||
        !finite_all(it.g.data(), n))
      return fail(nullptr, ABIP_E_INVALID_ARG, at + "non-finite input");
    it.tau = f.tau; it.theta = f.theta; it.kappa = f.kappa; it.cmu = f.mu / (f.beta > 0 ? f.beta : prm.beta);
    it.out_dA = dl_dA ? dl_dA[k] : nullptr;
    it.out_db = dl_db ? dl_db[k] : nullptr;
    it.out_dc = dl_dc ? dl_dc[k] : nullptr;
  }
  const int rc = run_backward(&tmp, items, static_cast<cudaStream_t>(stream));
  if (rc) g_err = tmp.err;
  return rc;
}

int64_t abip_state_size(const abip_handle* h) {
  if (!h) return 0;
  return (int64_t)h->m + 2 * (int64_t)h->n + 4;
}

int abip_get_state(const abip_handle* h, double* buf) {
  abip_handle* hm = const_cast<abip_handle*>(h);
  if (!h || !buf) return fail(hm, ABIP_E_INVALID_ARG, "NULL argument");
  if (!h->solved) return fail(hm, ABIP_E_NOT_SOLVED, "no solve has run on this handle");
  const int m = h->m, n = h->n;
  std::vector<double> out((size_t)m + 2 * n + 4);
  double tau, theta, kappa, mu;
  if (h->path == 0) {
    SolveCtl hc;
    cudaMemcpy(&hc, h->ctl, sizeof(hc), cudaMemcpyDeviceToHost);
    tau = hc.tau; theta = hc.theta; kappa = hc.kappa; mu = hc.mu;
    cudaMemcpy(out.data(), h->mixed ? h->gdd.y : h->gd64.y, m * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(out.data() + m, h->mixed ? h->gdd.x : h->gd64.x, n * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(out.data() + m + n + 2, h->mixed ? h->gdd.s : h->gd64.s, n * 8, cudaMemcpyDeviceToHost);
  } else {
    const DenseInst& I = h->hinst;
    tau = I.tau; theta = I.theta; kappa = I.kappa; mu = I.mu;
    cudaMemcpy(out.data(), I.y, m * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(out.data() + m, I.x, n * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(out.data() + m + n + 2, I.s, n * 8, cudaMemcpyDeviceToHost);
  }
  out[m + n] = tau;
  out[m + n + 1] = theta;
  out[m + 2 * n + 2] = kappa;
  out[m + 2 * n + 3] = mu;
  cudaError_t e = cudaMemcpy(buf, out.data(), out.size() * 8, is_device_ptr(buf) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
  if (e != cudaSuccess) return fail(hm, ABIP_E_CUDA, std::string("state copy: ") + cudaGetErrorString(e));
  return ABIP_OK;
}

int abip_set_state(abip_handle* h, const double* buf) {
  if (!h || !buf) return fail(h, ABIP_E_INVALID_ARG, "NULL argument");
  const int m = h->m, n = h->n;
  const size_t len = (size_t)m + 2 * (size_t)n + 4;
  std::vector<double> v(len);
  if (is_device_ptr(buf)) {
    if (cudaMemcpy(v.data(), buf, len * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(h, ABIP_E_CUDA, "reading the state");
  } else {
    std::memcpy(v.data(), buf, len * 8);
  }
  if (!finite_all(v.data(), len)) return fail(h, ABIP_E_INVALID_ARG, "state has non-finite entries");
  for (int j = 0; j < n; ++j)
    if (!(v[m + j] > 0) || !(v[m + n + 2 + j] > 0)) return fail(h, ABIP_E_INVALID_ARG, "x and s must be > 0");
  if (!(v[m + n] > 0) || !(v[m + 2 * n + 2] > 0) || !(v[m + 2 * n + 3] > 0))
    return fail(h, ABIP_E_INVALID_ARG, "tau, kappa and mu must be > 0");
  h->resume_state = std::move(v);
  h->resume = true;
  return ABIP_OK;
}

void abip_free(abip_handle* h) {
  if (!h) return;
  if (h->arena) cudaFree(h->arena);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
}

const char* abip_status_str(int32_t status) {
  switch (status) {
    case ABIP_UNSOLVED: return "unsolved";
    case ABIP_OPTIMAL: return "optimal";
    case ABIP_PRIMAL_INFEASIBLE: return "primal_infeasible";
    case ABIP_DUAL_INFEASIBLE: return "dual_infeasible";
    case ABIP_MAX_ITER: return "max_iter";
    default: return "unknown";
  }
}

const char* abip_last_error(const abip_handle* h) {
  if (h) return h->err.c_str();
  return g_err.c_str();
}

int abip_ldl_analyze(const abip_matrix* A, int32_t* perm, int64_t* col_counts, int64_t* nnz_l) {
  int rc = validate_matrix(nullptr, A);
  if (rc) return rc;
  if (A->on_device) return fail(nullptr, ABIP_E_INVALID_ARG, "abip_ldl_analyze reads host matrices only");
  HostCSR hA;
  bool f32 = false;
  rc = read_matrix_csr(nullptr, A, hA, f32);
  if (rc) return rc;
  abip::ldl_host::Symbolic sym;
  std::string why;
  if (!abip::ldl_host::analyze(hA, sym, why)) return fail(nullptr, ABIP_E_UNSUPPORTED, why);
  const int N = sym.N;
  if (perm) std::copy(sym.perm.begin(), sym.perm.end(), perm);
  if (col_counts)
    for (int p = 0; p < N; ++p) col_counts[p] = sym.Lp[p + 1] - sym.Lp[p];
  if (nnz_l) *nnz_l = sym.Lp[N];
  return ABIP_OK;
}

const char* abip_version(void) { return "abip-gb300 0.1 (sm_103a)"; }

}  // extern "C"
