#!/usr/bin/env python
"""Benchmark of the ABIP hot path on one GB300 (or N, one replica LP per GPU).

Workload: the large sparse planted LP  min c^T x, A x = b, x >= 0  with
A = [R  I_m] in CSR, m = 100000, n = 400000, R having 8 nonzeros per column at
uniform random rows with N(0,1) float32 values, and a planted optimal pair
(synthetic data, seeded).

One step = abip_setup (embedding constants, Jacobi diagonal, M^{-1} H, Schur
complement) + abip_solve running Algorithm 2 for a fixed budget of ADMM updates
(--max-admm, default 20000; every row of the hot path runs: projection by
Jacobi-PCG, A and A^T products, prox, dual update, residual and termination
reductions, mu decreases), inputs resident in HBM.

Value: ADMM updates per second, whole job (the headline metric lists LPs solved/s,
ADMM iter/s and HBM GB/s).  LPs solved to 1e-6 per second is reported beside it
and is 0 on this workload: ABIP with the paper's inner stop rule needs more than
the paper's 10^6-update cap to reach a 1e-6 gap at n = 400000 (measured: after
400000 updates the gap is 5e-4 at mu = 1e-6).  Also reported: the solve kernel's
achieved bandwidth against the measured HBM peak (roofline), an end-to-end number
through host buffers, and the FP64 CPU oracle on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl abip|reference]
Under torchrun (N > 1) every rank runs its own LP (weak scaling, no collective on
the data path; a barrier and a max over ranks around the timed region).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "sparse_planted_lp_m100000_n400000"
METRIC = "LPs solved/s to 1e-6 rel. KKT residual; ADMM iter/s; HBM GB/s vs peak"
UNIT = "ADMM iter/s"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="abip", choices=["abip", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "f64"])
    ap.add_argument("--m", type=int, default=100000, help="rows of A (default: the full workload)")
    ap.add_argument("--max-admm", type=int, default=20000, help="ADMM updates per step")
    ap.add_argument("--cg-tol", type=float, default=1e-8)
    ap.add_argument("--cg-rel", type=float, default=0.0)
    ap.add_argument("--alpha", type=float, default=1.8, help="over-relaxation (the paper's value is 1.8)")
    ap.add_argument("--gamma", type=float, default=0.1)
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="skip the LPs-solved/s legs of the other workloads")
    ap.add_argument("--svm-count", type=int, default=128, help="L1-SVM instances of the backward leg")
    ap.add_argument("--sice-d", type=int, default=128, help="dimension of the SICE leg (d column LPs)")
    ap.add_argument("--sice-cap", type=int, default=100000, help="ADMM update cap of the SICE leg")
    ap.add_argument("--svm-cap", type=int, default=2000, help="forward updates of the backward leg")
    ap.add_argument("--f64-updates", type=int, default=5000, help="ADMM updates of the FP64 arm of the sparse LP")
    ap.add_argument("--batch-count", type=int, default=256, help="LPs in the uneven-batch leg")
    ap.add_argument("--batch-cap", type=int, default=20000, help="ADMM update cap of the uneven-batch leg")
    ap.add_argument("--bp-cap", type=int, default=30000, help="ADMM update cap of the basis-pursuit leg")
    ap.add_argument("--flow-side", type=int, default=16, help="grid side of the direct-projection leg")
    ap.add_argument("--flow-cap", type=int, default=150000, help="ADMM update cap of the direct-projection leg")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)   # child process mode
    ap.add_argument("--admm-iters-hint", type=int, default=0, help=argparse.SUPPRESS)
    return ap.parse_args()


# --------------------------------------------------------------------------------------
# algorithmic bytes of the persistent solve kernel (one launch = one whole solve)
# --------------------------------------------------------------------------------------

def algorithmic_bytes(m, n, nnz, admm_iters, cg_iters, vec_bytes, val_bytes=4):
    """Minimum traffic of the ADMM iteration on a CSR A (one pass over a CSR matrix reads
    its values, column indices and row offsets: nnz (p + 4) + 8 (rows + 1) bytes):
      per ADMM update:   one pass over A, one over A^T, and 20 vector passes of n elements
                         (A x of the new iterate fused with the next projection's A d; A^T y
                         by the exact recurrence of the projection);
      per PCG iteration: one pass over A, one over A^T, and 6 vector passes of m elements;
    with p the bytes of a matrix value and q (vec_bytes) those of a vector element."""
    q = vec_bytes
    MA = nnz * (val_bytes + 4) + 8 * (m + 1)
    MAT = nnz * (val_bytes + 4) + 8 * (n + 1)
    return admm_iters * (MA + MAT + 20 * n * q) + cg_iters * (MA + MAT + 6 * m * q)


# DRAM traffic of the solve kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum at two update counts: a fixed fill and a per-update part), valid
# only for the kernel sources it was measured on; None once any of them has changed.
KERNEL_SOURCES = ("paper_1805_12344_gb300/csrc/grid_delta.cu", "paper_1805_12344_gb300/csrc/sell.cuh",
                  "paper_1805_12344_gb300/csrc/abip_device.cuh", "paper_1805_12344_gb300/csrc/sell_host.h")
# DRAM bytes of one solve launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum) at
# 20 and 60 updates, caches flushed before the launch: 596.0 MB and 1585.0 MB, so
# 101.5 MB fixed + 24.72 MB per update (profiles/grid_delta_kernel_solve_sparse_m100000.md);
# valid while the sources above are the ones measured.
TRAFFIC = {"sources_sha256": "c9e17702ca9d067a39c456c66b8e70d58bde0a93626023c2521eb21554d8e93f",
           "dram_bytes_fixed": 101535488, "dram_bytes_per_update": 24724185.6}


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_per_launch(admm_updates):
    if TRAFFIC["sources_sha256"] is None or TRAFFIC["sources_sha256"] != kernel_sources_hash():
        return None
    return TRAFFIC["dram_bytes_fixed"] + TRAFFIC["dram_bytes_per_update"] * admm_updates


# --------------------------------------------------------------------------------------
# LPs solved per second on the other workloads (run once, after the timed region)
# --------------------------------------------------------------------------------------

def _solved(infos):
    """Instances that ended with a Sec. 4.1 result (optimal or a certificate) within the cap."""
    return sum(1 for i in infos if i["status"] in (1, 2, 3))


def leg_sparse_f64(abip, W, lp, args, stream):
    """The same sparse LP on the plain FP64 path (FP64 vectors and products, FP32-exact
    values), setup + a fixed number of updates, inputs from host memory."""
    prm = abip.default_params(precision=abip.ABIP_PREC_F64, max_admm_iters=args.f64_updates, cg_tol=args.cg_tol,
                              alpha=args.alpha, gamma=args.gamma)
    h = abip.abip_setup(lp.A, lp.b, lp.c, prm)
    info = abip.abip_solve(h, stream=stream)
    abip.abip_free(h)
    alg = algorithmic_bytes(lp.m, lp.n, lp.A.nnz, info["admm_iters"], info["cg_iters"], 8)
    return {"workload": WORKLOAD, "precision": "f64", "admm_updates": info["admm_iters"],
            "cg_iters": info["cg_iters"], "kernel_s": info["kernel_s"],
            "admm_iter_per_s": info["admm_iters"] / info["kernel_s"],
            "hbm_gbs_algorithmic": alg / info["kernel_s"] / 1e9}


def leg_batch_uneven(abip, W, args):
    """Uneven batch (m ~ U{16..256}, n = round(m U[2,4]), 10 % infeasible twins): the same
    LPs in one persistent launch in FP64 and in mixed precision, same cap and tolerance.
    LPs solved/s counts optimal and certified-infeasible instances over the wall time of
    abip_solve_batch (host inputs, setup included)."""
    import time as _t
    lps = W.batch_uneven(count=args.batch_count)
    out = {"workload": f"batch_uneven_{args.batch_count}_of_4096_recipe", "count": len(lps),
           "cap_admm_updates": args.batch_cap, "eps": 1e-6}
    for name, prec in (("f64", abip.ABIP_PREC_F64), ("mixed", abip.ABIP_PREC_MIXED)):
        prm = abip.default_params(precision=prec, max_admm_iters=args.batch_cap)
        t0 = _t.perf_counter()
        infos, *_ = abip.abip_solve_batch([l.A for l in lps], [l.b for l in lps], [l.c for l in lps], prm,
                                          want_solution=False)
        wall = _t.perf_counter() - t0
        solved = _solved(infos)
        out[name] = {"lps_solved": solved, "wall_s": wall, "lps_solved_per_s": solved / wall,
                     "kernel_s": infos[0]["kernel_s"],
                     "admm_iter_per_s": sum(i["admm_iters"] for i in infos) / infos[0]["kernel_s"]}
    out["mixed_over_f64_lps_per_s"] = out["mixed"]["lps_solved_per_s"] / max(out["f64"]["lps_solved_per_s"], 1e-30)
    return out


def leg_basis_pursuit(abip, W, args):
    """Basis pursuit, 64 right-hand sides sharing D (2048 x 8192 float32, A = [D, -D]),
    tensor-core products (ABIP_PREC_MIXED_BF16), to 1e-6 within the cap; LPs solved/s over
    the wall time of abip_solve_batch_shared (host inputs, setup included)."""
    import time as _t
    sb = W.basis_pursuit()
    prm = abip.default_params(precision=abip.ABIP_PREC_MIXED_BF16, max_admm_iters=args.bp_cap)
    t0 = _t.perf_counter()
    infos, *_ = abip.abip_solve_batch_shared(sb.A, sb.bs, sb.cs, prm, want_solution=False)
    wall = _t.perf_counter() - t0
    solved = _solved(infos)
    return {"workload": "basis_pursuit_2048x8192_batch64", "precision": "mixed_bf16_tensor_cores",
            "cap_admm_updates": args.bp_cap, "eps": 1e-6, "lps_solved": solved, "wall_s": wall,
            "lps_solved_per_s": solved / wall, "setup_s": infos[0]["setup_s"], "kernel_s": infos[0]["kernel_s"],
            "max_admm_updates": max(i["admm_iters"] for i in infos)}


def leg_svm_backward(abip, W, args):
    """Differentiation of 128 L1-SVM LPs (512 x 1154) solved in one launch
    (mixed precision, `--svm-cap` updates, then MAX_ITER or optimal), then the gradients of
    ||x* - x_t||^2 with respect to c, b and A at each final iterate in one
    abip_backward_batch launch (Newton polish onto the central point of the final mu, then
    the adjoint through the LU of the reduced KKT matrix); wall times of both calls."""
    import time as _t
    lps = [W.l1_svm(seed=W.seed_for(W.L1_SVM) + k) for k in range(args.svm_count)]
    prm = abip.default_params(precision=abip.ABIP_PREC_MIXED, max_admm_iters=args.svm_cap)
    As, bs, cs = [l.A for l in lps], [l.b for l in lps], [l.c for l in lps]
    t0 = _t.perf_counter()
    infos, xs, ys, ss = abip.abip_solve_batch(As, bs, cs, prm)
    fwd = _t.perf_counter() - t0
    gs = [2.0 * (x - l.meta["x_target"]) for x, l in zip(xs, lps)]
    t0 = _t.perf_counter()
    dcs, dbs, dAs = abip.abip_backward_batch(As, bs, cs, xs, ys, ss, infos, gs, prm)
    bwd = _t.perf_counter() - t0
    return {"workload": f"l1_svm_512x1154_batch{len(lps)}", "forward_cap_admm_updates": args.svm_cap,
            "forward_wall_s": fwd, "forward_kernel_s": infos[0]["kernel_s"],
            "optimal": sum(1 for i in infos if i["status"] == abip.ABIP_OPTIMAL),
            "backward_wall_s": bwd, "backward_per_instance_ms": 1e3 * bwd / len(lps),
            "gradient_entries_per_instance": int(lps[0].A.size + lps[0].A.shape[0] + lps[0].A.shape[1])}


def leg_bb_beta(abip, W, args):
    """Barzilai-Borwein beta (Sec. 4.3) against a fixed beta on 64 LPs of the uneven-batch recipe,
    dense FP64 path, same cap and tolerance: LPs solved, ADMM updates and wall time of
    abip_solve_batch."""
    import time as _t
    lps = W.batch_uneven(count=64, seed=W.seed_for(W.BATCH_UNEVEN, 500))
    out = {"workload": "batch_uneven_64_of_4096_recipe", "precision": "f64", "cap_admm_updates": args.batch_cap,
           "eps": 1e-6}
    for name, bb in (("fixed_beta", 0), ("bb_beta", 1)):
        prm = abip.default_params(max_admm_iters=args.batch_cap, bb_beta=bb)
        t0 = _t.perf_counter()
        infos, *_ = abip.abip_solve_batch([l.A for l in lps], [l.b for l in lps], [l.c for l in lps], prm,
                                          want_solution=False)
        wall = _t.perf_counter() - t0
        solved = _solved(infos)
        out[name] = {"lps_solved": solved, "wall_s": wall, "lps_solved_per_s": solved / wall,
                     "admm_updates": int(sum(i["admm_iters"] for i in infos))}
    return out


def leg_grid_flow_direct(abip, W, args):
    """The sparse direct projection (Sec. 4.4, LDL^T of the quasi-definite system) on a
    planted min-cost flow LP over a side x side grid, whose I + A A^T (a grid Laplacian)
    makes Jacobi-PCG take many iterations per projection: one solve to 1e-6 through the
    factor, and the PCG path on the same LP for a capped number of updates (the two paths
    produce the same iterates up to rounding, so time per update compares them)."""
    side = args.flow_side
    lp = W.grid_flow(side)
    s = abip.Solver(lp.A, lp.b, lp.c, linsys=abip.ABIP_LINSYS_SPARSE_LDL, max_admm_iters=args.flow_cap)
    info, *_ = s.solve()
    s.close()
    _, _, nnz_l = abip.abip_ldl_analyze(lp.A)
    out = {"workload": f"grid_flow_{side}x{side}", "m": lp.m, "n": lp.n, "nnz_l": nnz_l, "eps": 1e-6,
           "cap_admm_updates": args.flow_cap,
           "direct": {"status": abip.STATUS_NAMES.get(info["status"], "?"), "admm_updates": info["admm_iters"],
                      "setup_s": info["setup_s"], "kernel_s": info["kernel_s"],
                      "lps_solved_per_s": (1.0 / (info["setup_s"] + info["kernel_s"])) if info["status"] == 1 else 0.0,
                      "us_per_update": 1e6 * info["kernel_s"] / max(1, info["admm_iters"]),
                      "obj_rel_err": abs(info["obj"] - lp.p_star) / max(1.0, abs(lp.p_star))}}
    s = abip.Solver(lp.A, lp.b, lp.c, linsys=abip.ABIP_LINSYS_PCG, max_admm_iters=600, cg_max_iter=5000)
    info2, *_ = s.solve()
    s.close()
    out["pcg_600_updates"] = {"kernel_s": info2["kernel_s"], "us_per_update": 1e6 * info2["kernel_s"] / max(1, info2["admm_iters"]),
                              "cg_iters_per_update": info2["cg_iters"] / max(1, info2["admm_iters"])}
    out["direct_speedup_per_update"] = out["pcg_600_updates"]["us_per_update"] / max(1e-9, out["direct"]["us_per_update"])
    return out


def leg_sice(abip, W, args):
    """Sparse inverse covariance estimation (Sec. 5.2; a synthetic covariance stands in for
    the UCI data): the d column LPs in general form go through the host presolve (bounds
    rewritten, Ruiz scaling), all presolve to one matrix, are solved as shared-A batches
    (tensor cores) to 1e-6 and postsolved; LPs solved/s over the whole pipeline."""
    import time as _t
    d = args.sice_d
    S, lam = W.sice(d)
    gs = [W.sice_general_lp(S, lam, j) for j in range(d)]
    t0 = _t.perf_counter()
    Ps = [abip.Presolved(g.A, g.b, g.c, g.l, g.w) for g in gs]
    lps = [P.lp() for P in Ps]
    t_pre = _t.perf_counter() - t0
    A = lps[0][0].to_dense()
    prm = abip.default_params(precision=abip.ABIP_PREC_MIXED_BF16, max_admm_iters=args.sice_cap)
    t1 = _t.perf_counter()
    infos, xs, ys, _ = abip.abip_solve_batch_shared(A, [b for _, b, _ in lps], [c for _, _, c in lps], prm)
    t_solve = _t.perf_counter() - t1
    t2 = _t.perf_counter()
    objs = [P.postsolve(x, y)[3] for P, x, y in zip(Ps, xs, ys)]
    t_post = _t.perf_counter() - t2
    solved = _solved(infos)
    wall = t_pre + t_solve + t_post
    return {"workload": f"sice_d{d} (Sec. 5.2 LP, synthetic covariance)", "lps": d, "eps": 1e-6,
            "cap_admm_updates": args.sice_cap,
            "standard_form": [int(A.shape[0]), int(A.shape[1])], "lps_solved": solved,
            "presolve_s": t_pre, "solve_wall_s": t_solve, "postsolve_s": t_post, "lps_solved_per_s": solved / wall,
            "max_admm_updates": max(i["admm_iters"] for i in infos), "sum_l1_norms": float(sum(objs))}


def leg_random_udv(abip, W, args):
    """The paper's random dense LP (Sec. 5.1, A = U^T D V) at the first shape of its
    Table 1, (m, n) = (500, 5000), one LP on the shared-A path (its products are GEMVs over
    every SM), mixed precision, to 1e-3 and to 1e-6 (and to 1e-6 with the adaptive decrease
    ratio); wall time of the C-ABI call with host inputs, setup included.  The paper's own figure (ABIP, 10.6 s, an 8-core 2.6 GHz
    laptop, tolerance unstated, about 1e-3) is context, not a target."""
    import time as _t
    lp = W.random_udv(500, 5000)
    out = {"workload": "random_udv_500x5000 (Sec. 5.1, Table 1 shape)", "p_star": lp.p_star,
           "paper_context": {"abip_s": 10.6, "hardware": "8-core 2.6 GHz laptop", "tolerance": "unstated (~1e-3)"}}
    # the last run: the adaptive decrease ratio (gamma from 0.1 up to 0.3 as the residual falls)
    for eps, gmax in ((1e-3, 0.0), (1e-6, 0.0), (1e-6, 0.3)):
        prm = abip.default_params(precision=abip.ABIP_PREC_MIXED, eps=eps, max_admm_iters=200000, gamma_max=gmax)
        t0 = _t.perf_counter()
        infos, *_ = abip.abip_solve_batch_shared(lp.A, [lp.b], [lp.c], prm, want_solution=False)
        wall = _t.perf_counter() - t0
        f = infos[0]
        key = f"eps_{eps:g}" + (f"_gamma_max_{gmax:g}" if gmax else "")
        out[key] = {"status": f["status_name"], "admm_updates": f["admm_iters"], "wall_s": wall,
                              "lps_solved_per_s": (1.0 if f["status"] == 1 else 0.0) / wall,
                              "rel_obj_err": abs(f["obj"] - lp.p_star) / max(1.0, abs(lp.p_star))}
    return out


def aggregate_ranks(total_s, solved, admm, dist_mod=None, device="cpu"):
    """Whole-job totals over the ranks: the timed region is the slowest rank's, the work
    (LPs solved, ADMM updates) is summed.  dist_mod: torch.distributed or None (one rank)."""
    if dist_mod is None:
        return float(total_s), float(solved), float(admm)
    import torch
    t = torch.tensor([total_s, float(solved), float(admm)], dtype=torch.float64, device=device)
    tmax = t[0:1].clone()
    work = t[1:3].clone()
    dist_mod.all_reduce(tmax, op=dist_mod.ReduceOp.MAX)
    dist_mod.all_reduce(work, op=dist_mod.ReduceOp.SUM)
    return float(tmax[0]), float(work[0]), float(work[1])


# L2 sector bandwidth of this part, from ncu on a GB300 of this machine: 188 L2 slices x
# lts__t_sectors peak_sustained (3 sectors / cycle / slice) x 32 B x lts__cycles_elapsed
# per second (2.007 GHz).  The ceiling of a kernel whose working set stays in L2.
L2_PEAK_GBS = 188 * 3 * 32 * 2.007


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# --------------------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# --------------------------------------------------------------------------------------
# CPU oracle sample (child process, single-threaded BLAS)
# --------------------------------------------------------------------------------------

def cpu_sample_main(args):
    """Time the FP64 oracle on the workload: its setup plus ADMM iterations for about
    `cpu_sample_s` seconds.  Prints one JSON object."""
    import numpy as np
    from oracle import abip_oracle as O
    from paper_1805_12344_gb300 import workloads as W
    lp = W.planted_sparse(args.m)
    A = lp.A.to_scipy()
    prm = O.Params(linsys=1, cg_tol=args.cg_tol, alpha=args.alpha, gamma=args.gamma)
    t0 = time.perf_counter()
    P = O.Problem(A, lp.b, lp.c)
    lin = O.make_linsys(P, prm)
    proj = O.Projection(P, lin)
    proj.cg_warm = prm.cg_warm
    setup_s = time.perf_counter() - t0
    st = O.initial_state(P)
    mu = prm.beta
    k = 0
    cg0 = lin.iters
    t1 = time.perf_counter()
    while time.perf_counter() - t1 < args.cpu_sample_s:
        if O.inner_residual_sq(P, st) <= mu:
            mu *= prm.gamma
            O.warm_start(st, prm.gamma, prm.warmstart)
            continue
        O.admm_step(P, proj, st, mu, prm)
        O.termination(P, st["y"], st["x"], st["s"], st["tau"], prm.eps,
                      float(np.linalg.norm(P.b)), float(np.linalg.norm(P.c)))
        k += 1
    it_s = (time.perf_counter() - t1) / max(k, 1)
    print(json.dumps({"setup_s": setup_s, "s_per_admm_iter": it_s, "admm_iters": k,
                      "cg_per_iter": (lin.iters - cg0) / max(k, 1), "cores": 1}))


def run_cpu_sample(args, admm_iters_per_step):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--m", str(args.m),
           "--cpu-sample-s", str(args.cpu_sample_s), "--cg-tol", str(args.cg_tol),
           "--alpha", str(args.alpha), "--gamma", str(args.gamma)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=900)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    step_s = d["setup_s"] + d["s_per_admm_iter"] * admm_iters_per_step
    return {
        "raw": d,
        "value": admm_iters_per_step / step_s,
        "unit": UNIT,
        "cores": d["cores"],
        "kind": "oracle",
        "sample": (f"FP64 numpy oracle, 1 thread, same LP and parameters: setup ({d['setup_s']:.2f} s) + "
                   f"{d['admm_iters']} ADMM updates ({d['s_per_admm_iter'] * 1e3:.1f} ms each, "
                   f"{d['cg_per_iter']:.1f} PCG iterations per update at cg_tol {args.cg_tol:g}), scaled to a "
                   f"step of setup + {admm_iters_per_step} updates"),
    }


def workload_config(args, m, n, nnz, world):
    """The `config` both arms print: the workload and the solver parameters of a step."""
    return {"workload": WORKLOAD, "m": m, "n": n, "nnz": int(nnz), "cg_tol": args.cg_tol, "cg_rel": args.cg_rel,
            "alpha": args.alpha, "gamma": args.gamma, "eps": 1e-6, "admm_updates_per_step": args.max_admm,
            "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas{world}"}


def reference_main(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, one bounded sample of the
    workload per step (its setup and the ADMM updates that fit in --cpu-sample-s); value and
    ms_per_step are those of the samples as run, the config is the GPU arm's."""
    if rank != 0:
        return
    times, updates = [], []
    cs = None
    for i in range(args.warmup + args.steps):
        cs = run_cpu_sample(args, args.max_admm)
        if i >= args.warmup:
            raw = cs.pop("raw")
            times.append(raw["setup_s"] + raw["s_per_admm_iter"] * raw["admm_iters"])
            updates.append(raw["admm_iters"])
    value = sum(updates) / sum(times)
    m = args.m
    sample = (f"each step: FP64 numpy oracle, 1 thread, on the same LP and parameters: setup + "
              f"{updates[-1]} ADMM updates ({times[-1]:.1f} s) of the {args.max_admm}-update step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, m, 4 * m, 25 * m, world),
        "sample_admm_updates_per_step": updates[-1],
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cs["cores"], "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": "the config's l2 and parallelism describe the GPU arm; this arm runs on the host cores",
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------

def main():
    args = parse()
    if args.cpu_sample:
        cpu_sample_main(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_main(args, rank, world)
        return

    import numpy as np
    import torch
    from paper_1805_12344_gb300 import abip, build, workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    L = abip.lib()
    dev = torch.device("cuda", local)

    lp = W.planted_sparse(args.m, seed=W.seed_for(W.SPARSE_PLANTED, rank))
    m, n, nnz = lp.m, lp.n, lp.A.nnz
    prm = abip.default_params(precision=abip.ABIP_PREC_MIXED if args.precision == "mixed" else abip.ABIP_PREC_F64,
                              max_admm_iters=args.max_admm, cg_tol=args.cg_tol, cg_rel=args.cg_rel,
                              alpha=args.alpha, gamma=args.gamma)
    # inputs resident in HBM
    rp_d = torch.from_numpy(lp.A.row_ptr).to(dev)
    ci_d = torch.from_numpy(lp.A.col_idx).to(dev)
    va_d = torch.from_numpy(lp.A.val).to(dev)
    b_d = torch.from_numpy(lp.b).to(dev)
    c_d = torch.from_numpy(lp.c).to(dev)
    x_d = torch.empty(n, dtype=torch.float64, device=dev)
    y_d = torch.empty(m, dtype=torch.float64, device=dev)
    s_d = torch.empty(n, dtype=torch.float64, device=dev)
    M = abip.abip_matrix()
    M.m, M.n, M.fmt, M.dtype, M.on_device = m, n, abip.ABIP_CSR, abip.ABIP_F32, 1
    M.row_ptr, M.col_idx, M.val, M.nnz = rp_d.data_ptr(), ci_d.data_ptr(), va_d.data_ptr(), nnz
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    import ctypes as C

    def step():
        h = C.c_void_p()
        rc = L.abip_setup(C.byref(M), b_d.data_ptr(), c_d.data_ptr(), C.byref(prm), C.byref(h))
        if rc != 0:
            raise abip.AbipError(rc, L.abip_last_error(None).decode())
        info = abip.abip_info()
        rc = L.abip_solve(h, x_d.data_ptr(), y_d.data_ptr(), s_d.data_ptr(), C.byref(info), stream.cuda_stream)
        err = L.abip_last_error(h).decode()
        L.abip_free(h)
        if rc != 0:
            raise abip.AbipError(rc, err)
        return info.as_dict()

    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    step_ms = []
    infos = []
    for _ in range(args.steps):
        flush.fill_(2.0)                       # L2 flush between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        infos.append(info)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    total_s = sum(step_ms) * 1e-3
    solved = sum(1 for i in infos if i["status"] == abip.ABIP_OPTIMAL)
    admm = sum(i["admm_iters"] for i in infos)
    total_s, solved, admm = aggregate_ranks(total_s, solved, admm, dist, dev)
    value = admm / total_s

    # roofline of the persistent solve kernel (one launch per step)
    vec_bytes = 4 if args.precision == "mixed" else 8
    last = infos[-1]
    alg = algorithmic_bytes(m, n, nnz, last["admm_iters"], last["cg_iters"], vec_bytes)
    achieved = alg / last["kernel_s"] / 1e9
    peak, peak_kind = measured_peaks()
    traffic = traffic_per_launch(last["admm_iters"]) if args.precision == "mixed" else None

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e and rank == 0:
        xh, yh, sh = np.zeros(n), np.zeros(m), np.zeros(n)
        torch.cuda.synchronize()
        flush.fill_(3.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hh = abip.abip_setup(lp.A, lp.b, lp.c, prm)
        inf = abip.abip_solve(hh, xh, yh, sh, stream=stream)
        abip.abip_free(hh)
        e2e_s = time.perf_counter() - t0
        h2d = lp.A.row_ptr.nbytes + lp.A.col_idx.nbytes + lp.A.val.nbytes + lp.b.nbytes + lp.c.nbytes
        d2h = xh.nbytes + yh.nbytes + sh.nbytes
        e2e = {"value": inf["admm_iters"] / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "seconds": e2e_s,
               "status": inf["status_name"]}

    legs = None
    if rank == 0 and not args.no_legs:
        legs = {}
        for key, fn in (("sparse_f64_arm", lambda: leg_sparse_f64(abip, W, lp, args, stream)),
                        ("batch_uneven", lambda: leg_batch_uneven(abip, W, args)),
                        ("basis_pursuit", lambda: leg_basis_pursuit(abip, W, args)),
                        ("random_udv", lambda: leg_random_udv(abip, W, args)),
                        ("svm_backward", lambda: leg_svm_backward(abip, W, args)),
                        ("bb_beta", lambda: leg_bb_beta(abip, W, args)),
                        ("sice", lambda: leg_sice(abip, W, args)),
                        ("grid_flow_direct", lambda: leg_grid_flow_direct(abip, W, args))):
            try:
                legs[key] = fn()
            except Exception as ex:  # a leg must not sink the main line
                legs[key] = {"failed": str(ex)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = run_cpu_sample(args, int(last["admm_iters"]))
        except Exception as ex:  # the baseline must not sink the GPU line
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(step_ms) / len(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": workload_config(args, m, n, nnz, world),
            "precision": args.precision,
            "lps_solved_per_s": solved / total_s,
            "lps_solved_note": ("0 on this workload: the paper's inner stop needs more than its 1e6-update cap "
                                "to reach a 1e-6 gap at n = 400000 (the gap falls like n mu / tau^2)"),
            "hbm_gbs_algorithmic": achieved,
            "status": [i["status_name"] for i in infos],
            "admm_iters": last["admm_iters"], "cg_iters": last["cg_iters"], "outer_iters": last["outer_iters"],
            "final": {"pres": last["pres"], "dres": last["dres"], "dgap": last["dgap"], "obj": last["obj"],
                      "p_star": lp.p_star},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": ("grid_delta_kernel (persistent solve, mixed precision)"
                                    if args.precision == "mixed" else "grid_kernel (persistent solve, FP64)"),
                         "kernel_s": last["kernel_s"], "algorithmic_bytes": alg,
                         "l2": {"peak": L2_PEAK_GBS, "frac": achieved / L2_PEAK_GBS, "unit": "GB/s",
                                "peak_kind": "ncu L2 sector peak of this GB300 (188 slices x 3 sectors/cycle "
                                             "x 32 B x 2.007 GHz)"}},
            "clocks": ck,
            "gpu_launches": int(sum(i["launches"] for i in infos)) + 1 * len(infos),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "lps_solved_legs": legs,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
