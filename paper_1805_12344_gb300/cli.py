"""Command-line runs of the generated workloads through the library (timing and status).

    python -m paper_1805_12344_gb300.cli shared --m 2048 --nd 8192 --batch 64 --precision bf16
    python -m paper_1805_12344_gb300.cli batch --count 64 --precision mixed
    python -m paper_1805_12344_gb300.cli svm --precision mixed --max-admm 4000
    python -m paper_1805_12344_gb300.cli flow --side 16 --linsys ldl --precision f64

Prints one JSON line per run: statuses, ADMM updates, device time of setup and
iterations as the library reports them (abip_info.setup_s / kernel_s).
"""
from __future__ import annotations

import argparse
import json
import time

from . import abip, workloads as W

PRECISION = {"f64": abip.ABIP_PREC_F64, "mixed": abip.ABIP_PREC_MIXED, "bf16": abip.ABIP_PREC_MIXED_BF16}


def _summary(kind, infos, wall, extra):
    st = [f["status_name"] for f in infos]
    return dict(kind=kind, count=len(infos), statuses={k: st.count(k) for k in sorted(set(st))},
                admm_iters_max=max(f["admm_iters"] for f in infos),
                admm_iters_total=sum(f["admm_iters"] for f in infos),
                setup_s=infos[0]["setup_s"], kernel_s=infos[0]["kernel_s"], wall_s=wall, **extra)


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    sh = sub.add_parser("shared", help="basis pursuit batch sharing one dictionary")
    sh.add_argument("--m", type=int, default=2048)
    sh.add_argument("--nd", type=int, default=8192)
    sh.add_argument("--batch", type=int, default=64)
    bt = sub.add_parser("batch", help="uneven batch of dense planted LPs")
    bt.add_argument("--count", type=int, default=64)
    sv = sub.add_parser("svm", help="L1-SVM LPs: one through abip_setup/abip_solve, or a batch")
    sv.add_argument("--d", type=int, default=64)
    sv.add_argument("--N", type=int, default=512)
    sv.add_argument("--batch", type=int, default=0, help="solve this many instances (seeds seed..seed+batch-1) in one batch")
    fl = sub.add_parser("flow", help="planted min-cost flow LP on a grid (sparse path, PCG or the direct projection)")
    fl.add_argument("--side", type=int, default=16)
    fl.add_argument("--linsys", choices=["pcg", "ldl"], default="ldl")
    for p in (sh, bt, sv, fl):
        p.add_argument("--precision", choices=sorted(PRECISION), default="mixed")
        p.add_argument("--max-admm", type=int, default=1000000)
        p.add_argument("--eps", type=float, default=1e-6)
        p.add_argument("--seed", type=int, default=None)
    a = ap.parse_args(argv)
    abip.lib()
    prm = abip.default_params(precision=PRECISION[a.precision], max_admm_iters=a.max_admm, eps=a.eps)
    t0 = time.time()
    if a.cmd == "shared":
        sb = W.basis_pursuit(a.m, a.nd, batch=a.batch, seed=a.seed)
        t0 = time.time()
        infos, *_ = abip.abip_solve_batch_shared(sb.A, sb.bs, sb.cs, prm, want_solution=False)
        solved = sum(1 for f in infos if f["status"] == abip.ABIP_OPTIMAL)
        out = _summary("basis_pursuit_shared", infos, time.time() - t0,
                       dict(m=a.m, n=2 * a.nd, precision=a.precision,
                            ms_per_cycle=1e3 * infos[0]["kernel_s"] / max(1, max(f["admm_iters"] for f in infos)),
                            lps_solved_per_s=solved / (infos[0]["kernel_s"] + infos[0]["setup_s"])))
    elif a.cmd == "batch":
        lps = W.batch_uneven(count=a.count, seed=a.seed)
        t0 = time.time()
        infos, *_ = abip.abip_solve_batch([l.A for l in lps], [l.b for l in lps], [l.c for l in lps], prm,
                                          want_solution=False)
        out = _summary("batch_uneven", infos, time.time() - t0, dict(precision=a.precision))
    elif a.cmd == "flow":
        lp = W.grid_flow(a.side, seed=a.seed)
        linsys = abip.ABIP_LINSYS_SPARSE_LDL if a.linsys == "ldl" else abip.ABIP_LINSYS_PCG
        s = abip.Solver(lp.A, lp.b, lp.c, linsys=linsys, precision=PRECISION[a.precision], max_admm_iters=a.max_admm,
                        eps=a.eps)
        t0 = time.time()
        info, *_ = s.solve()
        s.close()
        out = _summary("grid_flow", [info], time.time() - t0,
                       dict(side=a.side, m=lp.m, n=lp.n, linsys=a.linsys, precision=a.precision,
                            cg_iters_per_update=info["cg_iters"] / max(1, info["admm_iters"]),
                            us_per_update=1e6 * info["kernel_s"] / max(1, info["admm_iters"])))
    elif a.batch > 0:
        base = W.seed_for(W.L1_SVM) if a.seed is None else a.seed
        lps = [W.l1_svm(d=a.d, N=a.N, seed=base + k) for k in range(a.batch)]
        t0 = time.time()
        infos, *_ = abip.abip_solve_batch([l.A for l in lps], [l.b for l in lps], [l.c for l in lps], prm,
                                          want_solution=False)
        wall = time.time() - t0
        solved = sum(1 for f in infos if f["status"] == abip.ABIP_OPTIMAL)
        out = _summary("l1_svm_batch", infos, wall, dict(m=a.N, n=2 * a.d + 2 + 2 * a.N, precision=a.precision,
                                                         lps_solved_per_s=solved / infos[0]["kernel_s"]))
    else:
        lp = W.l1_svm(d=a.d, N=a.N, seed=a.seed)
        s = abip.Solver(lp.A, lp.b, lp.c, linsys=0, precision=PRECISION[a.precision], max_admm_iters=a.max_admm,
                        eps=a.eps)
        t0 = time.time()
        info, *_ = s.solve()
        s.close()
        out = _summary("l1_svm", [info], time.time() - t0,
                       dict(m=lp.A.shape[0], n=lp.A.shape[1], precision=a.precision,
                            us_per_update=1e6 * info["kernel_s"] / max(1, info["admm_iters"])))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
