"""BiCGStab + FD iteration counts on the configurations of the paper's collocation tables.

    python -m paper_1705_04384_gb300.paper_tables [--tols 1e-6 1e-8]

Table 2 (quarter ring, h^-1 = 128 .. 1024, p = 2 .. 5) and Table 4 (revolved quarter
ring, h^-1 = 16 .. 64, p = 2 .. 5) of Sec. 5 report BiCGStab + FD iterations in halves.
The paper states neither its tolerance (Matlab's ``bicgstab`` defaults to 1e-6) nor its
source term (K = I); here f = 1 on the ring r in [1, 2], x0 = 0, and the counts are
printed for each tolerance next to the paper's, with the GPU time of one solve (setup
excluded; the paper's times are single-core Matlab times including setup).
"""

import argparse
import time

import numpy as np
import torch

from .api import Problem

# iterations from Sec. 5, Table 2 (collocation, quarter of ring) and Table 4
# (collocation, revolved quarter ring), BiCGStab + P
PAPER = {
    ("quarter", 128): [13.5, 13.5, 12.0, 12.0],
    ("quarter", 256): [13.5, 13.5, 13.5, 13.5],
    ("quarter", 512): [13.5, 13.5, 13.5, 13.5],
    ("quarter", 1024): [13.5, 13.5, 13.5, 13.5],
    ("revolved", 16): [16.0, 15.5, 17.5, 17.5],
    ("revolved", 32): [16.5, 18.5, 20.5, 22.0],
    ("revolved", 64): [17.5, 19.5, 21.5, 22.5],
}
PS = [2, 3, 4, 5]


def run(tols, max_iter=500):
    rows = []
    for (dom, hinv), paper in PAPER.items():
        d, geo = (2, "annulus") if dom == "quarter" else (3, "revolved")
        for p, pit in zip(PS, paper):
            t0 = time.perf_counter()
            P = Problem(d, hinv, p, geo, 1.0, 2.0)
            torch.cuda.synchronize()
            t_setup = time.perf_counter() - t0
            b = torch.ones(P.N, dtype=torch.float64, device="cuda")
            res = {}
            for tol in tols:
                P.solve_bicgstab(b, tol=tol, max_iter=max_iter)  # graph capture, warm-up
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                x, info = P.solve_bicgstab(b, tol=tol, max_iter=max_iter)
                e1.record()
                torch.cuda.synchronize()
                res[tol] = (info["iters"], e0.elapsed_time(e1), info["relres_true"], info["status"])
            rows.append((dom, hinv, p, P.N, pit, t_setup, res))
            P.close()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--tols", type=float, nargs="+", default=[1e-6, 1e-8])
    a = ap.parse_args()
    rows = run(a.tols)
    head = "| domain | h^-1 | p | N | paper | " + " | ".join(
        f"ours tol {t:g} (iters / ms)" for t in a.tols) + " | setup s |"
    print(head)
    print("|" + "---|" * (head.count("|") - 1))
    for dom, hinv, p, N, pit, ts, res in rows:
        cells = " | ".join(f"{res[t][0]:.1f} / {res[t][1]:.2f}" for t in a.tols)
        print(f"| {dom} | {hinv} | {p} | {N} | {pit:.1f} | {cells} | {ts:.2f} |")
    bad = [(r[0], r[1], r[2]) for r in rows for t in a.tols if r[6][t][3] != 0]
    if bad:
        print("not converged:", bad)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
