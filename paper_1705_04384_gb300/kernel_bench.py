"""Time one operation of the library in isolation (CUDA events on the call stream).

    python -m paper_1705_04384_gb300.kernel_bench --op fd|operator|solve \
        --d 3 --ne 64 --p 3 --precision fp64 --reps 20
    python -m paper_1705_04384_gb300.kernel_bench --op fp64peak

Used to attribute time to kernels and as the small, self-contained command for
ncu captures.  Prints one JSON line with the mean time per call.
"""

import argparse
import json

import numpy as np
import torch

from .api import Problem, measure_fp64_peak


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="fd", choices=["fd", "operator", "solve", "fp64peak"])
    ap.add_argument("--d", type=int, default=3)
    ap.add_argument("--ne", type=int, default=64)
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--geometry", default="annulus")
    ap.add_argument("--scheme", default="collocation", choices=["collocation", "wq"],
                    help="discretization: collocation (Sec. 2.2) or weighted-quadrature "
                         "Galerkin (Sec. 2.3)")
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--max-iter", type=int, default=200,
                    help="Krylov workspace of --op solve (steps)")
    ap.add_argument("--nrhs", type=int, default=1,
                    help="right-hand sides of --op solve (solved in lockstep, iga_solve_multi)")
    a = ap.parse_args()
    if a.op == "fp64peak":
        # the FP64 ceiling (iga_fp64_probe): best of a.reps timed launches per probe kind
        r = measure_fp64_peak(reps=1000, trials=a.reps, mixed=True)
        print(json.dumps({"op": "fp64peak", "gflops_dmma": r["dmma"], "gflops_fma": r["fma"],
                          "gflops_peak": r["peak"], "gflops_both_split_warps": r["split"],
                          "gflops_both_in_each_warp": r["interleaved"], "trials": a.reps}))
        return
    P = Problem(a.d, a.ne, a.p, geometry=a.geometry, precision=a.precision, scheme=a.scheme)
    g = torch.Generator(device="cpu").manual_seed(0)
    b = torch.randn(P.N, dtype=torch.float64, generator=g).cuda()
    out = torch.empty_like(b)
    if a.op == "solve" and a.nrhs > 1:
        P.prepare(a.nrhs, a.max_iter)
        B = torch.randn(a.nrhs, P.N, dtype=torch.float64, generator=g).cuda()
    s = torch.cuda.current_stream()
    last = {}

    def call():
        if a.op == "fd":
            P.precond_apply(b, out=out)
        elif a.op == "operator":
            P.apply_operator(b, out=out)
        elif a.nrhs > 1:
            last["info"] = P.solve_multi(B, tol=1e-8, max_iter=a.max_iter)[1]
        else:
            last["info"] = P.solve(b, tol=1e-8, max_iter=a.max_iter, out=out)[1]

    for _ in range(a.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(a.reps):
        e0.record(s)
        call()
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e3)
    print(json.dumps({"op": a.op, "scheme": a.scheme, "d": a.d, "ne": a.ne, "p": a.p, "n": P.n,
                      "N": P.N,
                      "nrhs": a.nrhs,
                      "precision": a.precision, "us_mean": float(np.mean(times)),
                      "us_min": float(np.min(times)), "reps": a.reps,
                      "iters": (np.asarray(last["info"]["iters"]).tolist()
                                if "info" in last else None)}))
    P.close()


if __name__ == "__main__":
    main()
