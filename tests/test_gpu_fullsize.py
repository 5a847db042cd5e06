"""The batched and served forms on their full workloads, in the configuration bench.py
times: every solve must converge to the FP64 true residual 1e-8 (computed by the
library in FP64), and sampled solves are checked against the oracle's collocation rows
at sampled points (the full systems are too large to assemble on the CPU in seconds).
The served requests must also give the same bits alone as in the mix."""

import numpy as np
import pytest
import torch

import workload as W
from tests.oracle_ref import ref

pytestmark = pytest.mark.gpu


def _sampled_residual(d, ne, p, r0, r1, b, x, seed, count=16):
    R = ref(d, ne, p, "annulus", r0, r1, assemble=False)
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([[0, R.N - 1], rng.integers(0, R.N, count)]))
    return np.max(np.abs(b[idx] - R.rows(idx) @ x)) / np.linalg.norm(b)


def test_batched_full_workload():
    """256 2D problems (n_elem U{32..512}, p U{2..6}, r0 U[0.5,1.5]) x 8 Gaussian rhs,
    TF32 FD, throughput reduction grid, one iga_solve_batched call (as bench.py)."""
    from paper_1705_04384_gb300.api import Problem, solve_batched
    specs = W.batched_problems(count=256)
    probs, rhs, outs = [], [], []
    try:
        for sp in specs:
            P = Problem(2, sp["n_elem"], sp["p"], "annulus", sp["r0"], sp["r1"],
                        precision="tf32", stream=torch.cuda.Stream(), grid="throughput")
            P.prepare(sp["nrhs"], 50)
            probs.append(P)
            rhs.append(torch.from_numpy(W.gaussian_rhs(P.N, sp["nrhs"], sp["rhs_seed"])).cuda())
            outs.append(torch.empty_like(rhs[-1]))
        torch.cuda.synchronize()
        res = solve_batched(probs, rhs, outs, tol=1e-8, max_iter=50)
        torch.cuda.synchronize()
        assert int(res["nrhs"].sum()) == 256 * 8
        assert np.all(res["status"] == 0)
        assert float(res["relres_true"].max()) <= 1.05e-8
        # oracle rows for the largest problem, a p = 2 and a p = 6 one (right-hand side 0)
        big = int(np.argmax([P.N for P in probs]))
        p2 = next(i for i, sp in enumerate(specs) if sp["p"] == 2)
        p6 = next(i for i, sp in enumerate(specs) if sp["p"] == 6)
        for q in (big, p2, p6):
            sp = specs[q]
            b = rhs[q][0].cpu().numpy()
            x = outs[q][0].cpu().numpy()
            err = _sampled_residual(2, sp["n_elem"], sp["p"], sp["r0"], sp["r1"], b, x, q)
            assert err <= 1.05e-8, (q, err)
    finally:
        for P in probs:
            P.close()


def test_served_full_distribution():
    """The first requests of the served workload (Poisson arrivals at 2000 req/s mixing
    2D n_elem U[64,1024], p U{2..6} and 3D n_elem U[32,160], p U{3..6}), through the
    bench's server configuration (TF32 FD, 64 in flight, 8 setup threads)."""
    from paper_1705_04384_gb300.api import Problem
    from paper_1705_04384_gb300.serve import Request, Server
    raw = W.served_requests(rate=2000.0, duration=0.006, seed=3)
    assert len(raw) >= 8
    reqs = [Request(i, r["t_arrival"], r["d"], r["n_elem"], r["p"],
                    rhs=lambda N, s=r["rhs_seed"]: W.gaussian_rhs(N, 1, s)[0],
                    r0=r["r0"], r1=r["r1"]) for i, r in enumerate(raw)]
    srv = Server(precision="tf32", tol=1e-8, max_iter=100, max_inflight=64, setup_threads=8,
                 keep_solutions=True)
    try:
        done = srv.run(reqs, realtime=False)
        assert len(done) == len(reqs)
        for r in done:
            assert r.status == 0 and r.relres <= 1.05e-8, (r.rid, r.status, r.relres)
        # the two smallest: the same bits alone, and the oracle's rows at sampled points
        for r in sorted(done, key=lambda r: W.dofs(r.d, r.n_elem, r.p))[:2]:
            with Problem(r.d, r.n_elem, r.p, "annulus", r.r0, r.r1, precision="tf32",
                         grid=srv.grid) as P:
                b = r.rhs(P.N)
                x, info = P.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=100)
                assert info["iters"] == r.iters and np.array_equal(x.cpu().numpy(), r.x)
            assert _sampled_residual(r.d, r.n_elem, r.p, r.r0, r.r1, b, r.x, r.rid) <= 1.05e-8
    finally:
        srv.close()
