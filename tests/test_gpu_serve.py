"""Served form: requests admitted as slots and memory free up, overlapping on the
device; each result must be the same alone and in the mix (bitwise: every kernel
reduces in a fixed order), and must meet the FP64 true residual 1e-8."""

import numpy as np
import pytest
import torch

import workload as W
from tests.oracle_ref import ref

pytestmark = pytest.mark.gpu


def _requests(seed=7, count=18, spread=0.02):
    rng = np.random.default_rng(seed)
    shapes = [(2, 40, 3), (2, 57, 5), (3, 8, 3), (2, 33, 2), (3, 10, 6), (2, 90, 4)]
    from paper_1705_04384_gb300.serve import Request
    reqs = []
    t = 0.0
    for i in range(count):
        d, ne, p = shapes[int(rng.integers(len(shapes)))]
        t += float(rng.exponential(spread / count))
        seed_i = 1000 + i
        reqs.append(Request(i, t, d, ne, p,
                            rhs=lambda N, s=seed_i: W.gaussian_rhs(N, 1, s)[0]))
    return reqs


def _alone(req, precision, grid):
    from paper_1705_04384_gb300.api import Problem
    with Problem(req.d, req.n_elem, req.p, "annulus", req.r0, req.r1, precision=precision,
                 grid=grid) as P:
        b = torch.from_numpy(req.rhs(P.N)).cuda()
        x, info = P.solve(b, tol=1e-8, max_iter=100)
        return x.cpu().numpy(), info


@pytest.mark.parametrize("precision,budget", [("tf32", None), ("fp64", None), ("tf32", 60e6)])
def test_served_results_equal_alone(precision, budget):
    from paper_1705_04384_gb300.serve import Server, latency_stats
    reqs = _requests()
    srv = Server(precision=precision, max_inflight=6, keep_solutions=True,
                 mem_budget=None if budget is None else int(budget))
    done = srv.run(reqs, realtime=True)
    stats = latency_stats(done)
    srv.close()
    assert len(done) == len(reqs) and stats["completed"] == len(reqs)
    if budget is not None:
        assert srv.setups > 6  # the small budget forced evictions and re-setup
    for r in done:
        assert r.status == 0 and r.relres <= 1.05e-8
        x, info = _alone(r, precision, srv.grid)
        assert info["iters"] == r.iters
        assert np.array_equal(x, r.x), r.rid
    # oracle residual on a few of them
    for r in done[:4]:
        R = ref(r.d, r.n_elem, r.p)
        b = r.rhs(R.N)
        assert np.linalg.norm(b - R.A @ r.x) / np.linalg.norm(b) <= 1.05e-8
