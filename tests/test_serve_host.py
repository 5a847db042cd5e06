"""Host logic of the served form (paper_1705_04384_gb300/serve.py) on the CPU.

The request loop, admission, the per-shape handle pool, the device-memory budget with
least-recently-used eviction and the time limit do not need a GPU: here the problem
handle is a fake whose asynchronous solve writes x = 2 b at enqueue (in stream order,
before the queued host copy of x) and reports ready after a set number of polls, and
the CUDA stream and device contexts are no-ops.
"""

import contextlib
import threading

import numpy as np
import pytest
import torch

from paper_1705_04384_gb300 import serve


class FakeStream:
    def __init__(self, *a, **k):
        pass

    def synchronize(self):
        pass


class FakeProblem:
    live = 0
    created = []
    lock = threading.Lock()
    polls_to_finish = 3

    def __init__(self, d, n_elem, p, geometry, r0, r1, precision, device, stream, grid):
        self.d, self.n_elem, self.p = d, n_elem, p
        self.N = (n_elem + p - 2) ** d
        self.device = torch.device("cpu")
        self.stream = stream
        self.closed = False
        self._left = None
        with FakeProblem.lock:
            FakeProblem.live += 1
            FakeProblem.created.append((d, n_elem, p, r0, r1))

    def prepare(self, nrhs, max_iter):
        pass

    def solve_async(self, b, x, tol, max_iter):
        assert self._left is None, "a second solve enqueued on a busy handle"
        x.copy_(2.0 * b)
        self._left = FakeProblem.polls_to_finish

    def ready(self):
        self._left -= 1
        return self._left <= 0

    def collect(self):
        assert self._left is not None and self._left <= 0
        self._left = None
        return {"iters": np.array([7]), "relres_true": np.array([1e-9]),
                "status": np.array([0])}

    def close(self):
        assert not self.closed
        self.closed = True
        with FakeProblem.lock:
            FakeProblem.live -= 1


class CpuSlot(serve._Slot):
    def __init__(self, problem, nbytes, key):
        self.P, self.nbytes, self.key = problem, nbytes, key
        self.busy, self.last_used, self.req = False, 0.0, None
        self.b = torch.empty(problem.N, dtype=torch.float64)
        self.x = torch.empty_like(self.b)
        self.h_rhs = torch.empty_like(self.b)
        self.h_x = torch.empty_like(self.b)


@pytest.fixture
def fake_device(monkeypatch):
    FakeProblem.live, FakeProblem.created, FakeProblem.polls_to_finish = 0, [], 3
    monkeypatch.setattr(serve, "Problem", FakeProblem)
    monkeypatch.setattr(serve, "_Slot", CpuSlot)
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "stream", lambda s=None: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "device", lambda d=None: contextlib.nullcontext())
    yield


def _requests(shapes, seed=0, spacing=0.0):
    rng = np.random.default_rng(seed)
    out = []
    for i, (d, ne, p) in enumerate(shapes):
        N = (ne + p - 2) ** d
        out.append(serve.Request(i, i * spacing, d, ne, p, rng.standard_normal(N)))
    return out


class Watch(serve.Server):
    """Records the in-flight count, the reserved bytes and the pool at every admission."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.max_inflight_seen = 0
        self.max_reserved_seen = 0
        self.max_per_key_seen = 0
        self.admissions = []

    def _start(self, s, req, now):
        super()._start(s, req, now)
        busy = sum(1 for ss in self.pool.values() for x in ss if x.busy)
        self.max_inflight_seen = max(self.max_inflight_seen, busy)
        self.max_reserved_seen = max(self.max_reserved_seen, self.reserved)
        self.max_per_key_seen = max(self.max_per_key_seen,
                                    max(len(v) for v in self.pool.values()))
        self.admissions.append((req.rid, busy))


def test_every_request_completes_with_its_own_result(fake_device):
    shapes = [(2, 8, 3), (3, 4, 2), (2, 8, 3), (2, 10, 4), (3, 4, 2), (2, 8, 3)] * 4
    reqs = _requests(shapes)
    rhs = {r.rid: r.rhs.copy() for r in reqs}
    srv = serve.Server(device="cpu", mem_budget=1 << 40, keep_solutions=True, max_inflight=4,
                       setup_threads=2)
    done = srv.run(reqs, realtime=False)
    srv.close()
    assert sorted(r.rid for r in done) == list(range(len(shapes)))
    for r in done:
        np.testing.assert_array_equal(r.x, 2.0 * rhs[r.rid])
        assert (r.iters, r.relres, r.status) == (7, 1e-9, 0)
        assert r.t_arrival <= r.t_admit <= r.t_done
    assert FakeProblem.live == 0  # close() released every handle


def test_inflight_and_per_shape_limits(fake_device):
    shapes = [(2, 8, 3)] * 30 + [(2, 9, 3)] * 10
    srv = Watch(device="cpu", mem_budget=1 << 40, max_inflight=5, max_per_key=3)
    done = srv.run(_requests(shapes), realtime=False)
    srv.close()
    assert len(done) == 40
    assert srv.max_inflight_seen <= 5
    assert srv.max_per_key_seen <= 3
    # requests of one shape share its handles: at most max_per_key setups per shape
    assert srv.setups <= 6


def test_memory_budget_with_lru_eviction(fake_device):
    # three shapes, budget for two handles of the largest: the idle least recently used
    # handle is closed to make room
    need = {s: serve.handle_bytes(s[0], (s[1] + s[2] - 2) ** s[0], 100, "tf32")
            for s in [(2, 40, 3), (2, 41, 3), (2, 42, 3)]}
    budget = 2 * max(need.values()) + 1
    shapes = [(2, 40, 3), (2, 41, 3), (2, 42, 3), (2, 40, 3), (2, 42, 3), (2, 41, 3)]
    srv = Watch(device="cpu", mem_budget=budget, max_inflight=2, max_per_key=1)
    done = srv.run(_requests(shapes), realtime=False)
    assert len(done) == 6
    assert srv.max_reserved_seen <= budget
    assert srv.reserved <= budget
    # every shape got a handle, but at most two were ever held at once: a handle was
    # evicted to make room (waiting requests of shapes with a handle go first, so no
    # evicted shape had to be set up again here)
    assert srv.setups >= 3
    assert sum(len(v) for v in srv.pool.values()) <= 2
    assert FakeProblem.live <= 2
    srv.close()
    assert srv.reserved == 0 and FakeProblem.live == 0


def test_request_above_the_budget_is_refused(fake_device):
    srv = serve.Server(device="cpu", mem_budget=1000)
    with pytest.raises(RuntimeError, match="above the budget"):
        srv.run(_requests([(2, 8, 3)]), realtime=False)
    srv.close()


def test_arrivals_are_admitted_while_others_are_in_flight(fake_device):
    # slow solves (many polls each): later requests of a ready shape must be admitted
    # before the earlier ones finish, i.e. several solves overlap
    FakeProblem.polls_to_finish = 200
    srv = Watch(device="cpu", mem_budget=1 << 40, max_inflight=8, max_per_key=8)
    done = srv.run(_requests([(2, 8, 3)] * 16), realtime=False)
    srv.close()
    assert len(done) == 16
    assert max(b for _, b in srv.admissions) >= 4


def test_time_limit_stops_admission_and_drains(fake_device):
    # arrivals spread over 100 s, a 0.2 s limit: only the first arrivals are served,
    # and every admitted request completes
    reqs = _requests([(2, 8, 3)] * 20, spacing=5.0)
    srv = serve.Server(device="cpu", mem_budget=1 << 40)
    done = srv.run(reqs, realtime=True, time_limit=0.2)
    srv.close()
    assert 1 <= len(done) < 20
    assert all(r.status == 0 and r.t_done is not None for r in done)


def test_latency_stats():
    class R:
        def __init__(self, t0, t1, ne, p, it):
            self.t_arrival, self.t_done, self.n_elem, self.p, self.d, self.iters = (
                t0, t1, ne, p, 2, it)

    st = serve.latency_stats([R(0.0, 0.010, 8, 3, 5), R(0.5, 0.530, 8, 3, 6)])
    assert st["completed"] == 2
    assert st["p50_ms"] == pytest.approx(20.0)
    assert st["span_s"] == pytest.approx(0.53)
    assert st["dof_iters"] == 81 * 11
    assert serve.latency_stats([]) == {"completed": 0}


def test_warm_shapes_go_first_and_setups_are_bounded(fake_device):
    """A request whose shape has an idle handle is admitted ahead of older requests that
    wait for a setup, and no more than setup_threads setups run at once."""
    FakeProblem.polls_to_finish = 2
    shapes = [(2, 8 + i, 3) for i in range(12)] + [(2, 8, 3)] * 6
    srv = Watch(device="cpu", mem_budget=1 << 40, max_inflight=4, setup_threads=2)
    seen = []
    orig = srv._start_setup

    def spy(req):
        seen.append(len(srv.setting_up))
        return orig(req)

    srv._start_setup = spy
    done = srv.run(_requests(shapes), realtime=False)
    srv.close()
    assert len(done) == len(shapes)
    assert max(seen) <= 1  # at most one other setup running when a new one starts
    order = [rid for rid, _ in srv.admissions]
    # the repeated shape (2, 8, 3) is set up first; its later requests (ids 12..17) are
    # admitted before most of the other shapes' first requests
    assert order.index(12) < order.index(11)


def test_dropped_requests_are_counted(fake_device):
    reqs = _requests([(2, 8, 3)] * 10, spacing=5.0)
    srv = serve.Server(device="cpu", mem_budget=1 << 40)
    done = srv.run(reqs, realtime=True, time_limit=0.2)
    srv.close()
    assert len(done) + srv.dropped == 10
