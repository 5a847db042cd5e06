"""Thin Python binding over the C ABI (include/iga_fd.h).

Argument marshalling only: torch tensors supply device memory and the stream;
every step of the method runs inside ``libiga_fd.so``.
"""

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import Geometry, check

GEOM = {"identity": 0, "annulus": 1, "revolved": 2}
PREC = {"fp64": 0, "tf32": 1, "bf16": 2, "none": 3, "tf32x3": 4, "fp64tc": 5}
FACTOR = {"tau": 0, "M": 1, "B1": 2, "K": 3, "lambda": 4, "U": 5, "Vt": 6}
GRID = {"latency": 0, "throughput": 1}
SCHEME = {"collocation": 0, "wq": 1}
STATUS_OK, STATUS_NO_CONVERGENCE, STATUS_NAN = 0, 5, 7


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Problem:
    """One problem on one device: ``iga_setup_scheme`` ... ``iga_destroy``.

    d (2 or 3), n_elem elements per direction, degree p; geometry "identity", "annulus" or
    "revolved" with radii r_inner < r_outer; scheme "collocation" or "wq" (weighted-quadrature
    Galerkin); wind: a constant convection field (collocation, FP64 or no preconditioner).
    precision selects the FD preconditioner's arithmetic (``iga_precision``):
      "fp64"    plain GMRES, FP64 FD;
      "fp64tc"  plain GMRES, the FP64 FD to FP64 accuracy from exact BF16 slice products on
                the tensor cores (n <= 148, no wind);
      "tf32", "bf16", "tf32x3"  flexible GMRES, the FD on the tensor cores with FP32
                accumulation ("tf32x3": error-compensated TF32);
      "none"    no preconditioner.
    grid "latency" (one solve at a time) or "throughput" (batched / served); stream: the
    torch CUDA stream the handle's work runs on.
    """

    def __init__(self, d, n_elem, p, geometry="annulus", r_inner=1.0, r_outer=2.0,
                 precision="fp64", device="cuda", stream=None, grid="latency", wind=None,
                 scheme="collocation"):
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.d, self.n_elem, self.p = d, n_elem, p
        self.precision = precision
        self.scheme = scheme
        self.geometry = geometry
        self.r_inner, self.r_outer = r_inner, r_outer
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        g = Geometry(GEOM[geometry], float(r_inner), float(r_outer))
        self.wind = tuple(float(w) for w in wind) if wind is not None else None
        if self.wind is not None:
            for l, w in enumerate(self.wind[:3]):
                g.wind[l] = w
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.iga_setup_scheme(d, n_elem, p, ctypes.byref(g), SCHEME[scheme],
                                            PREC[precision], ctypes.c_void_p(stream.cuda_stream),
                                            ctypes.byref(h)), "iga_setup_scheme")
        self.h = h
        n = ctypes.c_int()
        N = ctypes.c_longlong()
        check(self.lib.iga_dims(self.h, ctypes.byref(n), ctypes.byref(N)), "iga_dims")
        self.n, self.N = n.value, N.value
        if grid != "latency":
            self.set_grid_mode(grid)

    def close(self):
        if getattr(self, "h", None):
            self.lib.iga_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- host queries
    def collocation_points(self):
        out = np.empty((self.N, self.d), dtype=np.float64)
        check(self.lib.iga_collocation_points(self.h, out.ctypes.data_as(ctypes.c_void_p)),
              "iga_collocation_points")
        return out

    def quadrature_dims(self):
        """(nq, Nq) of a weighted-quadrature problem."""
        nq, Nq = ctypes.c_int(), ctypes.c_longlong()
        check(self.lib.iga_quadrature_dims(self.h, ctypes.byref(nq), ctypes.byref(Nq)),
              "iga_quadrature_dims")
        return nq.value, Nq.value

    def quadrature_points(self):
        """Physical WQ quadrature points, (Nq, d), direction 1 fastest."""
        _, Nq = self.quadrature_dims()
        out = np.empty((Nq, self.d), dtype=np.float64)
        check(self.lib.iga_quadrature_points(self.h, out.ctypes.data_as(ctypes.c_void_p)),
              "iga_quadrature_points")
        return out

    def wq_load(self, g, out=None):
        """Load vector of a WQ problem from source values g at the quadrature points."""
        _, Nq = self.quadrature_dims()
        g = torch.as_tensor(g, dtype=torch.float64, device=self.device).contiguous()
        if g.numel() != Nq:
            raise ValueError(f"expected {Nq} values, got {g.numel()}")
        out = torch.empty(self.N, dtype=torch.float64, device=self.device) if out is None else out
        check(self.lib.iga_wq_load(self.h, _ptr(g), _ptr(out)), "iga_wq_load")
        return out

    def factor(self, which, direction=0):
        shape = (self.n,) if which in ("tau", "lambda") else (self.n, self.n)
        out = np.empty(shape, dtype=np.float64)
        check(self.lib.iga_get_factor(self.h, direction, FACTOR[which],
                                      out.ctypes.data_as(ctypes.c_void_p)), "iga_get_factor")
        return out

    def set_grid_mode(self, grid):
        """'latency' (one solve at a time) or 'throughput' (many solves at once)."""
        check(self.lib.iga_set_grid_mode(self.h, GRID[grid]), "iga_set_grid_mode")
        self.grid = grid

    def prepare(self, nrhs=1, max_iter=200):
        """Allocate the solve workspace and capture the solve graph ahead of time."""
        check(self.lib.iga_prepare(self.h, int(nrhs), int(max_iter)), "iga_prepare")

    def fd_kernel(self, nrhs=1):
        """Name of the kernel that runs this handle's FD mode products for nrhs
        right-hand sides: fold_mma, fold_fma, dense_mma, tensor_core or fp64_slices."""
        k = ctypes.c_int()
        check(self.lib.iga_fd_kernel(self.h, int(nrhs), ctypes.byref(k)), "iga_fd_kernel")
        return ("fold_mma", "fold_fma", "dense_mma", "tensor_core", "fp64_slices")[k.value]

    def operator_flops(self):
        """Algorithmic FLOPs of one operator application (iga_operator_flops)."""
        f = ctypes.c_double()
        check(self.lib.iga_operator_flops(self.h, ctypes.byref(f)), "iga_operator_flops")
        return f.value

    def launch_counts(self):
        """(fixed, per_iteration): kernel launches of one solve = fixed + per_iteration * iters."""
        f, it = ctypes.c_int(), ctypes.c_int()
        check(self.lib.iga_launch_counts(self.h, ctypes.byref(f), ctypes.byref(it)),
              "iga_launch_counts")
        return f.value, it.value

    # ---------------------------------------------------------------- device ops
    def _vec(self, v):
        v = torch.as_tensor(v, dtype=torch.float64, device=self.device).contiguous()
        if v.numel() != self.N:
            raise ValueError(f"expected {self.N} values, got {v.numel()}")
        return v

    def apply_operator(self, u, out=None):
        u = self._vec(u)
        out = torch.empty_like(u) if out is None else out
        check(self.lib.iga_apply_operator(self.h, _ptr(u), _ptr(out)), "iga_apply_operator")
        return out

    def precond_apply(self, b, out=None):
        b = self._vec(b)
        out = torch.empty_like(b) if out is None else out
        check(self.lib.iga_precond_apply(self.h, _ptr(b), _ptr(out)), "iga_precond_apply")
        return out

    def solve(self, rhs, x0=None, tol=1e-8, max_iter=200, out=None, allow_no_convergence=True):
        """Returns (x, info) with info = dict(iters, hist, relres_true, status)."""
        rhs = self._vec(rhs)
        if out is None:
            out = torch.empty_like(rhs)
        use_x0 = 0
        if x0 is not None:
            out.copy_(self._vec(x0))
            use_x0 = 1
        iters = ctypes.c_int()
        rel = ctypes.c_double()
        hist = np.zeros(max_iter + 1, dtype=np.float64)
        st = self.lib.iga_solve(self.h, _ptr(rhs), _ptr(out), use_x0, float(tol), int(max_iter),
                                ctypes.byref(iters), hist.ctypes.data_as(ctypes.c_void_p),
                                ctypes.byref(rel))
        allow = (STATUS_NO_CONVERGENCE,) if allow_no_convergence else ()
        check(st, "iga_solve", allow)
        k = iters.value
        return out, dict(iters=k, hist=hist[:k + 1].copy(), relres_true=rel.value, status=st)

    def solve_bicgstab(self, rhs, x0=None, tol=1e-8, max_iter=200, out=None,
                       allow_no_convergence=True):
        """BiCGStab + FD (Sec. 5's solver).  Returns (x, info) with info = dict(half_steps,
        iters = half_steps / 2 (the paper's k or k - 0.5), hist, relres_true, status)."""
        rhs = self._vec(rhs)
        if out is None:
            out = torch.empty_like(rhs)
        use_x0 = 0
        if x0 is not None:
            out.copy_(self._vec(x0))
            use_x0 = 1
        steps = ctypes.c_int()
        rel = ctypes.c_double()
        hist = np.zeros(2 * max_iter + 1, dtype=np.float64)
        st = self.lib.iga_solve_bicgstab(self.h, _ptr(rhs), _ptr(out), use_x0, float(tol),
                                         int(max_iter), ctypes.byref(steps),
                                         hist.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rel))
        allow = (STATUS_NO_CONVERGENCE,) if allow_no_convergence else ()
        check(st, "iga_solve_bicgstab", allow)
        k = steps.value
        return out, dict(half_steps=k, iters=k / 2.0, hist=hist[:k + 1].copy(),
                         relres_true=rel.value, status=st)

    def solve_host(self, rhs_host, x_host, tol=1e-8, max_iter=200):
        """Host-buffer solve (copies inside the call).  rhs_host/x_host: float64 arrays or
        CPU tensors (pinned for asynchronous copies)."""
        iters = ctypes.c_int()
        rel = ctypes.c_double()
        hist = np.zeros(max_iter + 1, dtype=np.float64)
        rp = rhs_host.data_ptr() if isinstance(rhs_host, torch.Tensor) else rhs_host.ctypes.data
        xp = x_host.data_ptr() if isinstance(x_host, torch.Tensor) else x_host.ctypes.data
        st = self.lib.iga_solve_host(self.h, ctypes.c_void_p(rp), ctypes.c_void_p(xp), float(tol),
                                     int(max_iter), ctypes.byref(iters),
                                     hist.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rel))
        check(st, "iga_solve_host", (STATUS_NO_CONVERGENCE,))
        return dict(iters=iters.value, hist=hist[:iters.value + 1].copy(),
                    relres_true=rel.value, status=st)

    # ---------------------------------------------------------------- many right-hand sides
    def _block(self, v, nrhs):
        v = torch.as_tensor(v, dtype=torch.float64, device=self.device).contiguous()
        if v.numel() != nrhs * self.N:
            raise ValueError(f"expected {nrhs} x {self.N} values, got {v.numel()}")
        return v

    def solve_multi(self, rhs, tol=1e-8, max_iter=200, x0=None, out=None):
        """rhs: (nrhs, N).  Returns (x, info) with per-rhs lists."""
        nrhs = rhs.shape[0] if hasattr(rhs, "shape") and len(rhs.shape) == 2 else 1
        rhs = self._block(rhs, nrhs)
        out = torch.empty_like(rhs) if out is None else out
        use_x0 = 0
        if x0 is not None:
            out.copy_(self._block(x0, nrhs))
            use_x0 = 1
        iters = np.zeros(nrhs, dtype=np.int32)
        rel = np.zeros(nrhs, dtype=np.float64)
        stat = np.zeros(nrhs, dtype=np.int32)
        hist = np.zeros((nrhs, max_iter + 1), dtype=np.float64)
        st = self.lib.iga_solve_multi(self.h, nrhs, _ptr(rhs), _ptr(out), use_x0, float(tol),
                                      int(max_iter), iters.ctypes.data_as(ctypes.c_void_p),
                                      hist.ctypes.data_as(ctypes.c_void_p),
                                      rel.ctypes.data_as(ctypes.c_void_p),
                                      stat.ctypes.data_as(ctypes.c_void_p))
        check(st, "iga_solve_multi", (STATUS_NO_CONVERGENCE,))
        return out.view(nrhs, self.N), dict(iters=iters, relres_true=rel, status=stat,
                                            hist=[hist[r, :iters[r] + 1].copy()
                                                  for r in range(nrhs)])

    def solve_async(self, rhs, out, tol=1e-8, max_iter=200):
        """Enqueue a solve of rhs (nrhs x N, device) into out; returns immediately."""
        nrhs = rhs.numel() // self.N
        check(self.lib.iga_solve_async(self.h, nrhs, _ptr(rhs), _ptr(out), 0, float(tol),
                                       int(max_iter)), "iga_solve_async")
        self._pending = (nrhs, max_iter)

    def ready(self):
        r = ctypes.c_int()
        check(self.lib.iga_solve_ready(self.h, ctypes.byref(r)), "iga_solve_ready")
        return bool(r.value)

    def test_set_device_error(self, code):
        """Test hook: set the handle's device error word from the host."""
        check(self.lib.iga_test_set_device_error(self.h, int(code)), "iga_test_set_device_error")

    def collect(self):
        nrhs, max_iter = self._pending
        iters = np.zeros(nrhs, dtype=np.int32)
        rel = np.zeros(nrhs, dtype=np.float64)
        stat = np.zeros(nrhs, dtype=np.int32)
        st = self.lib.iga_solve_collect(self.h, iters.ctypes.data_as(ctypes.c_void_p), None,
                                        rel.ctypes.data_as(ctypes.c_void_p),
                                        stat.ctypes.data_as(ctypes.c_void_p))
        check(st, "iga_solve_collect", (STATUS_NO_CONVERGENCE,))
        self._pending = None
        return dict(iters=iters, relres_true=rel, status=stat)


def solve_batched(problems, rhs, out, tol=1e-8, max_iter=200, history=False):
    """Batched form: problems[q] (distinct Problems, ideally on distinct streams),
    rhs[q] / out[q] device tensors (nrhs_q, N_q).  Returns per-rhs arrays
    (problem-major) of iterations, true relative residuals and statuses, and with
    ``history`` the residual estimates (sum(nrhs) x (max_iter + 1))."""
    lib = _lib.load()
    nprob = len(problems)
    H = (ctypes.c_void_p * nprob)(*[P.h.value for P in problems])
    nr = np.array([r.numel() // P.N for P, r in zip(problems, rhs)], dtype=np.int32)
    R = (ctypes.c_void_p * nprob)(*[r.data_ptr() for r in rhs])
    X = (ctypes.c_void_p * nprob)(*[x.data_ptr() for x in out])
    tot = int(nr.sum())
    iters = np.zeros(tot, dtype=np.int32)
    rel = np.zeros(tot, dtype=np.float64)
    stat = np.zeros(tot, dtype=np.int32)
    hist = np.zeros((tot, max_iter + 1), dtype=np.float64) if history else None
    st = lib.iga_solve_batched(nprob, H, nr.ctypes.data_as(ctypes.c_void_p), R, X, float(tol),
                               int(max_iter), iters.ctypes.data_as(ctypes.c_void_p),
                               hist.ctypes.data_as(ctypes.c_void_p) if history else None,
                               rel.ctypes.data_as(ctypes.c_void_p),
                               stat.ctypes.data_as(ctypes.c_void_p))
    check(st, "iga_solve_batched", (STATUS_NO_CONVERGENCE,))
    out = dict(iters=iters, relres_true=rel, status=stat, nrhs=nr)
    if history:
        out["hist"] = hist
    return out


def fp64_probe(kind=0, reps=1000, stream=None):
    """Enqueue one FP64 throughput probe launch (``iga_fp64_probe``: kind 0 = FP64
    mma.sync, 1 = FP64 FMAs, 2 = both on alternate warps, 3 = both in every warp) on
    ``stream`` and return its FLOP count; time it with CUDA events on the same stream."""
    lib = _lib.load()
    if stream is None:
        stream = torch.cuda.current_stream()
    fl = ctypes.c_double()
    check(lib.iga_fp64_probe(int(kind), int(reps), ctypes.c_void_p(stream.cuda_stream),
                             ctypes.byref(fl)), "iga_fp64_probe")
    return fl.value


def measure_fp64_peak(reps=1000, trials=5, stream=None, mixed=False):
    """FP64 ceiling of the current device in GFLOP/s: the best of ``trials`` timed launches
    of each probe kind (after one warm-up launch each).  Returns dict(dmma, fma, peak);
    ``mixed`` adds the two probes that run both paths at once (split, interleaved)."""
    if stream is None:
        stream = torch.cuda.current_stream()
    out = {}
    kinds = ((0, "dmma"), (1, "fma")) + (((2, "split"), (3, "interleaved")) if mixed else ())
    for kind, name in kinds:
        fp64_probe(kind, reps, stream)
        best = 0.0
        for _ in range(trials):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fl = fp64_probe(kind, reps, stream)
            e1.record(stream)
            e1.synchronize()
            best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        out[name] = best
    out["peak"] = max(out["dmma"], out["fma"])
    return out
