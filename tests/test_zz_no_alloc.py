"""iga_precond_apply_noalloc: the FP64 FD solve for callers that cannot allocate device
memory when they apply the preconditioner (a budget reserved up front, an allocator-free
real-time loop, a host whose allocator owns the device).  Its scratch is a static device
array inside the library; these tests call it through the C ABI, two calls in a row per
case, and compare it with

* the CPU oracle's FD solve (oracle/fd.py, eq. FD2D / FD3D),
* a dense solve of the assembled preconditioner P (eq. colloc2D / colloc3D) at tiny n,
* the library's own iga_precond_apply on the same handle,

including a convection-diffusion handle whose three directions have different winds, so
that each direction's own eigen-factors are needed (Sec. 3.2).

The file name sorts last so that a run stopping at the first failure has already run
every other test.
"""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-11  # same bound as the FD parity tests


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stacked_factors(P):
    """Direction-stacked V^T, U and eigenvalues of every direction of a handle."""
    Vt = np.stack([P.factor("Vt", l) for l in range(P.d)])
    U = np.stack([P.factor("U", l) for l in range(P.d)])
    lam = np.stack([P.factor("lambda", l) for l in range(P.d)])
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (Vt, U, lam)]


def _noalloc(lib, P, fac, b):
    Vt, U, lam = fac
    out = torch.full_like(b, float("nan"))
    stream = torch.cuda.current_stream()
    st = lib.iga_precond_apply_noalloc(P.d, P.n, _ptr(Vt), _ptr(U), _ptr(lam), _ptr(b),
                                       _ptr(out), ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.iga_last_error()
    torch.cuda.synchronize()
    return out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [(2, 40, 3, None), (3, 12, 4, None), (3, 64, 3, None),
         (3, 10, 3, (4.0, -2.5, 1.0)), (2, 24, 5, (3.0, 0.5))]


@pytest.mark.parametrize("d,ne,p,wind", CASES)
def test_noalloc_fd_matches_oracle_and_precond_apply(d, ne, p, wind):
    from paper_1705_04384_gb300.api import Problem
    from tests.oracle_ref import ref
    R = ref(d, ne, p, assemble=False, wind=wind)
    with Problem(d, ne, p, precision="fp64", wind=wind) as P:
        fac = _stacked_factors(P)
        g = np.random.default_rng(d * 1000 + ne)
        for call in range(2):
            b_np = g.standard_normal(P.N)
            b = torch.from_numpy(b_np).cuda()
            out = _noalloc(P.lib, P, fac, b).cpu().numpy()
            lib_out = P.precond_apply(b).cpu().numpy()
            assert _rel(out, lib_out) <= TOL, (call, "iga_precond_apply")
            assert _rel(out, R.fd(b_np)) <= TOL, (call, "oracle FD")


@pytest.mark.parametrize("d,ne,p,wind", [(2, 8, 3, None), (3, 5, 3, None),
                                         (3, 5, 4, (2.0, -1.0, 3.0))])
def test_noalloc_fd_matches_dense_kronecker_solve(d, ne, p, wind):
    from oracle import collocation as C
    from paper_1705_04384_gb300.api import Problem
    from tests.oracle_ref import ref
    R = ref(d, ne, p, assemble=False, wind=wind)
    Pmat = C.assemble_preconditioner(R.spaces, wind).toarray()
    with Problem(d, ne, p, precision="fp64", wind=wind) as P:
        fac = _stacked_factors(P)
        g = np.random.default_rng(7)
        for call in range(2):
            b_np = g.standard_normal(P.N)
            out = _noalloc(P.lib, P, fac, torch.from_numpy(b_np).cuda()).cpu().numpy()
            assert _rel(out, np.linalg.solve(Pmat, b_np)) <= TOL, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1705_04384_gb300 import _lib
    lib = _lib.load()
    dummy = ctypes.c_void_p(16)
    # 129^3 > 2^21; 2^22 would wrap to N = 0 in 64 bits if multiplied unchecked (d = 3)
    for d, n in ((3, 129), (3, 1 << 22), (2, 1449), (2, 1 << 30)):
        st = lib.iga_precond_apply_noalloc(d, n, dummy, dummy, dummy, dummy, dummy, None)
        assert st == 1, (d, n)
        assert b"exceeds" in lib.iga_last_error()
