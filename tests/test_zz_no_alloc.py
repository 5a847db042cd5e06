"""iga_precond_apply_noalloc: the FD solve for callers that cannot allocate device
memory when they apply the preconditioner (a budget reserved up front, an
allocator-free real-time loop, a host whose allocator owns the device).  Its scratch
is a static device array inside the library; these tests call it through the C ABI
and compare it with iga_precond_apply on two calls in a row.

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


@pytest.mark.parametrize("d,ne,p", [(2, 40, 3), (3, 12, 4), (3, 64, 3)])
def test_noalloc_fd_matches_precond_apply_twice(d, ne, p):
    from paper_1705_04384_gb300.api import Problem
    with Problem(d, ne, p) as P:
        lib = P.lib
        Vt = torch.from_numpy(P.factor("Vt")).cuda()
        U = torch.from_numpy(P.factor("U")).cuda()
        lam = torch.from_numpy(P.factor("lambda")).cuda()
        stream = torch.cuda.current_stream()
        g = torch.Generator().manual_seed(d * 100 + ne)
        for call in range(2):
            b = torch.randn(P.N, dtype=torch.float64, generator=g).cuda()
            ref = P.precond_apply(b)
            out = torch.full_like(b, float("nan"))
            st = lib.iga_precond_apply_noalloc(d, P.n, _ptr(Vt), _ptr(U), _ptr(lam), _ptr(b),
                                               _ptr(out), ctypes.c_void_p(stream.cuda_stream))
            assert st == 0, lib.iga_last_error()
            torch.cuda.synchronize()
            err = torch.linalg.norm(out - ref).item() / torch.linalg.norm(ref).item()
            assert err <= TOL, (call, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1705_04384_gb300 import _lib
    lib = _lib.load()
    dummy = ctypes.c_void_p(16)
    n = 129  # 129^3 > 2^21
    st = lib.iga_precond_apply_noalloc(3, n, dummy, dummy, dummy, dummy, dummy, None)
    assert st == 1
    assert b"exceeds" in lib.iga_last_error()
