"""ctypes loader for ``libiga_fd.so`` (the C ABI of include/iga_fd.h).

There is no fallback: if the shared library is missing, importing the binding
raises, naming the build command.
"""

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libiga_fd.so")

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int_p = ctypes.POINTER(ctypes.c_int)
c_ll_p = ctypes.POINTER(ctypes.c_longlong)


class Geometry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("r_inner", ctypes.c_double), ("r_outer", ctypes.c_double),
                ("wind", ctypes.c_double * 3)]


# name -> (restype, argtypes); mirrors include/iga_fd.h
PROTOTYPES = {
    "iga_setup": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Geometry),
                                 ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "iga_setup_scheme": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(Geometry), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "iga_dims": (ctypes.c_int, [ctypes.c_void_p, c_int_p, c_ll_p]),
    "iga_quadrature_dims": (ctypes.c_int, [ctypes.c_void_p, c_int_p, c_ll_p]),
    "iga_quadrature_points": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "iga_wq_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "iga_collocation_points": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "iga_get_factor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "iga_apply_operator": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "iga_precond_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "iga_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_int, c_int_p, ctypes.c_void_p, c_double_p]),
    "iga_solve_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_double, ctypes.c_int, c_int_p, ctypes.c_void_p,
                                      c_double_p]),
    "iga_solve_multi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "iga_solve_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int]),
    "iga_solve_ready": (ctypes.c_int, [ctypes.c_void_p, c_int_p]),
    "iga_solve_collect": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "iga_solve_batched": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "iga_test_set_device_error": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "iga_launch_counts": (ctypes.c_int, [ctypes.c_void_p, c_int_p, c_int_p]),
    "iga_fd_kernel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_int_p]),
    "iga_operator_flops": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "iga_prepare": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "iga_set_grid_mode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "iga_solve_bicgstab": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int, c_int_p,
                                          ctypes.c_void_p, c_double_p]),
    "iga_precond_apply_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p]),
    "iga_fp64_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, c_double_p]),
    "iga_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "iga_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "iga_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load():
    """Load the library once and attach the prototypes."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` "
                          "or `python -m paper_1705_04384_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class IgaError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.iga_status_string(status).decode()
        detail = lib.iga_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")
        self.status = status


def check(status, where, allow=()):
    if status != 0 and status not in allow:
        raise IgaError(status, where)
    return status
