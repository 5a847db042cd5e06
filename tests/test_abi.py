"""The C ABI library loads and exports every function include/iga_fd.h declares;
argument validation runs on the host (no GPU needed for these calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared_functions():
    names = []
    for fname in sorted(os.listdir(HEADER_DIR)):
        if not fname.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fname)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\**\s*(iga_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_04384_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1705_04384_gb300 import build
        build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("iga_setup", "iga_precond_apply", "iga_solve", "iga_apply_operator",
                     "iga_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_prototypes_cover_header(lib):
    from paper_1705_04384_gb300 import _lib
    assert set(_declared_functions()) <= set(_lib.PROTOTYPES)


def test_status_strings(lib):
    for s in range(9):
        assert lib.iga_status_string(s)
    assert lib.iga_status_string(0) == b"ok"


def test_invalid_arguments_rejected_on_host(lib):
    from paper_1705_04384_gb300._lib import Geometry
    g = Geometry(1, 1.0, 2.0)
    h = ctypes.c_void_p()
    assert lib.iga_setup(4, 32, 3, ctypes.byref(g), 0, None, ctypes.byref(h)) == 1
    assert b"d must be" in lib.iga_last_error()
    assert lib.iga_setup(2, 32, 9, ctypes.byref(g), 0, None, ctypes.byref(h)) == 1
    assert lib.iga_setup(2, 2, 3, ctypes.byref(g), 0, None, ctypes.byref(h)) == 1
    bad = Geometry(1, 2.0, 1.0)
    assert lib.iga_setup(2, 32, 3, ctypes.byref(bad), 0, None, ctypes.byref(h)) == 1
    assert lib.iga_setup(2, 32, 3, ctypes.byref(g), 7, None, ctypes.byref(h)) == 1
    assert lib.iga_setup(2, 32, 3, ctypes.byref(g), 6, None, ctypes.byref(h)) == 1
    assert lib.iga_setup(2, 32, 3, ctypes.byref(g), -1, None, ctypes.byref(h)) == 1
    assert lib.iga_setup(2, 32, 3, None, 0, None, ctypes.byref(h)) == 1
    assert lib.iga_dims(None, None, None) == 1
    assert lib.iga_solve(None, None, None, 0, 1e-8, 10, None, None, None) == 1
    assert lib.iga_destroy(None) == 0
    assert lib.iga_set_grid_mode(None, 0) == 1
    assert b"null handle" in lib.iga_last_error()
    w = Geometry(1, 1.0, 2.0)
    w.wind[1] = float("inf")
    assert lib.iga_setup(2, 32, 3, ctypes.byref(w), 0, None, ctypes.byref(h)) == 1
    assert b"wind" in lib.iga_last_error()


def test_every_handle_entry_point_rejects_a_null_handle(lib):
    """Argument checks happen on the host before any device work (so they run here)."""
    null = None
    calls = [
        ("iga_collocation_points", (null, null)),
        ("iga_get_factor", (null, 0, 0, null)),
        ("iga_apply_operator", (null, null, null)),
        ("iga_precond_apply", (null, null, null)),
        ("iga_solve_host", (null, null, null, 1e-8, 10, None, null, None)),
        ("iga_solve_multi", (null, 1, null, null, 0, 1e-8, 10, null, null, null, null)),
        ("iga_solve_async", (null, 1, null, null, 0, 1e-8, 10)),
        ("iga_solve_ready", (null, None)),
        ("iga_solve_collect", (null, null, null, null, null)),
        ("iga_launch_counts", (null, None, None)),
        ("iga_fd_kernel", (null, 1, None)),
        ("iga_operator_flops", (null, None)),
        ("iga_prepare", (null, 1, 10)),
        ("iga_solve_bicgstab", (null, null, null, 0, 1e-8, 10, None, null, None)),
        ("iga_test_set_device_error", (null, 1)),
    ]
    for name, args in calls:
        assert getattr(lib, name)(*args) == 1, name  # IGA_ERR_INVALID_ARG
        assert lib.iga_last_error(), name


def test_batch_and_noalloc_argument_checks(lib):
    assert lib.iga_solve_batched(0, None, None, None, None, 1e-8, 10, None, None, None,
                                 None) == 1
    assert b"batch" in lib.iga_last_error()
    # d outside 2..3, then a null factor pointer
    assert lib.iga_precond_apply_noalloc(4, 10, None, None, None, None, None, None) == 1
    assert lib.iga_precond_apply_noalloc(3, 10, None, None, None, None, None, None) == 1


def test_fp64_probe_argument_checks(lib):
    assert lib.iga_fp64_probe(4, 10, None, None) == 1
    assert lib.iga_fp64_probe(-1, 10, None, None) == 1
    assert lib.iga_fp64_probe(0, 0, None, None) == 1
    assert b"reps" in lib.iga_last_error()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback of any kind: without libiga_fd.so the binding raises and names the build."""
    from paper_1705_04384_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libiga_fd.so"))
    with pytest.raises(ImportError, match="build"):
        _lib.load()
    from paper_1705_04384_gb300.api import Problem
    with pytest.raises(ImportError, match="missing"):
        Problem(2, 8, 3)
