"""Build the in-tree shared library ``libiga_fd.so`` for sm_103a with nvcc.

Each translation unit under ``csrc/`` is compiled in parallel, then linked with
the CUDA runtime and cuSOLVER.  Usage: ``python -m paper_1705_04384_gb300.build``.
"""

import os
import shutil
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libiga_fd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home():
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.exists(os.path.join(home, "bin", "nvcc")):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cpp")))


def _compile(nvcc, src, extra):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc, "-c", src, "-o", obj, "-O3", "-std=c++17", "-lineinfo", *ARCH,
           "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills",
           *extra]
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, res


def build(verbose=False, extra=()):
    """Compile every source and link ``libiga_fd.so``; returns its path."""
    t0 = time.time()
    home = _cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(nvcc, s, list(extra)), srcs))
    failed = [r for r in results if r[2].returncode != 0]
    for src, _, res in results:
        if verbose or res.returncode != 0:
            if res.stdout.strip() or res.stderr.strip():
                sys.stderr.write(f"--- {os.path.basename(src)}\n{res.stdout}{res.stderr}\n")
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(os.path.basename(r[0]) for r in failed))
    objs = [r[1] for r in results]
    libdir = os.path.join(home, "lib64")
    tmp = LIB + ".tmp"
    link = [nvcc, "-shared", "-o", tmp, *objs, *ARCH, "-cudart", "shared",
            "-L" + libdir, "-lcusolver", "-Xlinker", "-rpath," + libdir]
    res = subprocess.run(link, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n" + res.stdout + res.stderr)
    os.replace(tmp, LIB)
    if verbose:
        sys.stderr.write(f"built {LIB} in {time.time() - t0:.1f} s\n")
    return LIB


if __name__ == "__main__":
    build(verbose=True)
