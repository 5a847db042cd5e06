"""Benchmark: GMRES + FD time-to-1e-8 and DOF-iterations per second on one GB300.

Workload (default): the 3D extruded thick quarter annulus r in [1,2], z in [0,1],
128 elements per direction, p = 4, 5, 6 (N = 2,197,000 / 2,248,091 / 2,299,968), forcing
from the manufactured solution plus the seeded 1e-3 perturbation, GMRES tol 1e-8.  One
step = one solve for each p (setup cached).  Four forms of the same solves:
  fp64    plain GMRES with the FP64 FD (the line's value),
  tf32    flexible GMRES with the FD mode products on the tensor cores in TF32 ("mixed"),
  tf32x3  the same with error-compensated TF32 (hi/lo operand split, three MMAs per step;
          "tf32x3"),
  fp64tc  plain GMRES with the FP64 FD on the BF16 tensor cores by exact integer slice
          products (FP64-accurate; "fp64tc"),
  bf16    the same with BF16 operands ("bf16"),
each with per-solve p50/p99, time to solution with and without setup, the error against
the FP64 oracle's solution (p = 4) and the roofline of its dominant kernel.  The FP64
ceiling is measured in the same run (iga_fp64_probe).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas (the
path does not shard); value = all ranks' DOF-iterations / max time over ranks.
"""

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workload as W  # noqa: E402

METRIC = "GMRES+FD time-to-1e-8 residual, DOF-iter/s (mixed vs FP64, 1 GB300); p50/p99"
UNIT = "DOF-iter/s"
WORKLOAD = "3d_annulus_ne128"
TOL = 1e-8
MAX_ITER = 200
ORACLE_P = 4  # degree of the problem the oracle solves in full (error reference, CPU baseline)
HBM_PEAK_FALLBACK = 6800.0  # GB/s, used only when MEASURED_PEAKS.json is absent
TEXTS = {
    "3d_annulus_ne128": "3d_annulus_ne128: 3D extruded quarter annulus r in [1,2], z in [0,1], 128 "
                        "elements/dir, p=4,5,6 (N=2197000/2248091/2299968), manufactured f + seeded "
                        "1e-3 perturbation, FD-GMRES to 1e-8 in FP64 (value), TF32 and BF16 "
                        "(flexible GMRES, FD on the tensor cores)",
    "3d_annulus_ne64": "3d_annulus_ne64: 3D extruded quarter annulus r in [1,2], z in [0,1], 64 "
                       "elements/dir, p=3,4,5 (N=274625/287496/300763), manufactured f + seeded "
                       "1e-3 perturbation, FD-GMRES to 1e-8",
    "3d_revolved_ne64": "3d_revolved_ne64: 3D quarter ring r in [1,2] revolved by pi/2 about the "
                        "axis (0,1,0) through (-1,-1,-1), 64 elements/dir, p=3,4,5, f = 1 + seeded "
                        "1e-3 perturbation, FD-GMRES to 1e-8",
    "3d_wind_ne64": "3d_wind_ne64: convection-diffusion -Lap + w.grad (Sec. 3.2) with w = (5,5,5) "
                    "on the 3D extruded quarter annulus, 64 elements/dir, p=3,4,5, f = 1 + seeded "
                    "1e-3 perturbation, FD of the wind-shifted pencils, FP64 FD-GMRES to 1e-8",
    "3d_wq_revolved_ne64": "3d_wq_revolved_ne64: weighted-quadrature Galerkin (Sec. 2.3) on the 3D "
                           "quarter ring revolved by pi/2 (Sec. 5), 64 elements/dir, p=3,4,5, WQ "
                           "load of f = 1 + seeded 1e-3 perturbation, FD of the Galerkin pencils "
                           "(P_wq), FD-GMRES to 1e-8 in FP64 (value), TF32 and BF16",
}
CONFIG = {"workload": TEXTS[WORKLOAD],
          "step": "one solve per p (setup cached); per form",
          "l2": "flushed between steps (512 MB write); inputs (17.6-18.4 MB per vector, Krylov "
                "bases of 0.4-0.9 GB) exceed L2 anyway",
          "parallelism": "replicas"}


def geometry_of(c):
    return c.get("geometry", "annulus")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="FP64 form only")
    ap.add_argument("--no-bicgstab", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 3d_annulus_ne64 secondary line (3D annulus, 64 elements)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-form key of the default line")
    ap.add_argument("--workload", default="3d_ne128",
                    choices=["3d_ne128", "3d_ne64", "3d_revolved_ne64", "3d_wind_ne64",
                             "3d_wq_revolved_ne64", "batched", "served"],
                    help="3d_ne128 (default bench line), 3d_ne64 (64 elements), 3d_revolved_ne64 "
                         "(Sec. 5's revolved ring), 3d_wind_ne64 (Sec. 3.2 convection-diffusion), "
                         "batched (256 2D problems x 8 rhs), served (Poisson request stream)")
    ap.add_argument("--precision", default="tf32", help="preconditioner precision for the "
                                                        "batched / served forms")
    ap.add_argument("--count", type=int, default=256, help="problems in the batched form")
    ap.add_argument("--rate", type=float, default=2000.0, help="offered load, requests/s")
    ap.add_argument("--window", type=float, default=10.0, help="served arrival window, s")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


# ------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------- helpers
def kernel_source_hash(files=("kernels_fd64.cu",)):
    """Hash of a kernel's source file(s) with comments and blank space removed, so that an
    edit of comments does not void the committed counters."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1705_04384_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def committed_traffic(summary="fd_fold_mma_3d_ne128.md", files=("kernels_fd64.cu",)):
    """dram bytes per launch of a kernel from its committed ncu summary, or None when the
    kernel source changed since the capture (or there is no summary)."""
    path = os.path.join(ROOT, "profiles", summary)
    vals = {}
    try:
        with open(path) as fh:
            for line in fh:
                if ":" in line and line.strip().split(":")[0] in (
                        "kernel_source_sha256_16", "traffic_bytes_per_launch"):
                    k, v = line.strip().split(":", 1)
                    vals[k] = v.strip()
    except OSError:
        return None
    if vals.get("kernel_source_sha256_16") != kernel_source_hash(files):
        return None
    return float(vals["traffic_bytes_per_launch"]) if "traffic_bytes_per_launch" in vals else None


def f64tc_issued_flops(n, d):
    """BF16 MMA FLOPs one FD apply of the FP64_TC form issues (kernels_fd_f64tc.cu's tiling:
    128-row tiles, 64-column tiles when the factor's 8 slices leave room for a 2-stage ring,
    else 32, every column tile at full width; 36 slice pairs per 16-wide K-step;
    2 x 128 x N x 16 per MMA)."""
    nchunks = (n + 63) // 64
    budget = 225 * 1024
    nt = 64 if budget - 8 * nchunks * 64 * 128 >= 2 * 128 * 128 else 32
    width = (n + nt - 1) // nt * nt
    ksteps = sum(min(4, (n - 64 * c + 15) // 16) for c in range(nchunks))
    row_tiles = (n ** (d - 1) + 127) // 128
    return 2.0 * d * row_tiles * 36 * ksteps * 2 * 128 * 16 * width


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def aggregate(units, seconds, device=None):
    """Replicas: the units (DOF-iterations) all ranks processed and the longest time any
    rank took (sum and max over the process group when one is initialised)."""
    try:
        import torch.distributed as dist
        active = dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1
    except ImportError:
        active = False
    if not active:
        return float(units), float(seconds)
    import torch
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def percentile(vals, q):
    return float(np.percentile(np.asarray(vals, dtype=np.float64), q)) if vals else None


def fold_flops_per_launch(n, d=3):
    """Algorithmic FLOPs of one folded FP64 FD mode product, averaged over the d forward
    (even block ne x ne, odd block no x no) and d inverse (ne pairs x n) launches."""
    ne, no = (n + 1) // 2, n // 2
    rows = n ** (d - 1)
    return 0.5 * (2.0 * rows * (ne * ne + no * no) + 2.0 * rows * ne * n)


def operator_flops_per_dof(W_band, d=3):
    """Algorithmic FLOPs per DOF of the operator on the extruded annulus (fields 11, 22, 33
    and the first-order term 1): 2 band passes along direction 3, 3 along direction 2 and 4
    band passes contracted along direction 1, each 2W FLOPs, plus 2 per contracted term."""
    assert d == 3
    return 2.0 * W_band * (2 + 3 + 4) + 2.0 * 4


# ------------------------------------------------------------------------- oracle (CPU)
def oracle_problem(name, p):
    """The oracle's view of one problem of a named 3D workload: spaces, matrix-free A_C
    (the definition of eq. collocation applied through the Kronecker identity: the CSR
    matrix of the 128-element 3D annulus has about 8e8 non-zeros), the FD preconditioner and the rhs; for the
    WQ workload the matrix-free A_wq (eq. WQapprox), the FD of P_wq and the WQ load."""
    from oracle import collocation as C, fd as F, geometry as Geo
    c = W.CONFIGS[name]
    if c.get("scheme") == "wq":
        from oracle import wq as Q
        spaces = [Q.WQSpace1D(c["n_elem"], p) for _ in range(c["d"])]
        fmap = Geo.make_map(geometry_of(c), c["d"], c["r0"], c["r1"])
        nq = int(np.prod([s.nq for s in spaces]))
        f = Q.wq_load(spaces, fmap, np.ones(nq))
        b = W.perturb(f, c["sigma"], c["seed"] + c["ps"].index(p))
        return Q.WQOperator(spaces, fmap), F.FD(spaces), b
    spaces = [C.Space1D(c["n_elem"], p) for _ in range(c["d"])]
    fmap = Geo.make_map(geometry_of(c), c["d"], c["r0"], c["r1"])
    A = C.CollocationOperator(spaces, fmap, c.get("wind"))
    pts = C.physical_points_grid(fmap, [s.tau for s in spaces])
    b = W.config_rhs(name, pts, c["ps"].index(p))
    fd = F.FD(spaces, c.get("wind"))
    return A, fd, b


def oracle_solve(name=None, p=ORACLE_P):
    """One full oracle GMRES+FD solve to 1e-8 (iteration phase timed) on the host cores."""
    from oracle import gmres as G
    name = name or WORKLOAD
    t0 = time.perf_counter()
    A, fd, b = oracle_problem(name, p)
    setup = time.perf_counter() - t0
    t0, c0 = time.perf_counter(), time.process_time()
    r = G.gmres(A, b, M=fd, tol=TOL, max_iter=MAX_ITER)
    dt, dc = time.perf_counter() - t0, time.process_time() - c0
    return dict(x=r["x"], iters=r["iters"], relres_true=r["relres_true"], seconds=dt,
                cpu_seconds=dc, setup_s=setup, N=b.shape[0], hist_last=float(r["hist"][-1]))


def run_reference(args):
    """The oracle timed on the host cores, one bounded sample of the workload per step:
    REF_ITERS GMRES+FD iterations of the p = ORACLE_P problem (Arnoldi by modified
    Gram-Schmidt, the FD solve of eq. FD3D, the matrix-free A_C)."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    from oracle import gmres as G
    A, fd, b = oracle_problem(WORKLOAD, ORACLE_P)
    N = b.shape[0]
    ref_iters = 3
    times, cpu_s, dofit = [], 0.0, 0
    r = None
    for it in range(args.warmup + args.steps):
        t0, c0 = time.perf_counter(), time.process_time()
        r = G.gmres(A, b, M=fd, tol=0.0, max_iter=ref_iters)
        dt, dc = time.perf_counter() - t0, time.process_time() - c0
        if it >= args.warmup:
            times.append(dt)
            cpu_s += dc
            dofit += N * r["iters"]
    tot = sum(times)
    value = dofit / tot
    cores = os.cpu_count()
    sample = (f"oracle GMRES+FD, {ref_iters} Arnoldi iterations per step of the p={ORACLE_P} "
              f"problem of {WORKLOAD} (N={N}), x0 = 0, matrix-free A_C (eq. collocation via the "
              f"Kronecker identity), FD of eq. FD3D, modified Gram-Schmidt; iteration phase only "
              f"(fields and eigendecomposition are setup)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": CONFIG,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "busy_cores": cpu_s / tot},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "last_relres_est": float(r["hist"][-1])}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1705_04384_gb300.api import Problem, measure_fp64_peak

    c = W.CONFIGS[WORKLOAD]
    d = c["d"]
    oracle_p = ORACLE_P if ORACLE_P in c["ps"] else c["ps"][0]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", HBM_PEAK_FALLBACK)
    hbm_note = "of measured" if "hbm_gbs" in peaks else "of fallback"

    # the FP64 ceiling of this GPU, measured now (iga_fp64_probe, best of 5 launches each)
    # and again right before the rooflines (GPU warm, after the timed solves); the best of
    # the two is the peak: a probe that ran while the clocks were still ramping up reads low
    fp64 = measure_fp64_peak(reps=1000, trials=5, stream=stream)
    fp64_peak = fp64["peak"]

    def make(prec):
        """Set up one problem per degree; setup time = iga_setup + iga_prepare (workspace and
        solve-graph capture), time to solution with setup = that + the first solve."""
        probs = []
        for i, p in enumerate(c["ps"]):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            P = Problem(d, c["n_elem"], p, geometry_of(c), c["r0"], c["r1"], precision=prec,
                        wind=c.get("wind"), device=dev, stream=stream,
                        scheme=c.get("scheme", "collocation"))
            P.prepare(1, MAX_ITER)
            torch.cuda.synchronize(dev)
            t_setup = time.perf_counter() - t0
            if c.get("scheme") == "wq":
                _, Nq = P.quadrature_dims()
                f = P.wq_load(torch.ones(Nq, dtype=torch.float64, device=dev)).cpu().numpy()
                rhs = torch.from_numpy(W.perturb(f, c["sigma"], c["seed"] + i)).to(dev)
            else:
                pts = P.collocation_points()
                rhs = torch.from_numpy(W.config_rhs(WORKLOAD, pts, i)).to(dev)
            x = torch.empty_like(rhs)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            _, info = P.solve(rhs, tol=TOL, max_iter=MAX_ITER, out=x)
            t_first = time.perf_counter() - t0
            probs.append(dict(p=p, P=P, rhs=rhs, x=x, setup_s=t_setup, first_s=t_first))
        return probs

    def run_step(probs, solver="gmres"):
        per = []
        for q in probs:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if solver == "gmres":
                _, info = q["P"].solve(q["rhs"], tol=TOL, max_iter=MAX_ITER, out=q["x"])
            else:
                _, info = q["P"].solve_bicgstab(q["rhs"], tol=TOL, max_iter=MAX_ITER, out=q["x"])
            e1.record(stream)
            per.append((q, info, e0, e1))
        torch.cuda.synchronize(dev)
        return [(q["p"], q["P"].N, info["iters"], e0.elapsed_time(e1) * 1e-3, info["relres_true"])
                for q, info, e0, e1 in per]

    def timed(probs, steps, warmup, solver="gmres"):
        for _ in range(warmup):
            run_step(probs, solver)
        results = []
        for _ in range(steps):
            flush.fill_(1.0)  # L2 flush between steps, outside the timed solves
            torch.cuda.synchronize(dev)
            results.append(run_step(probs, solver))
        return results

    def summarise(probs, res):
        t = sum(sum(s[3] for s in step) for step in res)
        u = sum(sum(s[1] * s[2] for s in step) for step in res)
        units, tt = aggregate(u, t, dev)
        solve_ms = [s[3] * 1e3 for st in res for s in st]
        by_p = {}
        for q in probs:
            ms = [s[3] * 1e3 for st in res for s in st if s[0] == q["p"]]
            by_p[str(q["p"])] = {"p50_ms": percentile(ms, 50), "p99_ms": percentile(ms, 99),
                                 "setup_ms": 1e3 * q["setup_s"],
                                 "tts_with_setup_ms": 1e3 * (q["setup_s"] + q["first_s"])}
        p50 = percentile(solve_ms, 50)
        return {"value": units / tt, "unit": UNIT,
                "iters": {str(s[0]): s[2] for s in res[-1]},
                "relres_true": {str(s[0]): s[4] for s in res[-1]},
                "p50_ms": p50, "p99_ms": percentile(solve_ms, 99), "max_ms": max(solve_ms),
                "solves": len(solve_ms),
                "solves_over_1p5x_p50": sum(1 for t in solve_ms if t > 1.5 * p50),
                "tts_warm_ms_per_step": 1e3 * tt / len(res), "by_p": by_p,
                "_units": units, "_t": tt}

    def launches_of(probs, res):
        tot = 0
        for step in res:
            for q, s in zip(probs, step):
                f, it = q["P"].launch_counts()
                tot += f + it * s[2]
        return tot

    def time_calls(fn, reps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) * 1e-3 / reps

    forms = ["fp64"] if args.no_mixed else ["fp64", "tf32", "tf32x3", "bf16", "fp64tc"]
    probs = {f: make(f) for f in forms}

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local_rank)
    clocks.start()
    res = {f: timed(probs[f], args.steps, args.warmup) for f in forms}
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    out = {f: summarise(probs[f], res[f]) for f in forms}
    for f in forms:
        out[f]["gpu_launches"] = launches_of(probs[f], res[f])
    main = out["fp64"]

    fp64_late = measure_fp64_peak(reps=1000, trials=5, stream=stream)
    fp64 = {k: max(fp64[k], fp64_late[k]) for k in fp64}
    fp64_peak = fp64["peak"]

    # dominant kernels, timed live on the bench stream (the p = ORACLE_P problem, n = 130)
    q4 = {f: next(q for q in probs[f] if q["p"] == oracle_p) for f in forms}
    P4 = q4["fp64"]["P"]
    n4, N4 = P4.n, P4.N
    buf = torch.empty_like(q4["fp64"]["rhs"])
    # FP64 form: the folded FD mode product (6 launches per FD apply)
    t_launch = time_calls(lambda: P4.precond_apply(q4["fp64"]["rhs"], out=buf), 10) / (2 * d)
    fl = fold_flops_per_launch(n4, d)
    fd_kind = P4.fd_kernel(1)
    if fd_kind == "fold_fma":
        fd_prof = ("fd_fold_fma_3d_ne128.md", ("kernels_fd64_fma.cu",),
                   "fd_fold_fma_kernel (folded FD mode product, FP64 FMAs)")
    elif fd_kind == "dense_mma":
        # pencils without reflection parity (a wind): dense products, 2 n^{d+1} FLOPs each
        fl = 2.0 * n4 ** (d + 1)
        fd_prof = ("fd_fold_mma_3d_ne128.md", ("kernels_fd64.cu",),
                   "fd_fold_mma_kernel, dense mode (FD mode product without parity, FP64 "
                   "mma.sync m8n8k4)")
    else:
        fd_prof = ("fd_fold_mma_3d_ne128.md", ("kernels_fd64.cu",),
                   "fd_fold_mma_kernel (folded FD mode product, FP64 mma.sync m8n8k4)")
    main["roofline"] = {
        "bound": "alu", "achieved": fl / t_launch / 1e9, "peak": fp64_peak, "unit": "GFLOP/s",
        "frac": fl / t_launch / 1e9 / fp64_peak,
        # the committed counters are of the 128-element 3D annulus (n = 130): other sizes have none
        "traffic": (committed_traffic(fd_prof[0], fd_prof[1])
                    if WORKLOAD == "3d_annulus_ne128" and n4 == 130 else None),
        "kernel": fd_prof[2],
        "per_launch_us": t_launch * 1e6, "flops_per_launch": fl,
        "dense_equivalent_flops_per_launch": 2.0 * n4 ** (d + 1),
        "peak_note": f"of measured: FP64 ceiling of this GPU measured in this run by "
                     f"iga_fp64_probe (mma.sync .f64 {fp64['dmma']:.0f}, FP64 FMA "
                     f"{fp64['fma']:.0f} GFLOP/s, each the best of a measurement before and "
                     f"one after the timed region; the larger is the peak)"}
    # operator (FP64 unit), the same in every form
    t_op = time_calls(lambda: P4.apply_operator(q4["fp64"]["rhs"], out=buf), 10)
    opf = P4.operator_flops()  # counted from the handle's pass plan (iga_operator_flops)
    wq = c.get("scheme") == "wq"
    main["roofline_operator"] = {
        "bound": "alu", "achieved": opf / t_op / 1e9, "peak": fp64_peak, "unit": "GFLOP/s",
        "frac": opf / t_op / 1e9 / fp64_peak,
        "kernel": (f"{2 * d} x wq_pass_kernel (expansion onto the quadrature grid and "
                   f"contraction by the WQ rules, one operator application)" if wq else
                   "band_pass + band_pass_multi + contract_pass (one operator application, "
                   "3 launches)"),
        "per_apply_us": t_op * 1e6, "flops_per_apply": opf}
    # precision forms: one FD apply (pack + 2d tensor-core mode products), graded against
    # the fused three-pass HBM floor of the FD (3 x 8 bytes per DOF)
    for f in forms[1:]:
        Pf = q4[f]["P"]
        t_fd = time_calls(lambda: Pf.precond_apply(q4[f]["rhs"], out=buf), 20)
        if f == "fp64tc":
            fl_issued = f64tc_issued_flops(n4, d)
            bf16_peak = peaks.get("bf16_tflops", 1900.0)
            out[f]["roofline"] = {
                "bound": "tensor", "achieved": fl_issued / t_fd / 1e12, "peak": bf16_peak,
                "unit": "TFLOP/s", "frac": fl_issued / t_fd / 1e12 / bf16_peak, "traffic": None,
                "kernel": "2d x (f64tc_split_kernel + f64tc_gemm_kernel) (one FD apply: BF16 "
                          "digit-slice products, 36 slice pairs per K-step)",
                "per_apply_us": t_fd * 1e6, "issued_flops_per_apply": fl_issued,
                "fp64_equivalent_tflops": 2.0 * d * 2.0 * n4 ** (d + 1) / t_fd / 1e12,
                "peak_note": ("of measured" if "bf16_tflops" in peaks else "of fallback") +
                             " dense BF16 (cuBLAS, burst); achieved = BF16 MMA FLOPs issued "
                             "(zero-padded K-steps and column tiles included); "
                             "fp64_equivalent_tflops = the dense FD's 2d x 2 n^(d+1) FP64 "
                             "FLOPs per apply over the same time"}
            continue
        by = 24.0 * N4
        tfl = 2.0 * d * 2.0 * n4 ** (d + 1)
        out[f]["roofline"] = {
            "bound": "hbm", "achieved": by / t_fd / 1e9, "peak": hbm_peak, "unit": "GB/s",
            "frac": by / t_fd / 1e9 / hbm_peak, "traffic": None,
            "kernel": "pack_kernel + 6 x tc_gemm_kernel (one FD apply, tcgen05 " + f + ")",
            "per_apply_us": t_fd * 1e6, "bytes_per_apply": by,
            "tensor_tflops": tfl / t_fd / 1e12,
            # error-compensated TF32 issues three MMAs per useful product
            "tensor_tflops_issued": (3 if f == "tf32x3" else 1) * tfl / t_fd / 1e12,
            "peak_note": hbm_note + " HBM copy bandwidth; bytes = the fused three-pass FD "
                         "floor (3 x 8 B/DOF)"}

    # end to end through the host-buffer entry point (FP64 form)
    e2e_times, e2e_dofit, h2d, d2h = [], 0, 0, 0
    host = []
    for q in probs["fp64"]:
        hr = torch.empty(q["P"].N, dtype=torch.float64, pin_memory=True)
        hr.copy_(q["rhs"].cpu())
        hx = torch.empty(q["P"].N, dtype=torch.float64, pin_memory=True)
        host.append((q["P"], hr, hx))
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        its = 0
        for P, hr, hx in host:
            info = P.solve_host(hr, hx, tol=TOL, max_iter=MAX_ITER)
            its += P.N * info["iters"]
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            e2e_times.append(dt)
            e2e_dofit += its
    for P, hr, hx in host:
        h2d += P.N * 8
        d2h += P.N * 8 + (MAX_ITER + 1) * 8 + 64
    eu, et = aggregate(e2e_dofit, sum(e2e_times), dev)
    e2e = {"value": eu / et, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # precision forms against the FP64 form's solution of the same right-hand side
    for f in forms[1:]:
        out[f]["rel_err_vs_fp64"] = {
            str(qa["p"]): float(torch.linalg.vector_norm(qb["x"] - qa["x"]) /
                                torch.linalg.vector_norm(qa["x"]))
            for qa, qb in zip(probs["fp64"], probs[f])}
        out[f]["speedup_vs_fp64_tts_warm"] = (main["tts_warm_ms_per_step"] /
                                              out[f]["tts_warm_ms_per_step"])

    # the GMRES solutions of the p = oracle_p problems, before the BiCGStab line reuses the
    # FP64 problems' solution buffers
    x4 = {f: q4[f]["x"].double().cpu().numpy() for f in forms}

    # Sec. 5's solver on the same problems: BiCGStab + FP64 FD, counted in halves
    bicg_out = None
    if not args.no_bicgstab:
        resb = timed(probs["fp64"], max(1, args.steps // 4), 1, "bicgstab")
        bs = summarise(probs["fp64"], resb)
        bicg_out = {"value": bs["value"], "unit": "DOF-iter/s (BiCGStab iterations)",
                    "iters": bs["iters"], "relres_true": bs["relres_true"],
                    "p50_ms": bs["p50_ms"], "tts_warm_ms_per_step": bs["tts_warm_ms_per_step"]}

    for f in forms:
        for q in probs[f]:
            q["P"].close()
    probs = None

    # the 64-element 3D annulus (3d_annulus_ne64, FP64 and TF32), a secondary key
    secondary = None
    if not args.no_secondary:
        secondary = run_secondary(args, dev, stream, flush)

    batched = None
    if not args.no_batched and world == 1:
        batched = run_batched(args, steps=3, warmup=1, emit=False)

    if rank != 0:
        return 0
    cpu = None
    oracle_err = None
    if world == 1 and not args.no_cpu_baseline:
        o = oracle_solve(WORKLOAD, oracle_p)
        cpu = {"value": o["N"] * o["iters"] / o["seconds"], "unit": UNIT,
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one full oracle GMRES+FD solve to 1e-8 of the p={oracle_p} problem of "
                         f"{WORKLOAD} (N={o['N']}, {o['iters']} iterations, {o['seconds']:.1f} s); "
                         f"matrix-free A_C (eq. collocation via the Kronecker identity), FD of eq. "
                         f"FD3D, modified Gram-Schmidt; iteration phase only; numpy/OpenBLAS "
                         f"threads = cores",
               "busy_cores": o["cpu_seconds"] / o["seconds"]}
        xo = o["x"]
        nx = float(np.linalg.norm(xo))
        oracle_err = {"p": oracle_p, "oracle_iters": o["iters"],
                      "oracle_relres_true": o["relres_true"]}
        for f in forms:
            e = float(np.linalg.norm(x4[f] - xo) / nx)
            out[f]["rel_err_vs_oracle"] = {str(oracle_p): e}
            oracle_err[f] = e
    for f in forms:
        out[f].pop("_units", None)
        out[f].pop("_t", None)
    line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main["tts_warm_ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": CONFIG,
            "p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"],
            "iters": main["iters"], "relres_true": main["relres_true"], "by_p": main["by_p"],
            "roofline": main["roofline"], "roofline_operator": main["roofline_operator"],
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": main["gpu_launches"],
            "clocks": clk, "fp64_peak_gflops": fp64,
            "rel_err_vs_oracle": oracle_err,
            "mixed": out.get("tf32"), "tf32x3": out.get("tf32x3"), "bf16": out.get("bf16"),
            "fp64tc": out.get("fp64tc"),
            "bicgstab": bicg_out,
            "secondary_3d_annulus_ne64": secondary, "batched": batched}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_secondary(args, dev, stream, flush, name="3d_annulus_ne64"):
    """The 3D annulus with 64 elements (p = 3, 4, 5): FP64 and TF32 forms, a few steps."""
    import torch
    from paper_1705_04384_gb300.api import Problem
    c = W.CONFIGS[name]
    out = {}
    for prec in ("fp64", "tf32"):
        probs = []
        for i, p in enumerate(c["ps"]):
            P = Problem(3, c["n_elem"], p, geometry_of(c), c["r0"], c["r1"], precision=prec,
                        device=dev, stream=stream)
            rhs = torch.from_numpy(W.config_rhs(name, P.collocation_points(), i)).to(dev)
            probs.append((p, P, rhs, torch.empty_like(rhs)))
        for _ in range(2):
            for p, P, rhs, x in probs:
                P.solve(rhs, tol=TOL, max_iter=MAX_ITER, out=x)
        times, units, its, ms = 0.0, 0.0, {}, []
        for _ in range(max(3, args.steps // 2)):
            flush.fill_(1.0)
            torch.cuda.synchronize(dev)
            for p, P, rhs, x in probs:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, info = P.solve(rhs, tol=TOL, max_iter=MAX_ITER, out=x)
                e1.record(stream)
                e1.synchronize()
                dt = e0.elapsed_time(e1) * 1e-3
                times += dt
                ms.append(dt * 1e3)
                units += P.N * info["iters"]
                its[str(p)] = info["iters"]
        out[prec] = {"value": units / times, "unit": UNIT, "iters": its,
                     "p50_ms": percentile(ms, 50), "p99_ms": percentile(ms, 99)}
        for p, P, rhs, x in probs:
            P.close()
    out["workload"] = TEXTS[name]
    return out


# ------------------------------------------------------------------------- batched form
def run_batched(args, steps=None, warmup=None, emit=True):
    """256 independent 2D quarter-annulus problems (n_elem ~ U{32..512}, p ~ U{2..6},
    r0 ~ U[0.5,1.5], r1 = r0 + 1), 8 seeded Gaussian right-hand sides each, all solved
    by one iga_solve_batched call per step (every problem's 8 rhs in lockstep in one
    graph, problems concurrent on their own streams).  Prints its own line (emit) or
    returns it as a dict (the batched key of the default line)."""
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    import torch
    from paper_1705_04384_gb300.api import Problem, solve_batched
    dev = torch.device("cuda", 0)
    specs = W.batched_problems(count=args.count)
    max_iter = 50
    t0 = time.perf_counter()
    probs, rhs, outs = [], [], []
    for sp in specs:
        P = Problem(2, sp["n_elem"], sp["p"], "annulus", sp["r0"], sp["r1"],
                    precision=args.precision, device=dev, stream=torch.cuda.Stream(dev),
                    grid="throughput")
        P.prepare(sp["nrhs"], max_iter)
        B = torch.from_numpy(W.gaussian_rhs(P.N, sp["nrhs"], sp["rhs_seed"])).to(dev)
        probs.append(P)
        rhs.append(B)
        outs.append(torch.empty_like(B))
    torch.cuda.synchronize(dev)
    setup_s = time.perf_counter() - t0
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(warmup):
        solve_batched(probs, rhs, outs, tol=TOL, max_iter=max_iter)
    clocks = ClockSampler(0)
    clocks.start()
    times, dofit, res = [], 0.0, None
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        res = solve_batched(probs, rhs, outs, tol=TOL, max_iter=max_iter)
        times.append(time.perf_counter() - t)
        its = res["iters"]
        off = 0
        for P, nr in zip(probs, res["nrhs"]):
            dofit += P.N * float(its[off:off + nr].sum())
            off += nr
    clk = clocks.stop()
    tot = sum(times)
    nsolves = int(res["nrhs"].sum())
    line = {"metric": METRIC + " [batched form]", "value": dofit / tot, "unit": UNIT,
            "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "dtype": f"f64 outer, {args.precision} FD", "data": "synthetic",
            "config": {"workload": f"batched: {len(probs)} 2D quarter-annulus problems, n_elem "
                                   f"U[32,512], p U{{2..6}}, r0 U[0.5,1.5], 8 Gaussian rhs each, "
                                   f"{args.precision} FD inside flexible GMRES, tol 1e-8",
                       "dofs_total": int(sum(P.N for P in probs)), "solves_per_step": nsolves,
                       "l2": "flushed between steps (512 MB write)"},
            "solves_per_s": nsolves * len(times) / tot,
            "iters": {"min": int(res["iters"].min()), "median": float(np.median(res["iters"])),
                      "max": int(res["iters"].max())},
            "relres_true_max": float(res["relres_true"].max()),
            "not_converged": int((res["status"] != 0).sum()),
            "setup_s": setup_s, "clocks": clk}
    for P in probs:
        P.close()
    del flush
    torch.cuda.empty_cache()
    if not emit:
        return line
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------- served form
def run_served(args):
    """Poisson request stream of mixed 2D (n_elem U[64,1024], p U{2..6}) and 3D
    (n_elem U[32,160], p U{3..6}) quarter-annulus solves with seeded Gaussian rhs,
    served by continuous batching.  Phase 1 offers ``--rate`` for ``--window`` s and
    measures the sustained capacity; phase 2 offers 0.8 x that capacity."""
    import torch
    from paper_1705_04384_gb300.serve import Request, Server, latency_stats

    def make(rate, window, seed):
        out = []
        for i, r in enumerate(W.served_requests(rate=rate, duration=window, seed=seed)):
            out.append(Request(i, r["t_arrival"], r["d"], r["n_elem"], r["p"],
                               rhs=lambda N, s=r["rhs_seed"]: W.gaussian_rhs(N, 1, s)[0],
                               r0=r["r0"], r1=r["r1"]))
        return out

    phases = []
    cap = None
    for phase, (rate, seed) in enumerate([(args.rate, 3), (None, 4)]):
        if rate is None:
            rate = max(1.0, 0.8 * cap)
        window = args.window if phase == 0 else max(args.window, 30.0 / rate)  # >= 30 requests
        reqs = make(rate, window, seed)
        srv = Server(precision=args.precision, tol=TOL, max_iter=100, max_inflight=64,
                     setup_threads=8)
        t = time.perf_counter()
        done = srv.run(reqs, realtime=True, time_limit=window)
        wall = time.perf_counter() - t
        st = latency_stats(done)
        st.update({"offered_rate": rate, "offered": len(reqs), "window_s": window,
                   "achieved_rate": len(done) / wall if wall > 0 else None,
                   "dropped_unadmitted": srv.dropped, "setups": srv.setups,
                   "setups_per_s": srv.setups / wall if wall > 0 else None,
                   "setup_thread_s": srv.setup_s, "wall_s": wall,
                   "not_converged": sum(1 for r in done if r.status != 0),
                   "relres_true_max": max((r.relres for r in done), default=None)})
        srv.close()
        phases.append(st)
        if phase == 0:
            cap = st["completed"] / wall if wall > 0 else 1.0
    # the serving engine on cached shapes: 48 shapes of the same distribution are set up
    # (untimed, one request each), then the stream draws its shapes from them only
    pool_keys = []
    for r in W.served_requests(rate=args.rate, duration=10.0, seed=5):
        k = (r["d"], r["n_elem"], r["p"])
        if k not in pool_keys:
            pool_keys.append(k)
        if len(pool_keys) == 48:
            break
    srv = Server(precision=args.precision, tol=TOL, max_iter=100, max_inflight=64,
                 setup_threads=8)
    warm = [Request(i, 0.0, d, ne, p, rhs=lambda N, s=9000 + i: W.gaussian_rhs(N, 1, s)[0])
            for i, (d, ne, p) in enumerate(pool_keys)]
    srv.run(warm, realtime=False)
    warm_phases = []
    wcap = None
    for phase, (rate, seed) in enumerate([(args.rate, 6), (None, 7)]):
        if rate is None:
            rate = max(1.0, 0.8 * wcap)
        window = args.window
        rng = np.random.Generator(np.random.PCG64(seed))
        reqs, t = [], 0.0
        while True:
            t += float(rng.exponential(1.0 / rate))
            if t > window:
                break
            d, ne, p = pool_keys[int(rng.integers(len(pool_keys)))]
            reqs.append(Request(len(reqs), t, d, ne, p,
                                rhs=lambda N, s=seed * 1000003 + len(reqs): W.gaussian_rhs(N, 1, s)[0]))
        setups0 = srv.setups
        t0 = time.perf_counter()
        done = srv.run(reqs, realtime=True, time_limit=window)
        wall = time.perf_counter() - t0
        st = latency_stats(done)
        st.update({"offered_rate": rate, "offered": len(reqs), "window_s": window,
                   "achieved_rate": len(done) / wall if wall > 0 else None,
                   "dropped_unadmitted": srv.dropped, "wall_s": wall,
                   "new_handles": srv.setups - setups0,
                   "not_converged": sum(1 for r in done if r.status != 0),
                   "relres_true_max": max((r.relres for r in done), default=None)})
        warm_phases.append(st)
        if phase == 0:
            wcap = st["completed"] / wall if wall > 0 else 1.0
    srv.close()
    line = {"metric": METRIC + " [served form]", "value": phases[1].get("solves_per_s"),
            "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": f"f64 outer, {args.precision} FD", "data": "synthetic",
            "config": {"workload": "served: Poisson arrivals, 50% 2D (n_elem U[64,1024], p "
                                   "U{2..6}), 50% 3D (n_elem U[32,160], p U{3..6}), quarter "
                                   "annulus r in [1,2], Gaussian rhs, tol 1e-8, continuous "
                                   "batching (64 in flight, memory-budget admission, warm "
                                   "shapes first, 8 concurrent setups)",
                       "window_s": args.window},
            "p50_ms": phases[1].get("p50_ms"), "p99_ms": phases[1].get("p99_ms"),
            "phase_offered": phases[0], "phase_0p8_capacity": phases[1],
            "cached_shapes": {"note": "the same engine with every shape already set up: 48 shapes "
                                      "of the same distribution (seed 5), one untimed request "
                                      "each, then Poisson streams over those shapes only",
                              "shapes": len(pool_keys), "phase_offered": warm_phases[0],
                              "phase_0p8_capacity": warm_phases[1]}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    global WORKLOAD
    named = {"3d_ne128": "3d_annulus_ne128", "3d_ne64": "3d_annulus_ne64",
             "3d_revolved_ne64": "3d_revolved_ne64", "3d_wind_ne64": "3d_wind_ne64",
             "3d_wq_revolved_ne64": "3d_wq_revolved_ne64"}
    if args.workload in named:
        WORKLOAD = named[args.workload]
        CONFIG["workload"] = TEXTS[WORKLOAD]
        if WORKLOAD != "3d_annulus_ne128":
            args.no_secondary = True
            args.no_batched = True
        if WORKLOAD == "3d_wind_ne64":
            args.no_mixed = True  # the wind path runs the FP64 FD only
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batched", "served"):
        # more hardware queues for many concurrent streams (read at CUDA init)
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
        return run_batched(args) if args.workload == "batched" else run_served(args)
    if not args.no_batched:
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
