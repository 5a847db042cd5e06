"""Benchmark: GMRES + FD time-to-1e-8 and DOF-iterations per second on one GB300.

Workload (default): the 3D extruded thick quarter annulus r in [1,2], z in [0,1],
64 elements per direction, p = 3, 4, 5 (N = 274,625 / 287,496 / 300,763), forcing
from the manufactured solution plus the seeded 1e-3 perturbation, GMRES tol 1e-8,
FP64 throughout.  One step = one solve for each p (cached setup).  The mixed
(TF32-FD flexible GMRES) form of the same solves is reported beside it.

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
WORKLOAD = "3d_annulus_ne64"
TOL = 1e-8
MAX_ITER = 200
FP64_PEAK_GFLOPS = 1250.0  # nominal GB300 FP64: 2 FMA/clk/SM x 152 SMs x 2.07 GHz x 2 FLOP
CONFIG = {"workload": f"{WORKLOAD}: 3D extruded quarter annulus r in [1,2], z in [0,1], 64 "
                      f"elements/dir, p=3,4,5 (N=274625/287496/300763), manufactured f + seeded "
                      f"1e-3 perturbation, FP64 FD-GMRES to 1e-8",
          "step": "one solve per p (setup cached)",
          "l2": "flushed between steps (512 MB write)", "parallelism": "replicas"}
REVOLVED_TEXT = ("3d_revolved_ne64: 3D quarter ring r in [1,2] revolved by pi/2 about the axis "
                 "(0,1,0) through (-1,-1,-1), 64 elements/dir, p=3,4,5, f = 1 + seeded 1e-3 "
                 "perturbation, FP64 FD-GMRES to 1e-8")


WIND_TEXT = ("3d_wind_ne64: convection-diffusion -Lap + w.grad (Sec. 3.2) with w = (5,5,5) on "
             "the 3D extruded quarter annulus, 64 elements/dir, p=3,4,5, f = 1 + seeded 1e-3 "
             "perturbation, FD of the wind-shifted pencils, FP64 FD-GMRES to 1e-8")


def geometry_of(c):
    return c.get("geometry", "annulus")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-bicgstab", action="store_true")
    ap.add_argument("--workload", default="3d_ne64",
                    choices=["3d_ne64", "3d_revolved_ne64", "3d_wind_ne64", "batched", "served"],
                    help="3d_ne64 (default bench line), 3d_revolved_ne64 (Sec. 5's revolved "
                         "ring, same measurement), 3d_wind_ne64 (Sec. 3.2 convection-diffusion), "
                         "batched (256 2D problems x 8 rhs), served (Poisson request stream)")
    ap.add_argument("--precision", default="tf32", help="preconditioner precision for the "
                                                        "batched / served forms")
    ap.add_argument("--count", type=int, default=256, help="problems in the batched form")
    ap.add_argument("--rate", type=float, default=2000.0, help="offered load, requests/s")
    ap.add_argument("--window", type=float, default=2.0, help="served arrival window, s")
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
def kernel_source_hash():
    """Hash of the dominant kernel's source file with comments and blank space removed, so
    that an edit of its comments does not void the committed counters."""
    h = hashlib.sha256()
    for f in ("kernels_fd64.cu",):
        with open(os.path.join(ROOT, "paper_1705_04384_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def committed_traffic(summary="fd_fold_mma_3d_ne64.md"):
    """dram bytes per launch of the dominant kernel from the committed ncu summary,
    or None when the kernel source changed since the capture."""
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
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return float(vals["traffic_bytes_per_launch"]) if "traffic_bytes_per_launch" in vals else None


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


# ------------------------------------------------------------------------- reference arm
def run_reference(args):
    """Time the FP64 CPU oracle on a bounded sample of the same workload."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    from oracle import collocation as C, fd as F, geometry as Geo, gmres as G
    c = W.CONFIGS[WORKLOAD]
    p = c["ps"][0]
    spaces = [C.Space1D(c["n_elem"], p) for _ in range(3)]
    fmap = Geo.make_map(geometry_of(c), 3, c["r0"], c["r1"])
    A = C.assemble_collocation(spaces, fmap, c.get("wind"))
    pts = C.physical_points(fmap, [s.tau for s in spaces])
    b = W.config_rhs(WORKLOAD, pts, 0)
    fd = F.FD(spaces, c.get("wind"))
    N = A.shape[0]
    times, cpu_s, dofit = [], 0.0, 0
    for it in range(args.warmup + args.steps):
        t0, c0 = time.perf_counter(), time.process_time()
        r = G.gmres(A, b, M=fd, tol=TOL, max_iter=MAX_ITER)
        dt, dc = time.perf_counter() - t0, time.process_time() - c0
        if it >= args.warmup:
            times.append(dt)
            cpu_s += dc
            dofit += N * r["iters"]
    tot = sum(times)
    value = dofit / tot
    cores = os.cpu_count()
    sample = (f"oracle GMRES+FD, one full solve to 1e-8 of the p={p} problem (N={N}, "
              f"{r['iters']} iterations) per step; iteration phase only (CSR assembly and "
              f"eigendecomposition are setup, outside the timer)")
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


def cpu_baseline_sample(budget_s=15.0):
    """The oracle as it stands on the host cores, bounded: full GMRES+FD solves to
    1e-8 of the p = 3 problem of the workload (iteration phase; CSR assembly and the
    eigendecomposition are setup), repeated until about ``budget_s`` seconds."""
    from oracle import collocation as C, fd as F, geometry as Geo, gmres as G
    c = W.CONFIGS[WORKLOAD]
    p = c["ps"][0]
    spaces = [C.Space1D(c["n_elem"], p) for _ in range(3)]
    fmap = Geo.make_map(geometry_of(c), 3, c["r0"], c["r1"])
    A = C.assemble_collocation(spaces, fmap, c.get("wind"))
    pts = C.physical_points(fmap, [s.tau for s in spaces])
    b = W.config_rhs(WORKLOAD, pts, 0)
    fd = F.FD(spaces, c.get("wind"))
    N = A.shape[0]
    dofit, spent, cpu_s, solves, its = 0, 0.0, 0.0, 0, 0
    while spent < budget_s and solves < 50:
        t0, c0 = time.perf_counter(), time.process_time()
        r = G.gmres(A, b, M=fd, tol=TOL, max_iter=MAX_ITER)
        spent += time.perf_counter() - t0
        cpu_s += time.process_time() - c0
        dofit += N * r["iters"]
        its = r["iters"]
        solves += 1
    return {"value": dofit / spent, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{solves} full solves to 1e-8 ({its} iterations each) of {WORKLOAD} p={p}, "
                      f"N={N}, iteration phase only; {spent:.1f} s; numpy/OpenBLAS threads = cores, "
                      f"scipy CSR matvec single-threaded",
            "busy_cores": cpu_s / spent}


# ------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1705_04384_gb300.api import Problem

    c = W.CONFIGS[WORKLOAD]
    stream = torch.cuda.current_stream(dev)

    def make(prec):
        probs = []
        for i, p in enumerate(c["ps"]):
            P = Problem(3, c["n_elem"], p, geometry_of(c), c["r0"], c["r1"], precision=prec,
                        wind=c.get("wind"),
                        device=dev, stream=stream)
            pts = P.collocation_points()
            rhs = torch.from_numpy(W.config_rhs(WORKLOAD, pts, i)).to(dev)
            probs.append((p, P, rhs, torch.empty_like(rhs)))
        return probs

    t_setup = time.perf_counter()
    fp64 = make("fp64")
    t_setup = time.perf_counter() - t_setup
    mixed = None
    if not args.no_mixed:
        try:
            mixed = make("tf32")
        except Exception as e:  # the mixed form is reported when it is built
            mixed = None
            mixed_err = str(e)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run_step(probs, record, solver="gmres"):
        per = []
        for p, P, rhs, x in probs:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if solver == "gmres":
                _, info = P.solve(rhs, tol=TOL, max_iter=MAX_ITER, out=x)
            else:
                _, info = P.solve_bicgstab(rhs, tol=TOL, max_iter=MAX_ITER, out=x)
            e1.record(stream)
            per.append((p, P, info, e0, e1))
        torch.cuda.synchronize(dev)
        out = []
        for p, P, info, e0, e1 in per:
            out.append((p, P.N, info["iters"], e0.elapsed_time(e1) * 1e-3, info["relres_true"]))
        return out

    def timed(probs, steps, warmup, solver="gmres"):
        for _ in range(warmup):
            run_step(probs, False, solver)
        results = []
        for _ in range(steps):
            flush.fill_(1.0)  # L2 flush between steps, outside the timed solves
            torch.cuda.synchronize(dev)
            results.append(run_step(probs, True, solver))
        return results

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local_rank)
    clocks.start()
    res64 = timed(fp64, args.steps, args.warmup)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    step_times = [sum(s[3] for s in step) for step in res64]
    dof_iters = [sum(s[1] * s[2] for s in step) for step in res64]
    all_units, total_t = aggregate(sum(dof_iters), sum(step_times), dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    value = all_units / total_t
    solve_ms = [s[3] * 1e3 for step in res64 for s in step]
    iters = {str(s[0]): s[2] for s in res64[-1]}
    relres = {str(s[0]): s[4] for s in res64[-1]}
    launches = 0
    for step in res64:
        for (p, P, rhs, x), s in zip(fp64, step):
            f, it = P.launch_counts()
            launches += f + it * s[2]

    # dominant kernel: the FP64 FD mode-product GEMM (6 launches per FD apply)
    p0, P0, rhs0, x0 = fp64[0]
    reps = 20
    flush.fill_(1.0)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    buf = torch.empty_like(rhs0)
    e0.record(stream)
    for _ in range(reps):
        P0.precond_apply(rhs0, out=buf)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_launch = e0.elapsed_time(e1) * 1e-3 / (reps * 6)
    n = P0.n
    ne, no = (n + 1) // 2, n // 2
    rows = n ** 2  # 3D: one row per (i2, i3) fiber
    # algorithmic FLOPs of one folded mode product, averaged over the d forward
    # (even block ne x ne, odd block no x no) and d inverse (ne pairs x n) launches
    flops = 0.5 * (2.0 * rows * (ne * ne + no * no) + 2.0 * rows * ne * n)
    achieved = flops / t_launch / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS,
                "unit": "GFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS,
                "traffic": committed_traffic(),
                "kernel": "fd_fold_mma_kernel (folded FD mode product, FP64 mma.sync m8n8k4)",
                "per_launch_us": t_launch * 1e6, "flops_per_launch": flops,
                "dense_equivalent_flops_per_launch": 2.0 * n ** 4,
                "peak_note": "nominal GB300 FP64 1.25 TFLOP/s (2 FMA/clk/SM x 152 SMs x 2.07 GHz); "
                             "of nominal. An FP64 mma.sync throughput probe on this GPU reached "
                             "1050 GFLOP/s"}

    # end to end through the host-buffer entry point
    e2e_times, e2e_dofit, h2d, d2h = [], 0, 0, 0
    host = []
    for p, P, rhs, x in fp64:
        hr = torch.empty(P.N, dtype=torch.float64, pin_memory=True)
        hr.copy_(rhs.cpu())
        hx = torch.empty(P.N, dtype=torch.float64, pin_memory=True)
        host.append((P, hr, hx))
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

    mixed_out = None
    if mixed is not None:
        resm = timed(mixed, args.steps, args.warmup)
        mt = sum(sum(s[3] for s in step) for step in resm)
        md = sum(sum(s[1] * s[2] for s in step) for step in resm)
        mu, mtx = aggregate(md, mt, dev)
        mixed_out = {"value": mu / mtx, "unit": UNIT,
                     "iters": {str(s[0]): s[2] for s in resm[-1]},
                     "relres_true": {str(s[0]): s[4] for s in resm[-1]},
                     "p50_ms": percentile([s[3] * 1e3 for st in resm for s in st], 50),
                     "p99_ms": percentile([s[3] * 1e3 for st in resm for s in st], 99),
                     "time_to_solution_ms_per_step": 1e3 * mt / len(resm)}
        # error of the precision form's solution against the FP64 form's (the FP64 GPU
        # solution equals the oracle's at a fixed step count to 1e-10; both stop at 1e-8)
        mixed_out["rel_err_vs_fp64"] = {
            str(p): float(torch.linalg.vector_norm(xm - x) / torch.linalg.vector_norm(x))
            for (p, _, _, x), (_, _, _, xm) in zip(fp64, mixed)}

    # Sec. 5's solver on the same problems: BiCGStab + FP64 FD; an iteration is a BiCG
    # step and a GMRES(1) step (two FD solves, two operator applications), counted in
    # halves as the paper does
    bicg_out = None
    if not args.no_bicgstab:
        resb = timed(fp64, max(1, args.steps // 2), args.warmup, "bicgstab")
        bt = sum(sum(s[3] for s in step) for step in resb)
        bd = sum(sum(s[1] * s[2] for s in step) for step in resb)
        bu, btx = aggregate(bd, bt, dev)
        bicg_out = {"value": bu / btx, "unit": "DOF-iter/s (BiCGStab iterations)",
                    "iters": {str(s[0]): s[2] for s in resb[-1]},
                    "relres_true": {str(s[0]): s[4] for s in resb[-1]},
                    "p50_ms": percentile([s[3] * 1e3 for st in resb for s in st], 50),
                    "time_to_solution_ms_per_step": 1e3 * bt / len(resb)}

    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / len(res64),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": CONFIG,
            "p50_ms": percentile(solve_ms, 50), "p99_ms": percentile(solve_ms, 99),
            "iters": iters, "relres_true": relres, "setup_s_cold": t_setup,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "mixed": mixed_out, "bicgstab": bicg_out}
    if mixed_out is None and not args.no_mixed:
        line["mixed_unavailable"] = mixed_err if "mixed_err" in locals() else "not built"
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------- batched form
def run_batched(args):
    """256 independent 2D quarter-annulus problems (n_elem ~ U{32..512}, p ~ U{2..6},
    r0 ~ U[0.5,1.5], r1 = r0 + 1), 8 seeded Gaussian right-hand sides each, all solved
    by one iga_solve_batched call per step (every problem's 8 rhs in lockstep in one
    graph, problems concurrent on their own streams)."""
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
    for _ in range(args.warmup):
        solve_batched(probs, rhs, outs, tol=TOL, max_iter=max_iter)
    clocks = ClockSampler(0)
    clocks.start()
    times, dofit, res = [], 0.0, None
    for _ in range(args.steps):
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
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
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
    print(json.dumps(line), flush=True)
    for P in probs:
        P.close()
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
        window = args.window if phase == 0 else max(args.window, 30.0 / rate)
        reqs = make(rate, window, seed)
        srv = Server(precision=args.precision, tol=TOL, max_iter=100, max_inflight=64,
                     setup_threads=8)
        t = time.perf_counter()
        done = srv.run(reqs, realtime=True, time_limit=window)
        wall = time.perf_counter() - t
        st = latency_stats(done)
        st.update({"offered_rate": rate, "offered": len(reqs), "window_s": window,
                   "dropped_unadmitted": len(reqs) - len(done), "setups": srv.setups,
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
                   "dropped_unadmitted": len(reqs) - len(done), "wall_s": wall,
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
                                   "batching (64 in flight, memory-budget admission, 8 setup "
                                   "threads)"},
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
    if args.workload in ("3d_revolved_ne64", "3d_wind_ne64"):
        global WORKLOAD
        WORKLOAD = args.workload
        CONFIG["workload"] = REVOLVED_TEXT if args.workload == "3d_revolved_ne64" else WIND_TEXT
        if args.workload == "3d_wind_ne64":
            args.no_mixed = True  # the wind path runs the FP64 FD only
        args.workload = "3d_ne64"
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "3d_ne64":
        # more hardware queues for many concurrent streams (read at CUDA init)
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
        return run_batched(args) if args.workload == "batched" else run_served(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
