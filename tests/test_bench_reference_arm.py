"""The reference arm of bench.py on CPU: the oracle timed on the host cores, one JSON line.

`bench.py --impl reference` times the FP64 oracle (GMRES + FD, Sec. 3-4) on a bounded sample
of the benchmark workload (a few Arnoldi iterations of its p = 4 problem per step) and prints
the same line as the GPU arm, with `"impl": "reference"`, a `cpu_baseline` that describes the
run and an `e2e` object with no host-device bytes.  One step checks the keys, their types and
that the sampled iterations reduced the residual.
"""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "LOCAL_RANK", "WORLD_SIZE")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])

    sys.path.insert(0, ROOT)
    import bench
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["steps"] == 1 and line["warmup"] == 0
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["config"]["workload"].startswith(bench.WORKLOAD)
    assert line["vs_baseline"] is None

    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == line["value"]
    assert cpu["unit"] == line["unit"] and cpu["cores"] >= 1 and cpu["sample"]
    assert 0 < cpu["busy_cores"] <= cpu["cores"] + 0.5
    e2e = line["e2e"]
    assert e2e == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}
    # the sampled Arnoldi iterations reduced the relative residual estimate (FD-preconditioned
    # GMRES on this problem gains more than a digit in three steps)
    assert 0 < line["last_relres_est"] < 0.1
