"""The benchmark's reference arm (the CPU oracle on every host core) prints one JSON
line with the workload's own metric, unit and config, for a single segment, a batch,
the fine search, the adjoint and the constrained lattice, without a GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload,unit", [("tiny", "templates/s"), ("uneven_small", "templates/s"),
                                           ("refine_2d", "candidates/s"), ("adjoint_2d", "candidates/s"),
                                           ("lattice_2d", "templates/s")])
def test_reference_arm_line(workload, unit):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload, "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["unit"] == unit and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1
    assert d["config"]["workload"] == workload
    # the oracle runs on every host core (one worker process per core), core count and CPU named
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert d["cpu_baseline"]["cpu"] and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
