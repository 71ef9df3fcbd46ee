"""bench.py --gpus N starts N ranks itself (one process per GPU under
torch.distributed.run) when it is not already running under torchrun, and refuses a
torchrun world size that differs from --gpus.  Driven here on the CPU through the
launcher's stub step: every rank takes its sky shard as the GPU path does and the
shards meet over gloo."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR",
                                                            "MASTER_PORT")}
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                          env=env, timeout=300, cwd=ROOT)


def test_gpus_2_launches_two_ranks_with_disjoint_sky_shards():
    r = _run(["--gpus", "2", "--stub", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout  # rank 0 alone prints
    d = lines[0]
    assert d["n_gpus"] == 2 and d["stub"] is True
    a, b = d["rank_shards"]
    assert len(a) == len(b) == d["config"]["nsky"]
    assert not set(a) & set(b)
    assert sorted(a + b) == list(range(2 * d["config"]["nsky"]))
    assert d["ms_per_step"] == 2.0  # the maximum over the ranks' 1.0 and 2.0


def test_gpus_1_runs_in_process():
    r = _run(["--gpus", "1", "--stub"])
    assert r.returncode == 0, r.stderr[-3000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["n_gpus"] == 1 and d["rank_shards"] == [list(range(d["config"]["nsky"]))]


def test_world_size_must_match_gpus():
    r = _run(["--gpus", "2", "--stub"], {"WORLD_SIZE": "1", "RANK": "0", "LOCAL_RANK": "0"})
    assert r.returncode != 0
    assert "WORLD_SIZE" in r.stderr
