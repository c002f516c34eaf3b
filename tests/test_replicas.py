"""Host side of the multi-GPU path (replicas: one independent frame per rank,
no data-path collective) on CPU processes over gloo, world size 2: the
slowest rank's time and the whole-job rate, and the reference arm's
rank-0-only rule under a two-rank launch."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2609_32375_gb300 import replicas
    r, w, local = replicas.rank_env()
    dist = replicas.init(w, "gloo")
    replicas.barrier(dist)
    step_ms = 10.0 + 5.0 * r                      # rank 1 is the slower one
    slowest = replicas.max_over_ranks(step_ms, dist)
    rate = replicas.job_rate(151.2, w, slowest / 1e3)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"rank": r, "world": w, "local": local, "slowest": slowest, "rate": rate,
                   "seed": replicas.frame_seed(r)}, f)
    replicas.finish(dist)


def test_replicas_take_the_slowest_rank_and_count_every_rank(tmp_path):
    port = _free_port()
    torch.multiprocessing.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["world"] == 2 and d["local"] == r
        assert d["slowest"] == 15.0                              # the max over ranks, on every rank
        assert d["rate"] == pytest.approx(2 * 151.2 / 0.015)    # both ranks' pixels / the slowest time
    assert res[0]["seed"] != res[1]["seed"]                     # independent frames


def test_single_process_needs_no_process_group():
    from paper_2609_32375_gb300 import replicas
    assert replicas.init(1) is None
    assert replicas.max_over_ranks(3.5, None) == 3.5
    replicas.barrier(None)
    replicas.finish(None)


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    """Under a two-rank launch the oracle arm prints one JSON line from rank
    0; rank 1 exits 0 without work."""
    outs = []
    for rank in (0, 1):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(_free_port()))
        p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                            "--steps", "1", "--warmup", "0", "--size", "256x192", "--ref-crop", "128"],
                           capture_output=True, text=True, env=env, cwd=str(tmp_path), timeout=300)
        assert p.returncode == 0, p.stderr[-2000:]
        outs.append([l for l in p.stdout.splitlines() if l.startswith("{")])
    assert len(outs[0]) == 1 and outs[1] == []
    line = json.loads(outs[0][0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
