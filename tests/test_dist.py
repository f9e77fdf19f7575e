"""Multi-process host logic on CPU (gloo, two ranks): the reductions that
turn per-rank timings into the whole-job rate, the reference arm's
rank-0-only rule, and the reference arm's JSON line."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    from paper_2607_20704_gb300 import dist
    assert dist.env() == (rank, world, rank)
    dist.init("gloo")
    dist.barrier()
    mx = dist.max_over_ranks(rank + 1.0)
    sm = dist.sum_over_ranks(rank + 1.0)
    # rank r processed 10 units in (1 + r) seconds
    rate, slowest = dist.throughput(10.0, 1.0 + rank)
    dist.finalize()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{mx} {sm} {rate} {slowest}\n")


def test_reductions_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        mx, sm, rate, slowest = map(float, (tmp_path / f"r{r}.txt").read_text().split())
        assert mx == 2.0 and sm == 3.0
        assert slowest == 2.0 and rate == pytest.approx(20.0 / 2.0)


def test_single_process_reductions_are_identity():
    from paper_2607_20704_gb300 import dist
    assert dist.max_over_ranks(3.5) == 3.5
    assert dist.throughput(12.0, 4.0) == (3.0, 4.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    """Rank 0 of the reference arm: one JSON line, the oracle timed on the
    host, with the keys the driver reads."""
    import json
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "leaf cell-updates/s"
    assert d["unit"] == "leaf cell-updates/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] >= 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    upd = d["config"]["cell_updates_per_step"]
    assert abs(d["value"] - upd / (d["ms_per_step"] * 1e-3)) <= 1e-6 * d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "sedov_l7-10_static_nested_balls"
    # the same config dict as the GPU arm prints for this mesh (the GPU
    # arm's counts come from the library; the ghost and leaf counts of the
    # mesh are pinned against the oracle by the parity tests)
    import bench
    from paper_2607_20704_gb300 import inputs
    prob = inputs.sedov()
    want = bench.workload_config(prob.n_oct, d["config"]["n_ghost_oct"], prob.leaf_cells(), upd, 1)
    assert d["config"] == want
    assert d["config"]["leaf_cells"] == 2416184 and d["config"]["n_ghost_oct"] == 14280
