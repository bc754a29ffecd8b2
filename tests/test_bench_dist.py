"""The multi-process side of bench.py on CPU (gloo, world size 2): ranks
agree on the slowest rank's time and the whole-job rate counts every rank's
hits; the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 * (rank + 1)   # rank 1 is the slower one
        q.put((rank, bench.job_rate(ms_local, hits_per_rank=1000, steps=5, world=world, dist=dist)))
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_over_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        ms_max, rate = got[rank]
        assert ms_max == 20.0
        assert rate == pytest.approx(1000 * 2 * 5 / 0.020)


def test_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    ms_max, rate = bench.job_rate(4.0, hits_per_rank=100, steps=2, world=1)
    assert ms_max == 4.0 and rate == pytest.approx(100 * 2 / 0.004)


def test_reference_arm_is_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0
    assert out.stdout.strip() == ""


def test_reference_arm_line():
    """Rank 0 of the reference arm times the oracle and prints one line with
    the contract's keys: impl, the same metric and unit, cpu_baseline of kind
    oracle, and an e2e object with no host-device bytes."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--scale", "0.002", "--ref-sample", "20000", "--steps", "2",
                          "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    import bench
    assert rec["impl"] == "reference" and rec["metric"] == bench.METRIC
    assert rec["unit"] == "hits/s" and rec["higher_is_better"] is True
    assert rec["steps"] == 2 and rec["warmup"] == 3 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["e2e"] == {"value": rec["value"], "unit": "hits/s", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}


def _tree_with_profile(tmp_path, monkeypatch, fields):
    """A copy of the kernel sources with a traffic.json captured "on" them."""
    import shutil
    import bench
    root = tmp_path / "repo"
    csrc = root / "paper_2412_11809_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(bench.ROOT, "paper_2412_11809_gb300", "csrc")
    for f in os.listdir(src):
        if f.endswith((".cu", ".cuh")):
            shutil.copy(os.path.join(src, f), csrc / f)
    (root / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec = {k: dict(v, source_sha=bench.kernel_source_sha()) for k, v in fields.items()}
    with open(root / "profiles" / "traffic.json", "w") as f:
        json.dump(rec, f)
    return root, csrc


def test_stored_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    """A stored ncu traffic figure is used only while the kernel sources hash
    to the value it was captured with; host-only files do not enter the hash."""
    import bench
    root, csrc = _tree_with_profile(tmp_path, monkeypatch, {
        "k_tile_link_table": {"dram_bytes_per_hit": 16.0},
        "step": {"dram_bytes_per_hit": 70.0}})
    assert bench.stored_traffic("k_tile_link_table", 1000) == pytest.approx(16.0 * 1000)
    assert bench.stored_step_traffic(1000) == pytest.approx(70.0 * 1000)
    with open(csrc / "filler.cu", "a") as f:          # host-only code: still valid
        f.write("\n// host-side change\n")
    assert bench.stored_traffic("k_tile_link_table", 1000) is not None
    with open(csrc / "link.cu", "a") as f:            # the kernel changed: no figure
        f.write("\n// kernel change\n")
    assert bench.stored_traffic("k_tile_link_table", 1000) is None
    assert bench.stored_step_traffic(1000) is None


def test_issue_roofline_from_stored_instruction_count(tmp_path, monkeypatch):
    """Warp instructions per hit (stored from ncu) x hits / kernel time against
    4 schedulers per SM at the sampled clock."""
    import bench
    _tree_with_profile(tmp_path, monkeypatch, {
        "k_tile_link_table": {"warp_instructions_per_hit": 20.5}})
    per_hit = bench.stored_profile("k_tile_link_table", "warp_instructions_per_hit")
    assert per_hit == pytest.approx(20.5)
    r = bench.issue_roofline("k_tile_link_table", 2**26, 2.0, 152, 2000.0)
    assert r["peak"] == pytest.approx(152 * 4 * 2000e6)
    assert r["achieved"] == pytest.approx(per_hit * 2**26 / 2e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert bench.issue_roofline("k_tile_link_table", 2**26, 2.0, 152, None) is None
    assert bench.issue_roofline("k_accumulate", 2**26, 2.0, 152, 2000.0) is None


def test_forest_depth_of_a_hand_built_forest():
    """Steps to the root of every node (the union-find depth metric)."""
    import numpy as np
    import bench
    # 0 <- 1 <- 2 <- 3, 2 <- 4; 5 <- 6
    d = bench.forest_depth(np.array([0, 0, 1, 2, 2, 5, 5], dtype=np.uint32))
    assert d == {"max": 3, "mean": pytest.approx(10 / 7), "nodes": 7, "roots": 2, "deeper_than_1": 3}
    assert bench.forest_depth(np.arange(5, dtype=np.uint32))["max"] == 0
