"""Host-side pieces of bench.py and the input generators (no GPU)."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as tmp

import bench
from paper_1103_4697_gb300 import workloads as W


def test_batch_arrays_match_generator():
    F, G = W.deg20_batch_arrays(3, 2000)
    ps = W.deg20_batch(3, 2000)
    for q in range(3):
        f = np.zeros((21, 21), dtype=np.int64)
        g = np.zeros((21, 21), dtype=np.int64)
        for j, r in enumerate(ps.f[q]):
            f[j, :len(r)] = r
        for j, r in enumerate(ps.g[q]):
            g[j, :len(r)] = r
        assert (F[q] == f).all() and (G[q] == g).all()
    fs, gs = W.deg20_pair(2000)
    assert (F[0] == np.array(fs)).all()


def test_generator_is_deterministic_and_in_range():
    a = W.Stream(5).signed_bits(16, 1000)
    b = W.Stream(5).signed_bits(16, 1000)
    assert a == b
    assert min(a) >= -2 ** 15 and max(a) <= 2 ** 15 - 1
    assert W.Stream(6).signed_bits(16, 10) != a[:10]
    u = W.Stream(1).uniform_int(4, 16, 5000)
    assert min(u) == 4 and max(u) == 16


def test_rank_seeds_disjoint():
    seeds = [set(range(bench.rank_seed_base(r, 4096), bench.rank_seed_base(r, 4096) + 4096)) for r in range(4)]
    assert bench.rank_seed_base(0) == 2000
    for i in range(4):
        for j in range(i + 1, 4):
            assert not seeds[i] & seeds[j]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    m = bench.reduce_max(10.0 + rank, world)
    out[rank] = m
    dist.destroy_process_group()


def test_reduce_max_gloo_two_ranks():
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    tmp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == 11.0


def _bench_reference(env_extra):
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    return p.returncode, [json.loads(l) for l in lines]


def test_reference_arm_line_and_other_ranks():
    """bench.py --impl reference (the oracle on the host cores): rank 0 prints one
    JSON line with the contract's keys; any other rank exits 0 and prints nothing."""
    rc, out = _bench_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert rc == 0 and out == []
    rc, out = _bench_reference({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert rc == 0 and len(out) == 1
    line = out[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "workload" in line["config"]


def test_traffic_figure_tracks_the_kernel_source(tmp_path, monkeypatch):
    """bench.py reports the committed ncu traffic of the evaluation kernel only while
    the hash of its source files matches the summary's; any edit of either file
    drops it to null."""
    import hashlib
    import json
    import shutil

    root = tmp_path / "r"
    files = ["paper_1103_4697_gb300/csrc/gbr_evalres.cu", "paper_1103_4697_gb300/csrc/gbr_elim.cuh"]
    for rel in files:
        (root / rel).parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), root / rel)
    summary = json.load(open(os.path.join(bench.ROOT, "profiles", "evalres_dram.json")))
    assert summary["source_files"] == files
    summary["source_sha"] = hashlib.sha256(b"".join(open(root / f, "rb").read() for f in files)).hexdigest()[:16]
    (root / "profiles").mkdir()
    json.dump(summary, open(root / "profiles" / "evalres_dram.json", "w"))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.traffic_for() == summary["bytes_per_launch_full"]
    with open(root / "paper_1103_4697_gb300/csrc/gbr_elim.cuh", "a") as fh:
        fh.write("\n")
    assert bench.traffic_for() is None
