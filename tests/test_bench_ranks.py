"""The multi-rank path of bench.py on CPU (gloo, world size 2): the whole-job reduction
(slowest rank's time, units summed over ranks) and the reference arm under torchrun, where
rank 0 alone times the oracle and prints the one JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    dist.init_process_group("gloo", rank=rank, world_size=2)
    sys.path.insert(0, ROOT)
    import bench
    ms, units = bench.combine_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1), "cpu")
    out[rank] = (ms, units)
    dist.destroy_process_group()


def test_combine_ranks_takes_slowest_time_and_sums_units():
    port = free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(port, out), nprocs=2, join=True)
        for r in (0, 1):
            assert out[r] == (15.0, 300.0)


def test_combine_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(3.5, 7.0, "cpu") == (3.5, 7.0)


def test_reference_arm_under_torchrun_prints_one_line():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--workload", "heat2d_63", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_dr_times_douglas_rachford_steps():
    """--fine dr: the reference arm times the oracle's DR steps, and the line's config says so
    (FP64, fine = dr) before any GPU is touched."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "heat2d_63",
           "--fine", "dr", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert d["config"]["fine"] == "dr" and d["config"]["precision"] == "fp64"
    assert "DR step" in d["cpu_baseline"]["sample"] and d["value"] > 0


def test_fine_dr_refuses_batch_and_adjoint_workloads():
    for w in ("batch256", "adjoint2d_511"):
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", w,
               "--fine", "dr", "--steps", "1", "--warmup", "3"]
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
        assert r.returncode != 0 and "single-problem workloads" in (r.stderr + r.stdout), w


def test_scalability_workload_recipe():
    """The Sec. 5.1 scalability workload: 99^2, q = 2 fine strips of overlap 1/16, q coarse strips
    of overlap 1/32, five iterations, the manufactured solution for the error."""
    sys.path.insert(0, ROOT)
    import bench
    cfg = bench.workload("dd_scal99_q8")
    assert cfg["n"] == (99, 99) and cfg["N"] == 32 and cfg["s"] == 100 and cfg["max_iter"] == 5
    assert cfg["boxes"] == (4, 1) and cfg["coarse_boxes"] == (16, 1)
    assert cfg["overlap"] == 1 / 16 and cfg["coarse_overlap"] == 1 / 32
    assert cfg["src_t"].shape == (32 * 100 + 1,)
