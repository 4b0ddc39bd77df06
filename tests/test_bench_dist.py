"""The multi-GPU path of bench.py on CPU: two gloo ranks, each an independent replica (no
collective on the data path); the whole-job value is every rank's updates over the slowest
rank's timed region."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms_local = [12.0, 20.0][rank]  # rank 1 is the slowest
    units_local = [1000, 3000][rank]
    ms, units, value = bench.aggregate(ms_local, units_local, dist, "cpu")
    dist.barrier()
    out[rank] = (ms, units, value)
    dist.destroy_process_group()


def test_two_replicas_aggregate_over_the_slowest_rank():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in range(2):
        ms, units, value = res[r]
        assert ms == 20.0 and units == 4000.0
        assert abs(value - 4000.0 / 0.020) < 1e-6


def test_single_process_aggregate_is_local():
    import bench

    assert bench.aggregate(10.0, 500) == (10.0, 500, 50000.0)


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the FP64 oracle on the host: one JSON line with the
    arm's metric and unit, impl "reference", its cpu_baseline and an e2e block without
    transfers (about 15 s on one core)."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "nnz-updates/s per epoch" and d["unit"] == "nnz-updates/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the workload's description is the GPU arm's own (bench.run_config), key for key
    cfg = d["config"]
    assert cfg["I"] == [4500, 15000, 5] and cfg["J"] == [10, 10, 5] and cfg["nnz_train"] == 27_000_000
    assert cfg["parallelism"] == "single GPU" and cfg["precision"] == "fp32" and cfg["small"] is False
    assert set(cfg) == {"workload", "I", "J", "nnz_train", "edges", "lam", "lam_g", "lr", "parallelism", "l2",
                        "small", "precision"}


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 times the oracle; the other ranks print nothing, exit 0."""
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=120, cwd=root,
                       env=env)
    assert r.returncode == 0 and not r.stdout.strip(), (r.returncode, r.stdout[-500:], r.stderr[-500:])
