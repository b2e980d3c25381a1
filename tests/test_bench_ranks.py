"""bench.py on several ranks (replicas only, no collective on the data path),
checked on the CPU with world-size-2 gloo process groups:

* every rank receives the slowest rank's time (the max over ranks);
* the whole-job value counts every rank's replica steps in that time;
* each rank steps its own seeded replica, rank 0 the single-GPU workload;
* under the reference arm the ranks other than 0 exit without work.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        from paper_1203_6208_gb300 import inputs
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")
        value = bench.job_value(ws, 5, ms)
        cfg, _ = inputs.preset("c4", alpha_factor=1.0, n_chains=4)
        R = bench.replica_chains(cfg, rank)
        q.put((rank, ms, value, R.tobytes()))
    finally:
        dist.destroy_process_group()


def test_timing_and_replicas_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, ms, value, R = q.get(timeout=120)
        out[rank] = (ms, value, R)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the max over ranks, on every rank; two replicas x 5 steps in 15 ms
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] == out[1][1] == pytest.approx(2 * 5 / 0.015)
    # each rank its own replica; rank 0 the single-GPU workload's chains
    sys.path.insert(0, ROOT)
    from paper_1203_6208_gb300 import inputs
    cfg, _ = inputs.preset("c4", alpha_factor=1.0, n_chains=4)
    assert out[0][2] != out[1][2]
    assert out[0][2] == inputs.make_chains(cfg).tobytes()


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_value(1, 4, 8.0) == pytest.approx(500.0)


def test_reference_arm_other_ranks_do_nothing(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    args = bench.parse()
    # returns before building or timing the oracle
    assert bench.run_reference(args) is None
