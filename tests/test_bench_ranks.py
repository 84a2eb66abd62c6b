"""The multi-rank parts of bench.py on CPU (gloo, world size 2): the step times are
reduced to their maximum over ranks on every rank, and the reference arm runs on rank
0 only (the other ranks exit without work or output)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5 * rank], "cpu")
        out[rank] = got
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0] == out[1] == [2.0, 10.0, 0.5]


def test_reference_arm_only_on_rank_zero(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = type("Args", (), {"steps": 1, "warmup": 0, "seed": 0, "gpus": 2})()
    bench.run_reference(args, 1)
    assert capsys.readouterr().out == ""
