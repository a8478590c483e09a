"""Replicas on N ranks (world size 2, gloo on the CPU): the bench's whole-job reduction takes the
slowest rank's time and the sweeps of all ranks, and the rank environment is read as torchrun sets it."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    bench = _load_bench()
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    got_ws, got_rank, got_local = bench.dist_env()
    ms, sweeps = bench.reduce_over_ranks(10.0 + 5.0 * rank, 6 + rank, ws)
    dist.destroy_process_group()
    q.put((rank, got_ws, got_rank, got_local, ms, sweeps))


def test_two_rank_reduction_is_max_time_and_total_sweeps():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    with socket.socket() as s_:
        s_.bind(("127.0.0.1", 0))
        port = s_.getsockname()[1]
    q = mp.Queue()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, got_rank, local, ms, sweeps in out:
        assert (ws, got_rank, local) == (2, rank, rank)
        assert ms == 15.0 and sweeps == 13.0


def test_single_rank_reduction_is_identity():
    bench = _load_bench()
    assert bench.reduce_over_ranks(3.5, 6, 1) == (3.5, 6)
