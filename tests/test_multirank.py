"""Replicas on several ranks (the bench under torchrun): the whole-job rate
sums the instances every rank converged and divides by the slowest rank's
time; ranks take disjoint seeds.  Two gloo ranks on CPU."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [100.0, 125.0][rank]
    conv = [300, 298][rank]
    out[rank] = bench.job_value(dist, torch.device("cpu"), ms, conv, 3)
    dist.barrier()
    dist.destroy_process_group()


def test_job_value_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        procs = [mp.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(world):
            ms, conv, value = out[r]
            assert ms == 125.0 and conv == 598
            assert abs(value - 598 * 3 / 0.125) < 1e-9


def test_ranks_take_disjoint_instances():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    seeds = [set(range(bench.rank_seed(r), bench.rank_seed(r) + 1216)) for r in range(8)]
    for a in range(8):
        for b in range(a + 1, 8):
            assert not seeds[a] & seeds[b]
    ms, conv, value = bench.job_value(None, None, 200.0, 304, 3)
    assert (ms, conv) == (200.0, 304) and abs(value - 304 * 3 / 0.2) < 1e-9
