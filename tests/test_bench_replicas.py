"""The multi-GPU form of the benchmark is N independent replicas (one droplet
per rank, no collective on the data path); its host logic -- the slowest
replica sets the time, whole-job rates, per-rank seeds, the reference arm on
rank 0 only -- runs here as world-size-2 gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w, _ = bench._dist()
        t = bench.reduce_max_over_ranks(10.0 + 5.0 * rank, w, "cpu")
        sc = bench._scenario(600, r)
        out[rank] = (r, w, t, sc.seed, sc.n)
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_own_seeds():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, t, seed, n) in res.items():
        assert (r, w) == (rank, world)
        assert t == 15.0              # max over ranks of 10 and 15 ms
        assert seed == rank and n == 600


def test_replica_rates_scale_with_world_size():
    import bench
    p1, s1 = bench.replica_rates(1, 1000, 2.0)
    p2, s2 = bench.replica_rates(2, 1000, 2.0)
    assert p1 == 1000 * 999 / 2e-3 and s1 == 1000 / 2e-3
    assert p2 == 2 * p1 and s2 == 2 * s1
    assert bench.reduce_max_over_ranks(3.5, 1, "cpu") == 3.5


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(argparse.Namespace(n=1000, steps=1, warmup=0))
    assert capsys.readouterr().out == ""
