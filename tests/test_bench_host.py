"""Host-side logic of bench.py: the replica aggregation and the max-over-ranks
reduction, run as two gloo ranks on the CPU (no GPU involved)."""

import os
import socket

import pytest

import bench

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, queue):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        bench.barrier()
        # each rank timed a different elapsed time; every rank must see the max
        m = bench.reduce_max(10.0 * (rank + 1))
        agg = bench.aggregate(m, steps=5, npts_per_rank=1000, world=w)
        queue.put((r, w, lr, m, agg))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_and_aggregate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1]
    for r, w, lr, m, agg in out:
        assert w == 2 and lr == r
        assert m == 20.0
        assert agg["ms_per_step"] == pytest.approx(4.0)
        # 4 ms per step over 2 x 1000 points = 2000 ns per point
        assert agg["value"] == pytest.approx(2000.0)


def test_single_process_helpers_are_identities(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.reduce_max(3.5) == 3.5
    bench.barrier()
    a = bench.aggregate(100.0, steps=10, npts_per_rank=10**6, world=1)
    assert a["ms_per_step"] == 10.0 and a["value"] == pytest.approx(10.0)


def test_work_model_and_peak():
    flops, nbytes = bench.stage_work("y_forward", 512, 384, 384)
    assert nbytes == 16.0 * 512 * 384 * 384
    assert flops == pytest.approx(256 * 384 * 5 * 384 * 8.584962500721156)
    assert bench.fp64_peak_tflops() == pytest.approx(1.25856)


def test_reference_arm_only_rank0_prints(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3", "--gpus", "2"]) == 0
    assert capsys.readouterr().out == ""
