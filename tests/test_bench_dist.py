"""The benchmark's multi-rank logic on CPU: two gloo ranks, barrier, max-over-ranks timing and
the whole-job weak-scaling throughput (each rank processes its own replica; no data exchange)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    bench.barrier(w)
    t = bench.reduce_max(1.0 + rank, w)
    v = bench.weak_scaling_value(1000, w, t)
    q.put((r, w, lr, t, v))
    dist.destroy_process_group()


def test_two_rank_weak_scaling_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    for _, _, _, t, v in res:
        assert t == 2.0 and v == pytest.approx(1000.0)  # 2 ranks x 1000 units in max(1, 2) s


def test_reference_arm_only_rank_zero_works(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(type("A", (), {"workload": "cube", "steps": 1, "warmup": 3, "S": 1})())
    assert capsys.readouterr().out == ""


def test_loglog_interpolation():
    import bench
    y, ext = bench.interp_loglog(1e-3, [1e-2, 1e-4], [1.0, 100.0])
    assert y == pytest.approx(10.0) and not ext
    y, ext = bench.interp_loglog(1e-5, [1e-2, 1e-4], [1.0, 100.0])
    assert y == pytest.approx(1000.0) and ext
