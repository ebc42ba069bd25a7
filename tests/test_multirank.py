"""The multi-rank path of bench.py on CPU: two gloo ranks (weak scaling, one
independently seeded box per rank, max-over-ranks time, summed work)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t, c = bench.combine_ranks(ms=[3.0, 5.0][rank], cells=[100.0, 250.0][rank], device="cpu")
    st = bench.headline_state(rank)
    dist.barrier()
    q.put((rank, t, c, float(st.pos.sum())))
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_and_seed_independently():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, c0, s0), (r1, t1, c1, s1) = out
    assert t0 == t1 == 5.0                 # the slowest rank's time
    assert c0 == c1 == 350.0               # work of all ranks
    assert s0 != s1                        # every rank evaluates its own box


def test_single_process_combine_is_identity():
    import bench
    assert bench.combine_ranks(2.5, 10.0, "cpu") == (2.5, 10.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(Args, ws=2, rank=1)
    assert capsys.readouterr().out == ""
