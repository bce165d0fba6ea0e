"""The multi-process path of the benchmark on CPU (gloo, world size 2): each rank
decomposes its own replica (the method needs no data-path collective, "replicas
only"), the job's step time is the maximum over ranks, and the whole-job value
counts every rank's units. The ranks run the FP64 oracle on a tiny tensor as
their per-rank work, so nothing here needs a GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, fake_ms, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    from oracle import tucker_oracle as O
    try:
        w, r, _ = bench._dist()
        assert (w, r) == (world, rank)
        # per-rank work: an independent replica (its own seed)
        p = W.planted(W.SEED_BASE + 90 + rank, (10, 9, 8), (3, 3, 2), "gauss", 1e-2, dtype=np.float64)
        res = O.st_hosvd_als(p.A, (3, 3, 2), eta=1e-10, seed=1)
        ms = bench._job_ms(fake_ms[rank], dist, device="cpu")
        value = bench._job_value(world, ms)
        out.put((rank, ms, value, float(O.rel_error(p.A, res.G, res.U))))
    finally:
        dist.destroy_process_group()


def test_two_rank_job_time_and_value():
    world = 2
    fake_ms = [2.5, 4.0]   # the slower rank sets the step time
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, fake_ms, out)) for r in range(world)]
    for pr in procs:
        pr.start()
    results = [out.get(timeout=120) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, ms, value, rel in results:
        assert ms == max(fake_ms)
        assert value == pytest.approx(world * 1e3 / max(fake_ms))
        assert 0.0 < rel < 0.05


def test_single_process_job_time_is_own():
    import bench
    assert bench._job_ms(3.0, None) == 3.0
    assert bench._job_value(1, 2.0) == pytest.approx(500.0)
