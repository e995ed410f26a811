"""The multi-GPU form (independent replicas, one per rank) exercised on CPU
with two gloo ranks: each rank runs its own oracle run with its own Philox
stream; timings combine as the maximum over ranks; no data-path collective."""
import os
import socket
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2405_16551_gb300 import problems, replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rid = replicas.replica_run_id(3, rank)
        o = problems.shift(6, seed=1)
        t0 = time.perf_counter()
        X, f, g, ev, _ = oracle.run(16, 6, 0.5, 0.9, -100, 100, 1, o, None, seed=1, max_generations=25,
                                    target_error=0.0, run_id=rid)
        dt = time.perf_counter() - t0 + 0.05 * rank  # ranks differ in time
        tmax = replicas.max_over_ranks([dt], dist)[0]
        q.put((rank, rid, X, g, ev, dt, tmax, replicas.job_rate(16 * 25, world, tmax)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, rid, X, g, ev, dt, tmax, rate = q.get(timeout=120)
        out[rank] = (rid, X, g, ev, dt, tmax, rate)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # each rank ran its own stream: the same as a single-process run of that stream
    o = problems.shift(6, seed=1)
    for rank, (rid, X, g, ev, dt, tmax, rate) in out.items():
        assert rid == 3 + rank and g == 25 and ev == 16 * 26
        Xs, *_ = oracle.run(16, 6, 0.5, 0.9, -100, 100, 1, o, None, seed=1, max_generations=25, target_error=0.0,
                            run_id=rid)
        assert np.array_equal(X, Xs)
    assert not np.array_equal(out[0][1], out[1][1])
    # the job time is the slowest rank's, and every rank agrees on it
    tmax = max(v[4] for v in out.values())
    assert all(v[5] == pytest.approx(tmax) for v in out.values())
    assert all(v[6] == pytest.approx(world * 16 * 25 / tmax) for v in out.values())


def test_replica_run_ids():
    assert replicas.replica_run_id(0, 5) == 5
    with pytest.raises(ValueError):
        replicas.replica_run_id((1 << 20) - 1, 1)
    assert replicas.max_over_ranks([1.5, 2.0]) == [1.5, 2.0]
    assert replicas.job_rate(100, 4, 2.0) == 200.0
