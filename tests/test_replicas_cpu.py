"""The multi-GPU form's host logic on two gloo ranks (CPU): disjoint item shards, the
max-over-ranks time and the whole-job rate.  The solver itself has no exchange step,
so this is the whole N > 1 path apart from the per-rank GPU work."""

import os
import socket

import numpy as np
import pytest

from paper_2208_02783_gb300 import replicas

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reps = [1, 4, 6]
        for step in range(3):
            mine = replicas.step_items(5, reps, 40, 8, step, rank, world)
            gathered = [None] * world
            dist.all_gather_object(gathered, [a.tolist() for a in mine])
            triples = [t for g in gathered for t in zip(*g)]
            assert len(triples) == 8 * world
            assert len(set(triples)) == len(triples)  # disjoint across ranks, distinct
            whole = replicas.step_items(5, reps, 40, 8 * world, step, 0, 1)
            assert set(triples) == set(zip(*[a.tolist() for a in whole]))
            assert all(k in reps for _, k, _ in triples)
        t = replicas.max_over_ranks(10.0 + rank)
        assert t == 10.0 + world - 1
        assert replicas.whole_job_rate(8, world, t) == pytest.approx(8 * world / t)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp

    mp.start_processes(_rank_main, args=(2, _free_port()), nprocs=2, join=True, start_method="spawn")


def test_single_process_fallbacks():
    assert replicas.max_over_ranks(3.5) == 3.5
    e, k, c = replicas.step_items(4, [0, 2], 10, 6, 0, 0, 1)
    assert len(e) == len(k) == len(c) == 6
    assert np.all((e >= 0) & (e < 4)) and np.all((c >= 0) & (c < 10)) and set(k) <= {0, 2}
    with pytest.raises(ValueError):
        replicas.step_items(1, [0], 3, 4, 0, 0, 1)
    with pytest.raises(ValueError):
        replicas.whole_job_rate(1, 1, 0.0)
