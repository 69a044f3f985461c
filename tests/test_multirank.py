"""The multi-rank (torchrun) path of bench.py on CPU with gloo, world size 2:
hypothesis batches are sharded across ranks with no overlap, each rank's
evaluation is independent (no data-path collective), and the timed region is
reduced as the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from synth import kb as K, programs as P
    warm, timed = bench.shard_batches(rank, world, 2, 3)
    ids = [None] * world
    td.all_gather_object(ids, warm + timed)
    # each rank scores its own shard (oracle as the stand-in evaluator)
    kb = K.generate(K.CONFIGS["small"].scaled(800, seed=5))
    okb = oracle.from_synth(kb)
    counts = []
    for b in timed:
        progs = bench.make_batch(kb, b, count=8)
        flat, offs = P.pack_batch(progs)
        c, _, errs = oracle.eval_batch(okb, flat, offs)
        assert not errs.any()
        counts.append(c)
    elapsed = 1.0 + rank          # rank 1 is the slow one
    mx = bench.max_over_ranks(elapsed)
    out[rank] = (ids, mx, np.concatenate(counts).sum())
    td.destroy_process_group()


def test_two_ranks_shard_and_max_time():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    ids0, mx0, _ = out[0]
    ids1, mx1, _ = out[1]
    assert ids0 == ids1
    flat = [b for r in ids0 for b in r]
    assert len(flat) == len(set(flat)) == world * 5, "batches are disjoint across ranks"
    assert mx0 == mx1 == 2.0
