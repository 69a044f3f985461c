"""The multi-device split of hypothesis batches (paper_2412_00802_gb300/schedule.py): the
paper's probe-timed static ratio split (Section V) and a dynamic host work queue, on CPU
ranks over gloo (world sizes 2 and 4).  Each rank scores its share with the oracle as a
stand-in evaluator and a planted slowdown; every hypothesis must be scored exactly once and
the gathered counts must equal one process's.  No GPU is involved: the hardware scaling curve
of this split is not measured here."""
import os
import socket
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2412_00802_gb300 import schedule as SC


def test_split_by_rates_tiles_the_batch_in_proportion():
    rng = np.random.default_rng(1)
    for _ in range(300):
        R = int(rng.integers(1, 9))
        rates = rng.uniform(0, 10, R) * (rng.uniform(size=R) > 0.2)
        H = int(rng.integers(0, 5000))
        g = int(rng.choice([1, 8, 64]))
        rs = SC.split_by_rates(rates, H, g)
        assert len(rs) == R and rs[0][0] == 0 and rs[-1][1] == H
        assert all(a <= b for a, b in rs) and all(rs[k][1] == rs[k + 1][0] for k in range(R - 1))
        eff = rates if rates.sum() > 0 else np.ones(R)
        units = -(-H // g)
        for (a, b), r in zip(rs, eff):
            n_units = -(-(b - a) // g) if b > a else 0
            assert abs(n_units - r / eff.sum() * units) < 1 + 1e-9
            if r == 0 and rates.sum() > 0:
                assert a == b
    assert SC.split_by_rates([1, 3], 8) == [(0, 2), (2, 8)]
    assert SC.split_by_rates([0, 0, 0], 7) == [(0, 3), (3, 5), (5, 7)]
    assert SC.split_by_rates([2, 1], 100, 64) == [(0, 64), (64, 100)]
    for bad in ([], [-1.0, 2.0], [float("nan")]):
        with pytest.raises(ValueError):
            SC.split_by_rates(bad, 10)


def test_probe_program_is_the_five_concept_conjunction():
    from synth import programs as P
    assert P.to_text(P.from_postfix(SC.probe_program(100))) == "(and (and (and (and A0 A1) A2) A3) A4)"
    assert P.to_text(P.from_postfix(SC.probe_program(2))) == "(and A0 A1)"


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, store_port, slow, out):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from synth import hyps, kb as K, programs as P
    kb = K.generate(K.CONFIGS["small"].scaled(600, seed=9))
    okb = oracle.from_synth(kb)
    progs = hyps.batch_hyps(kb, 31, 0, 240)
    H = len(progs)
    delay = 0.002 * slow[rank]        # this rank's device is slow[rank] times slower

    def score(b, e):
        flat, offs = P.pack_batch(progs[b:e])
        c, _, errs = oracle.eval_batch(okb, flat, offs)
        assert not errs.any()
        time.sleep(delay * (e - b))
        return c

    def probe():
        oracle.eval_program(okb, SC.probe_program(kb.n_concepts))
        time.sleep(delay * 8)

    # the paper's static split: probe, shares from the rates, one contiguous range per rank
    rates = SC.probe_rates(probe, reps=3, warmup=1)
    b, e = SC.split_by_rates(rates, H, 8)[rank]
    static = SC.gather_counts(np.arange(b, e), score(b, e), H)
    # the dynamic host queue: chunks of 16 to whichever rank is free
    store = td.TCPStore("127.0.0.1", store_port, world, rank == 0)
    q = SC.DynamicQueue(store, "batch0", H, 16)
    td.barrier()                      # every rank reaches the queue together
    idx, cs = [], []
    while (r := q.next()) is not None:
        idx.append(np.arange(*r))
        cs.append(score(*r))
    dyn = SC.gather_counts(np.concatenate(idx) if idx else np.zeros(0, np.int64),
                           np.concatenate(cs) if cs else np.zeros((0, 4), np.int64), H, dst=0)
    # a share scored twice is refused
    dup_err = None
    try:
        SC.gather_counts(np.arange(0, 4), score(0, 4), H)
    except RuntimeError as ex:
        dup_err = str(ex)
    out[rank] = (rates, (b, e), static, dyn, int(sum(len(i) for i in idx)), dup_err)
    td.destroy_process_group()


@pytest.mark.parametrize("world,slow", [(2, (1, 3)), (4, (1, 1, 2, 4))])
def test_static_and_dynamic_splits_score_every_hypothesis_once(world, slow):
    import oracle
    from synth import hyps, kb as K, programs as P
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), _free_port(), slow, out), nprocs=world, join=True)
    kb = K.generate(K.CONFIGS["small"].scaled(600, seed=9))
    want, _, _ = oracle.eval_batch(oracle.from_synth(kb), *P.pack_batch(hyps.batch_hyps(kb, 31, 0, 240)))
    shares = [out[r][1][1] - out[r][1][0] for r in range(world)]
    assert sum(shares) == 240
    fast, slowest = int(np.argmin(slow)), int(np.argmax(slow))
    assert shares[fast] > shares[slowest], shares            # the slower device gets a smaller share
    took = [out[r][4] for r in range(world)]
    assert sum(took) == 240 and took[fast] > took[slowest], took
    for r in range(world):
        assert np.array_equal(out[r][2], want)                # static split, gathered on every rank
        assert out[r][5] is not None and "more than one" in out[r][5]
    assert np.array_equal(out[0][3], want)                     # dynamic queue, gathered on rank 0
    assert all(out[r][3] is None for r in range(1, world))
