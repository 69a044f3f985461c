"""Parity at the workloads' full sizes (sampled): the 10,000,000-individual
single-hypothesis workload (32 Zipf(2.1) roles, ~2.6 G assertions) and the
4,000,000-individual search workload (64 Zipf(2.3) roles, planted examples).
The GPU evaluates in the configuration the benchmark uses; the oracle
recomputes a sample of the hypotheses over every individual."""
import os

import numpy as np
import pytest

import oracle
from synth import hyps, kb as K, programs as P
from tests.gpu_util import THREADS

pytestmark = pytest.mark.gpu


def _check_sample(kb, dkb, progs, sample):
    import paper_2412_00802_gb300 as H
    flat, offs = P.pack_batch(progs)
    counts = dkb.score(flat, offs)
    okb = oracle.from_synth(kb)
    sub = [progs[i] for i in sample]
    sflat, soffs = P.pack_batch(sub)
    oc, osets, errs = oracle.eval_batch(okb, sflat, soffs, threads=THREADS, keep_sets=True)
    assert not errs.any()
    for j, h in enumerate(sample):
        got = K.unpack_bits(dkb.eval(progs[h]), kb.n)          # one at a time, as the latency workload runs
        assert np.array_equal(got, osets[j].astype(bool)), h
        assert np.array_equal(counts[h].astype(np.int64), oc[j]), h
    return counts


def test_single_hypothesis_workload_full_size():
    import paper_2412_00802_gb300 as H
    kb = K.generate(K.CONFIGS["large"])
    dkb = H.DeviceKB.from_synth(kb)
    progs = hyps.chain_hyps(kb, 2002, 64)
    _check_sample(kb, dkb, progs, [0, 13, 31, 63])


def test_search_workload_kb_full_size():
    import paper_2412_00802_gb300 as H
    kb = K.generate(K.CONFIGS["search"])
    dkb = H.DeviceKB.from_synth(kb)
    progs = hyps.batch_hyps(kb, 5005, 0, 512, lmax=24, dmax=6)
    _check_sample(kb, dkb, progs, [0, 100, 333, 511])
