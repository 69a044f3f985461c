"""Helpers for the GPU tests: device KBs from synthetic or fixture KBs, and
oracle comparisons (element by element, bit-exact)."""
from __future__ import annotations

import os
from typing import List, Sequence

import numpy as np

import oracle
import paper_2412_00802_gb300 as H
from synth import kb as K
from synth import programs as P

THREADS = max(1, min(16, os.cpu_count() or 1))


def device_kb(kb: K.KB, flags: int = 0) -> H.DeviceKB:
    return H.DeviceKB.from_synth(kb, flags=flags)


def compare_batch(kb: K.KB, dkb: H.DeviceKB, progs: Sequence[np.ndarray], flags: int = 0,
                  sample: Sequence[int] = None, check_bits: bool = True):
    """Run the batch on the GPU; compare counts (all or a sample) and instance sets with the oracle."""
    flat, offs = P.pack_batch(progs)
    if check_bits:
        counts, bits = dkb.score(flat, offs, flags, out_bits=True)
    else:
        counts = dkb.score(flat, offs, flags)
        bits = None
    idx = list(range(len(progs))) if sample is None else list(sample)
    sub = [progs[i] for i in idx]
    sflat, soffs = P.pack_batch(sub)
    okb = oracle.from_synth(kb)
    oc, osets, errs = oracle.eval_batch(okb, sflat, soffs, threads=THREADS, keep_sets=check_bits)
    assert not errs.any()
    for j, h in enumerate(idx):
        if check_bits:
            got = K.unpack_bits(bits[h], kb.n)
            if not np.array_equal(got, osets[j].astype(bool)):
                bad = np.nonzero(got != osets[j].astype(bool))[0]
                raise AssertionError(f"hypothesis {h} ({P.to_text(P.from_postfix(progs[h]))[:200]}): "
                                     f"{bad.size} individuals differ, first {bad[:8]}")
            # bits past n and padding words are zero
            tail = bits[h].copy()
            assert not (tail[kb.w:]).any()
            if kb.n % 32:
                assert not (int(tail[kb.w - 1]) >> (kb.n % 32))
        assert np.array_equal(counts[h].astype(np.int64), oc[j]), (h, counts[h], oc[j])
    return counts, bits
