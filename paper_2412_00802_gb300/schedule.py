"""Splitting hypothesis batches across devices (one process per GPU).

The paper's multi-device scheduler (Section V) times a probe, a conjunction of
five concepts, on every device, gives each device a fixed share of every
batch in proportion to the speed it measured, and gathers the coverage counts
of every share.  Its evaluation (Section VI) finds that this static split stops
scaling once batches grow past about a thousand hypotheses, because a share
fixed by one probe does not follow what the hypotheses actually cost.  Both
ways of splitting are here, over torch.distributed (gloo or NCCL) and its
key-value store:

* ``probe_rates`` / ``split_by_rates``: the paper's static ratio split.  Every
  rank times the probe on its own device, the rates are all-gathered, and rank
  r evaluates a contiguous range of the batch whose length is proportional to
  its rate (largest-remainder rounding, so the ranges tile the batch exactly).
* ``DynamicQueue``: the alternative, a host work queue.  A shared counter in
  the process group's store hands out fixed-size chunks of the batch; a rank
  takes the next chunk whenever it finishes one, so a slower device simply
  takes fewer chunks.
* ``gather_counts``: every rank's (hypothesis index, counts) pairs to every
  rank (or rank 0), assembled into the batch's [H][4] counts, with a check that
  each hypothesis was scored exactly once.

Hypotheses are independent, so no collective touches the data path: the only
exchanges are the rates, the queue counter and the final counts.
"""
from __future__ import annotations

import time
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np


def _dist():
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()):
        return None
    return td


def split_by_rates(rates: Sequence[float], H: int, granularity: int = 1) -> List[Tuple[int, int]]:
    """Contiguous ranges [begin, end) of a batch of H hypotheses, one per rank, with lengths in
    proportion to the ranks' rates, in units of `granularity` hypotheses (the last unit may be
    partial).  Largest-remainder rounding: the ranges tile [0, H) exactly, and a rank's length
    differs from its exact share by less than one unit.  A rank with rate 0 gets nothing; if
    every rate is 0 the batch is split evenly."""
    r = np.asarray(rates, np.float64)
    if r.ndim != 1 or r.size == 0:
        raise ValueError("one rate per rank is needed")
    if np.any(~np.isfinite(r)) or np.any(r < 0):
        raise ValueError("rates must be finite and non-negative")
    if granularity < 1:
        raise ValueError("granularity must be >= 1")
    if r.sum() <= 0:
        r = np.ones_like(r)
    units = -(-H // granularity)                     # ceil
    exact = r / r.sum() * units
    n = np.floor(exact).astype(np.int64)
    left = units - int(n.sum())
    order = np.argsort(-(exact - n), kind="stable")  # largest remainders first, ties to the lower rank
    n[order[:left]] += 1
    out, at = [], 0
    for k in n:
        b = min(H, at * granularity)
        at += int(k)
        out.append((b, min(H, at * granularity)))
    return out


def probe_rates(probe: Callable[[], None], reps: int = 5, warmup: int = 2,
                timer: Callable[[], float] = time.perf_counter) -> List[float]:
    """Every rank runs `probe` (one evaluation of the probe conjunction on its own device, returning
    once it is done) warmup + reps times and reports reps / seconds; the rates of all ranks are
    all-gathered (without torch.distributed: this process's rate alone)."""
    for _ in range(warmup):
        probe()
    t0 = timer()
    for _ in range(reps):
        probe()
    dt = max(timer() - t0, 1e-12)
    rate = reps / dt
    td = _dist()
    if td is None:
        return [rate]
    got = [None] * td.get_world_size()
    td.all_gather_object(got, rate)
    return [float(x) for x in got]


class DynamicQueue:
    """A host work queue over the process group's key-value store: chunks of `chunk` hypotheses
    of a batch of H, handed out in order to whichever rank asks next.

    Every rank constructs it with the same name (one name per batch; the store's counter of that
    name starts at 0) and calls ``next()`` until it returns None.  ``store.add`` is atomic, so
    each chunk goes to exactly one rank."""

    def __init__(self, store, name: str, H: int, chunk: int):
        if chunk < 1:
            raise ValueError("chunk must be >= 1")
        self.store, self.key, self.H, self.chunk = store, f"hedl_queue/{name}", H, chunk

    def next(self) -> Optional[Tuple[int, int]]:
        k = int(self.store.add(self.key, 1)) - 1      # this rank's ticket
        b = k * self.chunk
        if b >= self.H:
            return None
        return b, min(self.H, b + self.chunk)


def gather_counts(index: np.ndarray, counts: np.ndarray, H: int, dst: Optional[int] = None) -> Optional[np.ndarray]:
    """Assemble a batch's coverage counts from every rank's share.  index: int64[k] the
    hypotheses this rank scored, counts: [k][4] their (TP, FP, FN, TN).  Returns the [H][4]
    counts on every rank (dst None) or on rank dst only (None elsewhere).  Raises if a
    hypothesis was scored by no rank or by more than one."""
    index = np.asarray(index, np.int64).reshape(-1)
    counts = np.asarray(counts).reshape(-1, 4)
    if index.size != counts.shape[0]:
        raise ValueError("one row of counts per index")
    td = _dist()
    parts = [(index, counts)]
    if td is not None:
        parts = [None] * td.get_world_size()
        if dst is None:
            td.all_gather_object(parts, (index, counts))
        else:
            td.gather_object((index, counts), parts if td.get_rank() == dst else None, dst=dst)
            if td.get_rank() != dst:
                return None
    seen = np.zeros(H, np.int64)
    out = np.zeros((H, 4), np.int64)
    for idx, c in parts:
        if idx.size and (idx.min() < 0 or idx.max() >= H):
            raise ValueError("a hypothesis index lies outside the batch")
        np.add.at(seen, idx, 1)
        out[idx] = c
    if np.any(seen != 1):
        raise RuntimeError(f"{int((seen == 0).sum())} hypotheses scored by no rank, "
                           f"{int((seen > 1).sum())} by more than one")
    return out


def probe_program(n_concepts: int) -> np.ndarray:
    """The paper's probe: a conjunction of five concepts (the first five, or all when the KB has
    fewer), as a postfix program (ATOM = op 1 with the concept id in bits 16..31, AND = op 5)."""
    k = max(1, min(5, n_concepts))
    prog = [1]
    for c in range(1, k):
        prog += [1 | (c << 16), 5]
    return np.array(prog, np.uint64)
