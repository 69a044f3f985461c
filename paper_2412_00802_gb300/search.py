"""Refinement beam search over hypotheses, evaluated exactly on the GPU.

Each step refines the beam into candidates (a caller-supplied seeded
generator), puts every candidate in canonical form (AND / OR operands sorted
by their canonical instruction bytes), drops duplicates, scores candidates
exactly in batches through the library (hedl_plan_batch / hedl_plan_execute:
one persistent, graph-replayed launch per batch), and keeps the best `width`
of old beam plus candidates in the total order
    accuracy desc, F1 desc, length asc, canonical bytes asc, position asc
(old beam members first, then candidates in generation order).

With a surrogate, candidates are evaluated in the order of their predicted
scores; each candidate's encoding carries, as its prior inputs, the exact
accuracy and F1 of the beam member it refines (candidate k refines member
k mod |beam|, the generator's convention, unless `parent_of` says
otherwise).  With pruning, only the predicted top fraction is evaluated, from
the step after `warmup_steps` on.  With `adaptive`, candidates are
evaluated in predicted order one batch at a time, and a step ends at the
first batch none of whose candidates would enter the beam.  With `online_epochs`, the surrogate is
trained after every step on the latest `online_window` candidates scored
exactly (with their priors), so it learns the search's own distribution.  Without pruning
the surrogate changes only the evaluation order, so the final beam is the
exhaustive search's.  Scores always come from exact evaluation.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

from . import hedl_canonical_batch


def canonical(prog: Sequence[int]) -> np.ndarray:
    """Canonical postfix (hedl_canonical_batch): every AND / OR has its operands in ascending byte order."""
    p = np.ascontiguousarray(prog, np.uint64)
    return hedl_canonical_batch(p, np.array([0, p.size], np.uint32))


@dataclass
class Entry:
    prog: np.ndarray        # canonical postfix
    acc: float
    f1: float
    counts: Tuple[int, int, int, int]

    def key(self, pos: int):
        return (-self.acc, -self.f1, len(self.prog), self.prog.tobytes(), pos)


def scores(counts: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    c = counts.astype(np.float64)
    tp, fp, fn, tn = c[:, 0], c[:, 1], c[:, 2], c[:, 3]
    tot = tp + fp + fn + tn
    acc = np.where(tot > 0, (tp + tn) / np.where(tot > 0, tot, 1), 0.0)
    den = 2 * tp + fp + fn
    f1 = np.where(den > 0, 2 * tp / np.where(den > 0, den, 1), 0.0)
    return acc, f1


def beam_update(beam: List[Entry], cands: List[Entry], width: int) -> List[Entry]:
    pool = list(beam) + list(cands)
    order = sorted(range(len(pool)), key=lambda i: pool[i].key(i))
    out, seen = [], set()
    for i in order:
        b = pool[i].prog.tobytes()
        if b in seen:
            continue
        seen.add(b)
        out.append(pool[i])
        if len(out) == width:
            break
    return out


@dataclass
class StepLog:
    step: int
    candidates: int
    evaluated: int
    best_acc: float
    seconds: float
    events: List[Tuple[float, float]] = field(default_factory=list)   # (time since start, best acc so far)
    times: dict = field(default_factory=dict)   # seconds in refine / surrogate / eval / learn


class BeamSearch:
    def __init__(self, dkb, refine: Callable[[List[np.ndarray], int, int], List[np.ndarray]], width: int = 64,
                 per_step: int = 8192, batch: int = 2048, surrogate=None, keep_fraction: Optional[float] = None,
                 parent_of: Optional[Callable[[int, int], int]] = None, online_epochs: int = 0,
                 warmup_steps: int = 0, online_lr: float = 1e-3, adaptive: bool = False,
                 online_window: int = 1 << 16):
        self.dkb = dkb
        self.refine = refine
        self.width = width
        self.per_step = per_step
        self.batch = batch
        self.surrogate = surrogate
        self.keep = keep_fraction
        self.parent_of = parent_of or (lambda k, n_beam: k % n_beam)
        self.online_epochs = online_epochs
        self.warmup_steps = warmup_steps
        self.online_lr = online_lr
        self.adaptive = adaptive
        self.online_window = online_window
        self._seen_X, self._seen_T = [], []

    def _score(self, progs: List[np.ndarray]):
        from .surrogate import exact_scores
        from . import hedl_sync_status
        flat = np.concatenate(progs).astype(np.uint64)
        offs = np.zeros(len(progs) + 1, np.uint32)
        np.cumsum([len(p) for p in progs], out=offs[1:])
        counts, _ = exact_scores(self.dkb, flat, offs)
        return counts.cpu().numpy().view(np.uint32)

    def run(self, start: List[np.ndarray], steps: int):
        t0 = time.perf_counter()
        beam = [Entry(canonical(p), 0.0, 0.0, (0, 0, 0, 0)) for p in start]
        c = self._score([e.prog for e in beam])
        a, f = scores(c)
        beam = [Entry(e.prog, float(a[i]), float(f[i]), tuple(int(x) for x in c[i])) for i, e in enumerate(beam)]
        beam = beam_update(beam, [], self.width)
        logs = []
        best = beam[0].acc
        for s in range(1, steps + 1):
            ts = time.perf_counter()
            tm = {}
            raw = self.refine([e.prog for e in beam], s, self.per_step)
            if isinstance(raw, tuple):       # (flat instructions, offsets)
                rflat, roffs = np.asarray(raw[0], np.uint64), np.asarray(raw[1], np.int64)
            else:
                rflat = np.concatenate(raw).astype(np.uint64) if len(raw) else np.zeros(0, np.uint64)
                roffs = np.zeros(len(raw) + 1, np.int64)
                np.cumsum([len(p) for p in raw], out=roffs[1:])
            canon = hedl_canonical_batch(rflat, roffs.astype(np.uint32))
            cands, parents, seen = [], [], {e.prog.tobytes() for e in beam}
            for k in range(len(roffs) - 1):
                cp = canon[roffs[k]:roffs[k + 1]]
                b = cp.tobytes()
                if b not in seen:
                    seen.add(b)
                    cands.append(cp)
                    parents.append(self.parent_of(k, len(beam)))
            order = list(range(len(cands)))
            X = None
            t1 = time.perf_counter()
            tm["refine"] = t1 - ts
            if self.surrogate is not None and cands:
                flat = np.concatenate(cands).astype(np.uint64)
                offs = np.zeros(len(cands) + 1, np.uint32)
                np.cumsum([len(p) for p in cands], out=offs[1:])
                prior = np.array([[beam[j].acc, beam[j].f1] for j in parents], np.float32)
                X = self.surrogate.encode(flat, offs, prior)
                Y = self.surrogate.predict(X).cpu().numpy()
                order = sorted(order, key=lambda i: (-Y[i, 0], -Y[i, 1], i))
                if self.keep is not None and s > self.warmup_steps:
                    order = order[:max(1, int(round(self.keep * len(order))))]
            t2 = time.perf_counter()
            tm["surrogate"] = t2 - t1
            entries = [None] * len(cands)
            log = StepLog(s, len(cands), len(order), best, 0.0)
            adaptive = self.adaptive and X is not None and s > self.warmup_steps
            evaluated = []
            for b0 in range(0, len(order), self.batch):
                ids = order[b0:b0 + self.batch]
                if adaptive:   # the width-th best key before this batch
                    pool = [e.key(i) for i, e in enumerate(beam)] + \
                           [entries[i].key(len(beam) + i) for i in evaluated]
                    thr = sorted(pool)[self.width - 1] if len(pool) >= self.width else None
                c = self._score([cands[i] for i in ids])
                a, f = scores(c)
                for j, i in enumerate(ids):
                    entries[i] = Entry(cands[i], float(a[j]), float(f[j]), tuple(int(x) for x in c[j]))
                evaluated += ids
                best = max(best, float(a.max()) if len(a) else best)
                log.events.append((time.perf_counter() - t0, best))
                # predicted order: a batch none of whose candidates would enter the beam ends the step
                if adaptive and thr is not None and not any(entries[i].key(len(beam) + i) < thr for i in ids):
                    break
            order = evaluated
            log.evaluated = len(evaluated)
            t3 = time.perf_counter()
            tm["eval"] = t3 - t2
            if self.online_epochs and X is not None:
                self._learn(X, order, entries)
            tm["learn"] = time.perf_counter() - t3
            log.times = tm
            beam = beam_update(beam, [e for e in entries if e is not None], self.width)
            log.best_acc = beam[0].acc
            log.seconds = time.perf_counter() - ts
            logs.append(log)
        return beam, logs

    def _learn(self, X, evaluated: List[int], entries: List[Entry]):
        """Train the surrogate on the latest `online_window` candidates scored exactly."""
        torch = self.surrogate.torch
        idx = torch.tensor(evaluated, dtype=torch.int64, device=X.device)
        self._seen_X.append(X.index_select(0, idx))
        self._seen_T.append(torch.tensor([[entries[i].acc, entries[i].f1] for i in evaluated], dtype=torch.float32,
                                         device=X.device))
        Xa, Ta = torch.cat(self._seen_X), torch.cat(self._seen_T)
        if Xa.shape[0] > self.online_window:
            Xa, Ta = Xa[-self.online_window:].contiguous(), Ta[-self.online_window:].contiguous()
            self._seen_X, self._seen_T = [Xa], [Ta]
        batch = min(1024, Xa.shape[0])
        self.surrogate.train(Xa, Ta, epochs=self.online_epochs, batch=batch, lr=self.online_lr,
                             seed=len(self._seen_X), tail_weight=None, schedule="const")
