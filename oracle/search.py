"""Oracle of the refinement beam search (TEST INFRASTRUCTURE): the plain
exhaustive path.  Every candidate is scored by the C oracle; the beam keeps
the best `width` of old beam plus new candidates in the total order
accuracy desc, F1 desc, length asc, canonical program bytes asc, position asc
(old beam first, then candidates in generation order), where the canonical
form orders the two operands of every AND / OR by their canonical bytes and
duplicates (equal canonical bytes) count once.  Written independently of the
GPU library's search; only the candidate generator (synth.refine) is shared,
as an input generator."""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import numpy as np

import oracle

_LEAF, _UNARY, _BINARY = (1, 2, 3, 12, 13, 14), (4, 7, 8, 9, 10, 11), (5, 6)


def _tree(prog: Sequence[int]):
    st = []
    for w in prog:
        w = int(w)
        op = w & 0xFF
        if op in _LEAF:
            st.append((w, []))
        elif op in _UNARY:
            st.append((w, [st.pop()]))
        else:
            y = st.pop()
            x = st.pop()
            st.append((w, [x, y]))
    return st[0]


def _emit(t) -> List[int]:
    w, kids = t
    parts = [_emit(k) for k in kids]
    if (w & 0xFF) in _BINARY:
        parts.sort(key=lambda p: np.array(p, np.uint64).tobytes())
    return [x for p in parts for x in p] + [w]


def canonical(prog: Sequence[int]) -> bytes:
    return np.array(_emit(_tree(prog)), np.uint64).tobytes()


def _key(bts: bytes, acc: float, f1: float, pos: int):
    return (-acc, -f1, len(bts) // 8, bts, pos)


def exhaustive(okb, refine: Callable[[List[np.ndarray], int, int], List[np.ndarray]], start: List[np.ndarray],
               steps: int, width: int, per_step: int, threads: int = 8) -> List[Tuple[bytes, Tuple[int, ...]]]:
    def score(progs_bytes: List[bytes]):
        progs = [np.frombuffer(b, np.uint64) for b in progs_bytes]
        flat = np.concatenate(progs)
        offs = np.zeros(len(progs) + 1, np.int64)
        np.cumsum([len(p) for p in progs], out=offs[1:])
        c, _, errs = oracle.eval_batch(okb, flat, offs, threads=threads)
        assert not errs.any()
        acc, f1 = oracle.accuracy_f1(c)
        return c, acc, f1

    def update(pool):  # pool: list of (bytes, acc, f1, counts)
        order = sorted(range(len(pool)), key=lambda i: _key(pool[i][0], pool[i][1], pool[i][2], i))
        out, seen = [], set()
        for i in order:
            if pool[i][0] in seen:
                continue
            seen.add(pool[i][0])
            out.append(pool[i])
            if len(out) == width:
                break
        return out

    b0 = [canonical(p) for p in start]
    c, a, f = score(b0)
    beam = update([(b0[i], float(a[i]), float(f[i]), tuple(int(x) for x in c[i])) for i in range(len(b0))])
    for s in range(1, steps + 1):
        raw = refine([np.frombuffer(e[0], np.uint64) for e in beam], s, per_step)
        seen = {e[0] for e in beam}
        cands = []
        for p in raw:
            b = canonical(p)
            if b not in seen:
                seen.add(b)
                cands.append(b)
        c, a, f = score(cands)
        beam = update(list(beam) + [(cands[i], float(a[i]), float(f[i]), tuple(int(x) for x in c[i]))
                                    for i in range(len(cands))])
    return [(e[0], e[3]) for e in beam]
