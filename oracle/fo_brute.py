"""First-order brute force for tiny KBs (TEST INFRASTRUCTURE).

Each constructor is written as the set comprehension of its first-order
translation, quantifying over the whole domain (quadratic in the number of
individuals, so only for n up to a few dozen).  It is a second evaluator,
structured differently from the C oracle (which scans assertion pairs), used
to pin it:

    (exists r C)   = { x | some y: r(x, y) and C(y) }
    (all r C)      = { x | every y: r(x, y) implies C(y) }
    (min n r C)    = { x | #{ y | r(x, y) and C(y) } >= n }
    (max n r C)    = { x | #{ y | r(x, y) and C(y) } <= n }
    (exactly n r C)= { x | #{ y | r(x, y) and C(y) } == n }
    r^-(x, y)      = r(y, x)
    (ge p t)       = { x | some v: p(x, v) and v >= t }   (float32 compare)
    (seq s v)      = { x | some u: s(x, u) and u = strings[v] }
    (contains s k) = { x | some u: s(x, u) and patterns[k] occurs in u }

under the closed-world reading (Section III-A of the paper): a fact not in
the KB is false, so NOT is the complement within the domain.  A property maps
an individual to one value or to several (a numeric concrete role, Section
III-B); either way the restriction asks for some value.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Set, Tuple

import numpy as np

_ATOM, _TOP, _BOT, _NOT, _AND, _OR = 1, 2, 3, 4, 5, 6
_EX, _ALL, _MIN, _MAX, _EXACT = 7, 8, 9, 10, 11
_GE, _LE, _EQ = 12, 13, 14
_SEQ, _SCONTAINS = 15, 16


class TinyKB:
    def __init__(self, n: int, concepts: Sequence[Set[int]], roles: Sequence[Set[Tuple[int, int]]],
                 props: Sequence[Dict[int, object]], str_roles: Sequence[Dict[int, Sequence[bytes]]] = (),
                 strings: Sequence[bytes] = (), patterns: Sequence[bytes] = ()):
        """props[p][x]: a float or a sequence of floats (x's values of p);
        str_roles[s][x]: x's string values of string role s; strings: the table SEQ
        names by index; patterns: the substrings SCONTAINS names by index."""
        self.n = n
        self.domain = range(n)
        self.concepts = [set(c) for c in concepts]
        self.roles = [set(r) for r in roles]
        self.props = [{int(k): tuple(np.float32(u) for u in (v if isinstance(v, (list, tuple)) else [v]))
                       for k, v in p.items()} for p in props]
        self.str_roles = [{int(k): [bytes(u) for u in v] for k, v in r.items()} for r in str_roles]
        self.strings = [bytes(x) for x in strings]
        self.patterns = [bytes(x) for x in patterns]

    def rel(self, r: int, inverse: bool, x: int, y: int) -> bool:
        return ((y, x) if inverse else (x, y)) in self.roles[r]


def evaluate(kb: TinyKB, prog: Sequence[int]) -> Set[int]:
    stack: List[Set[int]] = []
    D = kb.domain
    for w in prog:
        w = int(w)
        op, fl, a, b = w & 0xFF, (w >> 8) & 0xFF, (w >> 16) & 0xFFFF, (w >> 32) & 0xFFFFFFFF
        inv = bool(fl & 1)
        if op == _ATOM:
            stack.append(set(kb.concepts[a]))
        elif op == _TOP:
            stack.append(set(D))
        elif op == _BOT:
            stack.append(set())
        elif op == _NOT:
            X = stack.pop()
            stack.append({x for x in D if x not in X})
        elif op in (_AND, _OR):
            Y = stack.pop()
            X = stack.pop()
            stack.append(X & Y if op == _AND else X | Y)
        elif op == _EX:
            X = stack.pop()
            stack.append({x for x in D if any(kb.rel(a, inv, x, y) and y in X for y in D)})
        elif op == _ALL:
            X = stack.pop()
            stack.append({x for x in D if all((not kb.rel(a, inv, x, y)) or y in X for y in D)})
        elif op in (_MIN, _MAX, _EXACT):
            X = stack.pop()
            out = set()
            for x in D:
                k = len([y for y in D if kb.rel(a, inv, x, y) and y in X])
                if (op == _MIN and k >= b) or (op == _MAX and k <= b) or (op == _EXACT and k == b):
                    out.add(x)
            stack.append(out)
        elif op in (_GE, _LE, _EQ):
            t = np.array([b], dtype=np.uint32).view(np.float32)[0]
            vals = kb.props[a]
            out = set()
            for x in D:
                if any((op == _GE and v >= t) or (op == _LE and v <= t) or (op == _EQ and v == t)
                       for v in vals.get(x, ())):
                    out.add(x)
            stack.append(out)
        elif op == _SEQ:         # { x | some v: s(x, v) and v = strings[b] }
            vals = kb.str_roles[a]
            want = kb.strings[b] if b < len(kb.strings) else None
            stack.append({x for x in D if want is not None and any(v == want for v in vals.get(x, ()))})
        elif op == _SCONTAINS:   # { x | some v: s(x, v) and patterns[b] is a substring of v }
            vals = kb.str_roles[a]
            stack.append({x for x in D if any(kb.patterns[b] in v for v in vals.get(x, ()))})
        else:
            raise ValueError(f"bad op {op}")
    if len(stack) != 1:
        raise ValueError("program does not reduce to one concept")
    return stack[0]


def coverage(R: Set[int], pos: Set[int], neg: Set[int]) -> Tuple[int, int, int, int]:
    tp = len(R & pos)
    fp = len(R & neg)
    return tp, fp, len(pos) - tp, len(neg) - fp
