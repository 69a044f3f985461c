"""Seeded refinement operators for the beam search (candidate generation).

Every candidate of step s is a pure function of (seed, s, beam member m,
candidate number k): candidate k refines beam member k mod |beam| with an
operator drawn uniformly from
  0  add a conjunct      C  ->  (and C X)
  1  add a disjunct      C  ->  (or C X)
  2  wrap                C  ->  (some r C) | (all r C) | (min n r C)   (r^- with prob. 1/2, n in 1..4)
  3  tighten threshold   a data restriction inside C moves one step on its
                         property's 64-quantile grid: up for >=, down for <=
                         (if C has none, or it is at the grid's end: add a
                         conjunct instead)
X is a simple concept: an atom (prob. 1/2), a data restriction p >= t or
p <= t with t on the grid (prob. 3/10), or (some r A) (prob. 1/5).
Both the exhaustive and the surrogate-ordered search call the same
generator, so they see the identical candidate list.  ``refine_postfix`` is
the same generator on postfix arrays, run by the C helper in fastgen.c draw
for draw (a test checks the two agree).  This module draws candidates only;
it evaluates nothing.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from . import rng
from .programs import (AND, ATLEAST, ATOM, DGE, DLE, EXISTS, FORALL, OR, Node, bits_f32, f32_bits)

S_REFINE = 11 << 16
GRID = 64


class Refiner:
    def __init__(self, kb, seed: int):
        self.seed = seed
        self.n_concepts = kb.n_concepts
        self.n_roles = kb.n_roles
        self.n_props = kb.n_props
        self.grid = []
        for p in range(kb.n_props):
            v = kb.prop_vals[p]
            v = v[~np.isnan(v)]
            q = np.quantile(v, np.linspace(0.0, 1.0, GRID)).astype(np.float32) if v.size else np.zeros(1, np.float32)
            self.grid.append(np.unique(q))
        self._gflat = np.concatenate(self.grid).astype(np.float32) if self.grid else np.zeros(1, np.float32)
        self._goffs = np.zeros(len(self.grid) + 1, np.int64)
        np.cumsum([len(g) for g in self.grid], out=self._goffs[1:])

    def _rng(self, step: int, member: int, k: int) -> rng.Rng:
        return rng.Rng(self.seed, S_REFINE + (step << 40) + (member << 24) + k)

    def _simple(self, r: rng.Rng) -> Node:
        u = r.random()
        if u < 0.5 or (self.n_props == 0 and self.n_roles == 0):
            return Node(ATOM, r.randint(0, self.n_concepts - 1))
        if (u < 0.8 and self.n_props) or not self.n_roles:
            p = r.randint(0, self.n_props - 1)
            t = self.grid[p][r.randint(0, len(self.grid[p]) - 1)]
            return Node(DGE if r.random() < 0.5 else DLE, p, f32_bits(float(t)))
        return Node(EXISTS, r.randint(0, self.n_roles - 1), 0, r.random() < 0.5,
                    [Node(ATOM, r.randint(0, self.n_concepts - 1))])

    def _data_nodes(self, n: Node, path=(), out=None):
        if out is None:
            out = []
        if n.op in (DGE, DLE):
            out.append(path)
        for i, c in enumerate(n.kids):
            self._data_nodes(c, path + (i,), out)
        return out

    @staticmethod
    def _replace(n: Node, path, new: Node) -> Node:
        if not path:
            return new
        kids = list(n.kids)
        kids[path[0]] = Refiner._replace(kids[path[0]], path[1:], new)
        return Node(n.op, n.a, n.b, n.inv, kids)

    @staticmethod
    def _get(n: Node, path) -> Node:
        for i in path:
            n = n.kids[i]
        return n

    def refine_one(self, base: Node, step: int, member: int, k: int) -> Node:
        r = self._rng(step, member, k)
        op = r.randint(0, 3)
        if op == 3:
            paths = self._data_nodes(base)
            if paths:
                path = paths[r.randint(0, len(paths) - 1)]
                d = self._get(base, path)
                g = self.grid[d.a]
                t = np.float32(bits_f32(d.b))
                i = int(np.searchsorted(g, t))
                j = (i + 1 if i < len(g) and g[i] == t else i) if d.op == DGE else i - 1
                if 0 <= j < len(g):
                    return self._replace(base, path, Node(d.op, d.a, f32_bits(float(g[j]))))
            op = 0
        if op == 0:
            return Node(AND, kids=[base, self._simple(r)])
        if op == 1:
            return Node(OR, kids=[base, self._simple(r)])
        w = r.randint(0, 2)
        role = r.randint(0, self.n_roles - 1) if self.n_roles else 0
        inv = r.random() < 0.5
        if w == 0 or not self.n_roles:
            return Node(EXISTS, role, 0, inv, [base]) if self.n_roles else Node(AND, kids=[base, self._simple(r)])
        if w == 1:
            return Node(FORALL, role, 0, inv, [base])
        return Node(ATLEAST, role, r.randint(1, 4), inv, [base])

    def refine(self, beam: Sequence[Node], step: int, count: int) -> List[Node]:
        return [self.refine_one(beam[k % len(beam)], step, k % len(beam), k) for k in range(count)]

    def refine_postfix(self, beam: Sequence[np.ndarray], step: int, count: int):
        """``refine`` on postfix programs, in C: (flat uint64 instructions, offsets int64[count+1])."""
        from .kb import _fast
        bflat = np.ascontiguousarray(np.concatenate([np.asarray(b, np.uint64) for b in beam]), np.uint64)
        boffs = np.zeros(len(beam) + 1, np.int64)
        np.cumsum([len(b) for b in beam], out=boffs[1:])
        lens = boffs[1:] - boffs[:-1]
        M = len(beam)      # candidate k copies member k mod M and adds at most 3 instructions
        cap = int((count // M) * lens.sum() + lens[: count % M].sum() + 3 * count)
        out = np.zeros(max(cap, 1), np.uint64)
        offs = np.zeros(count + 1, np.int64)
        rc = _fast().fastgen_refine(self.seed, step, bflat.ctypes.data, boffs.ctypes.data, len(beam), count,
                                    self.n_concepts, self.n_roles, self.n_props, self._gflat.ctypes.data,
                                    self._goffs.ctypes.data, out.ctypes.data, out.size, offs.ctypes.data)
        if rc:
            raise RuntimeError("refinement output buffer too small")
        return out[: offs[-1]], offs

    def start(self) -> List[Node]:
        """Initial beam: the top concept."""
        from .programs import TOP
        return [Node(TOP)]
