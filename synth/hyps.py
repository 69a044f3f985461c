"""Seeded random hypotheses (postfix programs) with the workloads' shapes.

Length is the number of postfix instructions, depth the tree height with
leaves at depth 1.  ``gen_tree`` builds a tree of an exact (length, depth),
which is feasible iff depth <= length <= 2**depth - 1 (a unary chain is the
longest-for-depth shape's opposite; a full binary tree the largest).
Internal constructors are drawn uniformly from the feasible members of the
allowed set; a role restriction reads its role inverted with probability 1/2
and draws n uniformly from 1..4; leaves are an atomic concept with probability
0.8, otherwise a data-range restriction (>= or <=, equally likely) whose
threshold is a present value of the property at a random individual.  On a KB
with numeric concrete roles the restricted property is drawn over the
one-value properties and the numeric roles together; a numeric role takes >=,
<= or == equally likely, with a threshold drawn from its asserted values.  On
a KB with string concrete roles, half of the data leaves (all, without other
data) restrict a string role: equality with a uniform table string or
containment of a uniform pattern, equally likely.

Shared sub-concepts: a pool of 256 seeded subtrees of depth 2..4; whenever
the generator is about to build a subtree of depth >= 2 whose exact
(length, depth) matches pool entries, it takes one of them with probability
``share`` instead.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import rng
from .kb import KB
from .programs import (AND, ATLEAST, ATMOST, ATOM, DEQ, DGE, DLE, EXISTS, FORALL, NOT, OR, SCONTAINS, SEQ,
                       Node, f32_bits, pack_batch)

S_HYP = 7 << 16
S_POOL = 8 << 16
S_THRESH = 9 << 16

UNARY_DEFAULT = (NOT, EXISTS, FORALL, ATLEAST, ATMOST)
BINARY_DEFAULT = (AND, OR)


def feasible(L: int, D: int) -> bool:
    return 1 <= D <= L <= (1 << D) - 1


class TreeGen:
    def __init__(self, kb: KB, seed: int, unary=UNARY_DEFAULT, binary=BINARY_DEFAULT,
                 p_atom: float = 0.8, share: float = 0.0, pool_size: int = 256):
        self.n_concepts = kb.n_concepts
        self.n_roles = kb.n_roles
        self.n_props = kb.n_props
        self.props = kb.prop_vals
        self.n_num = kb.n_num_roles
        self.num_vals = kb.num_vals
        self.n_str = kb.n_str_roles
        self.n_strings = len(kb.strings)
        self.n_patterns = kb.n_patterns
        self.seed = seed
        self.unary = tuple(unary)
        self.binary = tuple(binary)
        self.p_atom = p_atom if self.n_props + self.n_num + self.n_str > 0 else 1.0
        self.share = share
        self.pool: Dict[Tuple[int, int], List[Node]] = {}
        if share > 0:
            prng = rng.Rng(seed, S_POOL)
            for _ in range(pool_size):
                while True:
                    D = prng.randint(2, 4)
                    L = prng.randint(D, min((1 << D) - 1, 9))
                    if feasible(L, D):
                        break
                t = self._gen(prng, L, D, allow_share=False)
                self.pool.setdefault((L, D), []).append(t)

    # -- leaves
    def _threshold(self, r: rng.Rng, p: int) -> float:
        vals = self.props[p]
        for _ in range(64):
            v = vals[r.randint(0, vals.size - 1)]
            if not np.isnan(v):
                return float(v)
        return 0.0

    def leaf(self, r: rng.Rng) -> Node:
        if self.n_concepts == 0 or r.random() >= self.p_atom:
            if self.n_str and (self.n_props + self.n_num == 0 or r.random() < 0.5):
                q = r.randint(0, self.n_str - 1)
                if self.n_patterns and r.random() < 0.5:
                    return Node(SCONTAINS, q, r.randint(0, self.n_patterns - 1))
                return Node(SEQ, q, r.randint(0, max(self.n_strings - 1, 0)))
            if self.n_num:
                p = r.randint(0, self.n_props + self.n_num - 1)
                if p >= self.n_props:
                    vals = self.num_vals[p - self.n_props]
                    t = float(vals[r.randint(0, vals.size - 1)]) if vals.size else 0.0
                    return Node((DGE, DLE, DEQ)[r.randint(0, 2)], p, f32_bits(t))
                op = DGE if r.random() < 0.5 else DLE
                return Node(op, p, f32_bits(self._threshold(r, p)))
            p = r.randint(0, self.n_props - 1)
            op = DGE if r.random() < 0.5 else DLE
            return Node(op, p, f32_bits(self._threshold(r, p)))
        return Node(ATOM, r.randint(0, self.n_concepts - 1))

    def _role(self, r: rng.Rng, op: int, kid: Node) -> Node:
        role = r.randint(0, self.n_roles - 1)
        inv = r.random() < 0.5
        n = r.randint(1, 4) if op in (ATLEAST, ATMOST) else 0
        return Node(op, role, n, inv, [kid])

    # -- exact shape
    def _gen(self, r: rng.Rng, L: int, D: int, allow_share: bool = True) -> Node:
        if D == 1:
            assert L == 1
            return self.leaf(r)
        if allow_share and self.share > 0 and (L, D) in self.pool and r.random() < self.share:
            return r.choice(self.pool[(L, D)])
        ops = []
        if feasible(L - 1, D - 1):
            ops += [op for op in self.unary if op == NOT or self.n_roles > 0]
        half = (1 << (D - 1)) - 1
        splits = [L1 for L1 in range(D - 1, min(half, L - 2) + 1) if 1 <= L - 1 - L1 <= half]
        if splits:
            ops += list(self.binary)
        if not ops:
            raise ValueError(f"infeasible shape ({L},{D})")
        op = r.choice(ops)
        if op in self.binary:
            L1 = r.choice(splits)
            L2 = L - 1 - L1
            lo = max(1, L2.bit_length())    # smallest depth that holds L2 nodes
            D2 = r.randint(lo, min(L2, D - 1))
            a = self._gen(r, L1, D - 1, allow_share)
            b = self._gen(r, L2, D2, allow_share)
            if r.random() < 0.5:
                a, b = b, a
            return Node(op, kids=[a, b])
        kid = self._gen(r, L - 1, D - 1, allow_share)
        if op == NOT:
            return Node(NOT, kids=[kid])
        return self._role(r, op, kid)

    def tree(self, stream: int, L: int, D: int) -> Node:
        return self._gen(rng.Rng(self.seed, stream), L, D)


def random_shape(r: rng.Rng, lmax: int, dmin: int, dmax: int, lmin: int = 1) -> Tuple[int, int]:
    while True:
        D = r.randint(dmin, dmax)
        L = r.randint(lmin, lmax)
        if feasible(L, D):
            return L, D


def small_hyps(kb: KB, seed: int, count: int, dmax: int = 4, **kw) -> List[np.ndarray]:
    """Hypotheses of depth <= dmax, length uniform over what the depth allows."""
    g = TreeGen(kb, seed, **kw)
    out = []
    for h in range(count):
        r = rng.Rng(seed, S_HYP + h)
        D = r.randint(1, dmax)
        L = r.randint(D, (1 << D) - 1)
        out.append(np.array(g._gen(r, L, D).postfix(), dtype=np.uint64))
    return out


def batch_hyps(kb: KB, seed: int, batch: int, count: int = 4096, lmax: int = 40, dmax: int = 8,
               share: float = 0.3, gen: Optional[TreeGen] = None) -> List[np.ndarray]:
    """Length uniform 1..lmax, depth uniform 1..dmax (resampled until feasible), shared pool."""
    g = gen or TreeGen(kb, seed, share=share)
    out = []
    for h in range(count):
        r = rng.Rng(seed, S_HYP + (batch << 20) + h)
        L, D = random_shape(r, lmax, 1, dmax)
        out.append(np.array(g._gen(r, L, D).postfix(), dtype=np.uint64))
    return out


def chain_hyps(kb: KB, seed: int, count: int = 64, depth: int = 6, chain: int = 3) -> List[np.ndarray]:
    """Depth-``depth`` hypotheses holding a chain of ``chain`` nested EXISTS / ATLEAST.

    Shape: (and CHAIN Y) with CHAIN = R1(R2(R3(X))) of depth depth-1 (X of depth
    depth-1-chain) and Y a random subtree of depth <= depth-1.
    """
    g = TreeGen(kb, seed)
    out = []
    for h in range(count):
        r = rng.Rng(seed, S_HYP + h)
        dx = depth - 1 - chain
        x = g._gen(r, r.randint(dx, min((1 << dx) - 1, 3)), dx)
        for _ in range(chain):
            op = EXISTS if r.random() < 0.5 else ATLEAST
            x = g._role(r, op, x)
        dy = r.randint(1, depth - 1)
        y = g._gen(r, r.randint(dy, min((1 << dy) - 1, 12)), dy)
        kids = [x, y] if r.random() < 0.5 else [y, x]
        root = Node(AND if r.random() < 0.5 else OR, kids=kids)
        out.append(np.array(root.postfix(), dtype=np.uint64))
    return out


def batch_arrays(progs: Sequence[np.ndarray]) -> Tuple[np.ndarray, np.ndarray]:
    return pack_batch(progs)
