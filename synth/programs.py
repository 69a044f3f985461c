"""Hypothesis programs: the 8-byte postfix instruction format and a text syntax.

A hypothesis (an ALCQI(D) concept, Section IV of the paper: a hypothesis is an
array of DL operations in consecutive memory) is stored as postfix
instructions, one uint64 each:

    bits  0..7   op
    bits  8..15  flags   (bit 0: the role is read inverted, r^-)
    bits 16..31  a       (concept id, role id, data-property id or string-role id)
    bits 32..63  b       (n of a cardinality restriction, the float32 bits of a
                          data-range threshold, a string id or a pattern id)

Ops (binary AND/OR; NOT and the role restrictions are unary; the rest are
leaves):

    1 ATOM c   2 TOP   3 BOT   4 NOT   5 AND   6 OR
    7 EXISTS r   8 FORALL r   9 ATLEAST r n   10 ATMOST r n   11 EXACTLY r n
    12 DGE p t   13 DLE p t   14 DEQ p t
    15 SEQ s v (a value of string role s is string v)
    16 SCONTAINS s k (a value of string role s contains pattern k)

The text syntax (for tests and fixtures) is prefix s-expressions:

    A3, TOP, BOT, (not X), (and X Y), (or X Y), (some r2 X), (some r2- X),
    (all r2 X), (min 2 r2 X), (max 2 r2 X), (exactly 2 r2 X),
    (ge p1 0.5), (le p1 0.5), (eq p1 0.5), (seq s0 17), (contains s0 3)

with r2- the inverse of role 2; ``(r-)-`` folds back to ``r`` (the suffix may
repeat: r2-- is r2).

This module only writes and reads the format; it evaluates nothing.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

ATOM, TOP, BOT, NOT, AND, OR = 1, 2, 3, 4, 5, 6
EXISTS, FORALL, ATLEAST, ATMOST, EXACTLY = 7, 8, 9, 10, 11
DGE, DLE, DEQ = 12, 13, 14
SEQ, SCONTAINS = 15, 16

OP_NAMES = {
    ATOM: "ATOM", TOP: "TOP", BOT: "BOT", NOT: "NOT", AND: "AND", OR: "OR",
    EXISTS: "EXISTS", FORALL: "FORALL", ATLEAST: "ATLEAST", ATMOST: "ATMOST",
    EXACTLY: "EXACTLY", DGE: "DGE", DLE: "DLE", DEQ: "DEQ", SEQ: "SEQ", SCONTAINS: "SCONTAINS",
}
ROLE_OPS = (EXISTS, FORALL, ATLEAST, ATMOST, EXACTLY)
COUNT_OPS = (ATLEAST, ATMOST, EXACTLY)
DATA_OPS = (DGE, DLE, DEQ)
STRING_OPS = (SEQ, SCONTAINS)
LEAF_OPS = (ATOM, TOP, BOT) + DATA_OPS + STRING_OPS
FLAG_INVERSE = 1


def f32_bits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", float(x)))[0]


def bits_f32(b: int) -> float:
    return struct.unpack("<f", struct.pack("<I", b & 0xFFFFFFFF))[0]


def insn(op: int, flags: int = 0, a: int = 0, b: int = 0) -> int:
    return (op & 0xFF) | ((flags & 0xFF) << 8) | ((a & 0xFFFF) << 16) | ((b & 0xFFFFFFFF) << 32)


def fields(w: int) -> Tuple[int, int, int, int]:
    w = int(w)
    return w & 0xFF, (w >> 8) & 0xFF, (w >> 16) & 0xFFFF, (w >> 32) & 0xFFFFFFFF


# --------------------------------------------------------------------------- trees
@dataclass
class Node:
    """Expression tree node used by the generators and the text syntax."""
    op: int
    a: int = 0            # concept / role / property / string-role id
    b: int = 0            # n, float32 bits of the threshold, string id or pattern id
    inv: bool = False     # role read inverted
    kids: List["Node"] = field(default_factory=list)

    def postfix(self, out: Optional[list] = None) -> list:
        if out is None:
            out = []
        for k in self.kids:
            k.postfix(out)
        out.append(insn(self.op, FLAG_INVERSE if self.inv else 0, self.a, self.b))
        return out

    def height(self) -> int:
        return 1 + max((k.height() for k in self.kids), default=0)

    def size(self) -> int:
        return 1 + sum(k.size() for k in self.kids)


def from_postfix(prog: Sequence[int]) -> Node:
    st: List[Node] = []
    for w in prog:
        op, fl, a, b = fields(w)
        if op in LEAF_OPS:
            st.append(Node(op, a, b))
        elif op in (NOT,) or op in ROLE_OPS:
            x = st.pop()
            st.append(Node(op, a, b, bool(fl & FLAG_INVERSE), [x]))
        elif op in (AND, OR):
            y = st.pop()
            x = st.pop()
            st.append(Node(op, a, b, False, [x, y]))
        else:
            raise ValueError(f"bad op {op}")
    if len(st) != 1:
        raise ValueError("program does not reduce to one concept")
    return st[0]


# --------------------------------------------------------------------------- text
_ROLE_WORD = {EXISTS: "some", FORALL: "all", ATLEAST: "min", ATMOST: "max", EXACTLY: "exactly"}
_DATA_WORD = {DGE: "ge", DLE: "le", DEQ: "eq"}
_WORD_ROLE = {v: k for k, v in _ROLE_WORD.items()}
_WORD_DATA = {v: k for k, v in _DATA_WORD.items()}
_STRING_WORD = {SEQ: "seq", SCONTAINS: "contains"}
_WORD_STRING = {v: k for k, v in _STRING_WORD.items()}


def to_text(n: Node) -> str:
    if n.op == ATOM:
        return f"A{n.a}"
    if n.op == TOP:
        return "TOP"
    if n.op == BOT:
        return "BOT"
    if n.op == NOT:
        return f"(not {to_text(n.kids[0])})"
    if n.op in (AND, OR):
        return f"({'and' if n.op == AND else 'or'} {to_text(n.kids[0])} {to_text(n.kids[1])})"
    if n.op in ROLE_OPS:
        r = f"r{n.a}{'-' if n.inv else ''}"
        if n.op in COUNT_OPS:
            return f"({_ROLE_WORD[n.op]} {n.b} {r} {to_text(n.kids[0])})"
        return f"({_ROLE_WORD[n.op]} {r} {to_text(n.kids[0])})"
    if n.op in DATA_OPS:
        return f"({_DATA_WORD[n.op]} p{n.a} {str(np.float32(bits_f32(n.b)))})"  # shortest float32 text
    if n.op in STRING_OPS:
        return f"({_STRING_WORD[n.op]} s{n.a} {n.b})"
    raise ValueError(n.op)


def _tokens(s: str) -> List[str]:
    return s.replace("(", " ( ").replace(")", " ) ").split()


def parse(text: str) -> Node:
    toks = _tokens(text)
    pos = 0

    def role(tok: str) -> Tuple[int, bool]:
        if not tok.startswith("r"):
            raise ValueError(f"expected role, got {tok}")
        body = tok[1:]
        inv = False
        while body.endswith("-"):       # (r^-)^- = r
            inv = not inv
            body = body[:-1]
        return int(body), inv

    def expr() -> Node:
        nonlocal pos
        t = toks[pos]
        pos += 1
        if t != "(":
            if t == "TOP":
                return Node(TOP)
            if t == "BOT":
                return Node(BOT)
            if t.startswith("A"):
                return Node(ATOM, int(t[1:]))
            raise ValueError(f"bad token {t}")
        head = toks[pos]
        pos += 1
        if head == "not":
            n = Node(NOT, kids=[expr()])
        elif head in ("and", "or"):
            x = expr()
            y = expr()
            n = Node(AND if head == "and" else OR, kids=[x, y])
        elif head in ("some", "all"):
            r, inv = role(toks[pos])
            pos += 1
            n = Node(_WORD_ROLE[head], r, 0, inv, [expr()])
        elif head in ("min", "max", "exactly"):
            k = int(toks[pos])
            r, inv = role(toks[pos + 1])
            pos += 2
            n = Node(_WORD_ROLE[head], r, k, inv, [expr()])
        elif head in _WORD_DATA:
            p = int(toks[pos][1:])
            t = float(toks[pos + 1])
            pos += 2
            n = Node(_WORD_DATA[head], p, f32_bits(t))
        elif head in _WORD_STRING:
            if not toks[pos].startswith("s"):
                raise ValueError(f"expected string role, got {toks[pos]}")
            n = Node(_WORD_STRING[head], int(toks[pos][1:]), int(toks[pos + 1]))
            pos += 2
        else:
            raise ValueError(f"bad head {head}")
        if toks[pos] != ")":
            raise ValueError("expected )")
        pos += 1
        return n

    n = expr()
    if pos != len(toks):
        raise ValueError("trailing tokens")
    return n


def compile_text(text: str) -> np.ndarray:
    return np.array(parse(text).postfix(), dtype=np.uint64)


def pack_batch(progs: Sequence[Sequence[int]]) -> Tuple[np.ndarray, np.ndarray]:
    """Concatenate programs into (insns uint64[total], offs uint32[H+1])."""
    offs = np.zeros(len(progs) + 1, dtype=np.uint32)
    for i, p in enumerate(progs):
        offs[i + 1] = offs[i] + len(p)
    flat = np.zeros(int(offs[-1]), dtype=np.uint64)
    for i, p in enumerate(progs):
        flat[offs[i]:offs[i + 1]] = np.asarray(p, dtype=np.uint64)
    return flat, offs
