"""The oracle: a plain CPU evaluator of ALCQI(D) hypotheses by set semantics.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import this package.  It shares
no code with the GPU library (``paper_2412_00802_gb300``) and never imports
it.

``hedl_oracle.c`` is the evaluator (byte-per-membership sets, role
assertions as (subject, object) pairs, numeric concrete-role assertions as
(subject, value) pairs and string concrete-role assertions as (subject, bytes)
pairs, the paper's Section III layout);
``fo_brute`` is a second, first-order-semantics evaluator in pure Python for
tiny inputs, used to pin the C one.  This wrapper only marshals arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hedl_oracle.c")
_LIB = os.path.join(_HERE, "libhedl_oracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", -1: "bad op", -2: "bad id", -3: "stack underflow", -4: "stack overflow",
          -5: "program does not reduce to one concept", -6: "empty program", -7: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _KB(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64),
                ("n_concepts", ctypes.c_int32),
                ("concept_member", ctypes.c_void_p),
                ("n_roles", ctypes.c_int32),
                ("role_off", ctypes.c_void_p),
                ("subj", ctypes.c_void_p),
                ("obj", ctypes.c_void_p),
                ("n_props", ctypes.c_int32),
                ("prop", ctypes.c_void_p),
                ("n_num_roles", ctypes.c_int32),
                ("num_off", ctypes.c_void_p),
                ("num_subj", ctypes.c_void_p),
                ("num_val", ctypes.c_void_p),
                ("n_str_roles", ctypes.c_int32),
                ("str_off", ctypes.c_void_p),
                ("str_subj", ctypes.c_void_p),
                ("str_val_off", ctypes.c_void_p),
                ("str_val", ctypes.c_void_p),
                ("n_strings", ctypes.c_int64),
                ("tbl_off", ctypes.c_void_p),
                ("tbl", ctypes.c_void_p),
                ("n_patterns", ctypes.c_int64),
                ("pat_off", ctypes.c_void_p),
                ("pat", ctypes.c_void_p)]


def _byte_table(items) -> Tuple[np.ndarray, np.ndarray]:
    """A list of byte strings as (int64 offsets [len+1], uint8 bytes)."""
    items = [bytes(x) for x in items]
    off = np.zeros(len(items) + 1, np.int64)
    if items:
        np.cumsum([len(x) for x in items], out=off[1:])
    return off, np.frombuffer(b"".join(items), np.uint8).copy()


def load(path: str):
    """Load an oracle shared library from ``path`` and declare its signatures."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    L.oracle_validate.argtypes = [P, P, ctypes.c_int64]
    L.oracle_validate.restype = ctypes.c_int
    L.oracle_eval.argtypes = [P, P, ctypes.c_int64, P]
    L.oracle_eval.restype = ctypes.c_int
    L.oracle_score.argtypes = [ctypes.c_int64, P, P, P, P]
    L.oracle_score.restype = None
    L.oracle_eval_batch.argtypes = [P, P, P, ctypes.c_int64, P, P, ctypes.c_int32, P, P, P, P]
    L.oracle_eval_batch.restype = ctypes.c_int64
    L.oracle_eval_bytes.argtypes = [P, P, ctypes.c_int64, P, P]
    L.oracle_eval_bytes.restype = ctypes.c_int
    L.oracle_score_bytes.argtypes = [ctypes.c_int64]
    L.oracle_score_bytes.restype = ctypes.c_int64
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib



def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class OracleKB:
    """A KB in the oracle's own layout (bytes per membership, assertion pairs)."""
    n: int
    member: np.ndarray        # uint8 [C][n]
    role_off: np.ndarray      # int64 [R+1]
    subj: np.ndarray          # uint32 [E]
    obj: np.ndarray           # uint32 [E]
    prop: np.ndarray          # float32 [P][n]
    pos: np.ndarray           # uint8 [n]
    neg: np.ndarray           # uint8 [n]
    # numeric concrete roles (property ids n_props + q): (subject, value) assertions per role
    num_off: np.ndarray = None    # int64 [Q+1]
    num_subj: np.ndarray = None   # uint32 [M]
    num_val: np.ndarray = None    # float32 [M]
    # string concrete roles: (subject, value bytes) assertions per role, the string table and the patterns
    str_off: np.ndarray = None      # int64 [S_roles+1]
    str_subj: np.ndarray = None     # uint32 [A]
    str_val_off: np.ndarray = None  # int64 [A+1]
    str_val: np.ndarray = None      # uint8
    tbl_off: np.ndarray = None      # int64 [n_strings+1]
    tbl: np.ndarray = None          # uint8
    pat_off: np.ndarray = None      # int64 [n_patterns+1]
    pat: np.ndarray = None          # uint8

    def __post_init__(self):
        if self.num_off is None:
            self.num_off = np.zeros(1, np.int64)
            self.num_subj = np.zeros(0, np.uint32)
            self.num_val = np.zeros(0, np.float32)
        if self.str_off is None:
            self.str_off = np.zeros(1, np.int64)
            self.str_subj = np.zeros(0, np.uint32)
            self.str_val_off, self.str_val = _byte_table([])
            self.tbl_off, self.tbl = _byte_table([])
            self.pat_off, self.pat = _byte_table([])
        names = ("member", "role_off", "subj", "obj", "prop", "pos", "neg", "num_off", "num_subj", "num_val",
                 "str_off", "str_subj", "str_val_off", "str_val", "tbl_off", "tbl", "pat_off", "pat")
        for name in names:
            setattr(self, name, np.ascontiguousarray(getattr(self, name)))
        opt = lambda a: _ptr(a) if a.size else None
        self._c = _KB(self.n, self.member.shape[0], _ptr(self.member) if self.member.size else None,
                      self.role_off.size - 1, _ptr(self.role_off), _ptr(self.subj) if self.subj.size else None,
                      _ptr(self.obj) if self.obj.size else None, self.prop.shape[0],
                      _ptr(self.prop) if self.prop.size else None,
                      self.num_off.size - 1, _ptr(self.num_off),
                      _ptr(self.num_subj) if self.num_subj.size else None,
                      _ptr(self.num_val) if self.num_val.size else None,
                      self.str_off.size - 1, _ptr(self.str_off), opt(self.str_subj), _ptr(self.str_val_off),
                      opt(self.str_val), self.tbl_off.size - 1, _ptr(self.tbl_off), opt(self.tbl),
                      self.pat_off.size - 1, _ptr(self.pat_off), opt(self.pat))

    @property
    def cptr(self):
        return ctypes.addressof(self._c)

    @classmethod
    def from_parts(cls, n: int, member: np.ndarray, edges: Sequence[Tuple[np.ndarray, np.ndarray]],
                   prop: np.ndarray, pos: np.ndarray, neg: np.ndarray,
                   num_roles: Sequence[Tuple[np.ndarray, np.ndarray]] = (),
                   str_roles: Sequence[Tuple[np.ndarray, Sequence[bytes]]] = (),
                   strings: Sequence[bytes] = (), patterns: Sequence[bytes] = (),
                   str_arrays: Optional[Tuple[np.ndarray, ...]] = None) -> "OracleKB":
        """edges: per role (subjects, objects); each pair must appear at most once.
        num_roles: per numeric concrete role (subjects, float values), any order.
        str_roles: per string concrete role (subjects, value byte strings), any order;
        strings: the table SEQ indexes; patterns: the substrings SCONTAINS indexes.
        str_arrays: the string assertions already laid out (role offsets, subjects,
        value offsets, value bytes), instead of str_roles."""
        offs = [0]
        subj, obj = [], []
        for s, o in edges:
            s = np.asarray(s, dtype=np.uint32)
            o = np.asarray(o, dtype=np.uint32)
            if s.size:
                if int(s.max()) >= n or int(o.max()) >= n:
                    raise ValueError("assertion names an individual >= n")
                key = s.astype(np.uint64) * np.uint64(max(n, 1)) + o.astype(np.uint64)
                # strictly increasing keys are duplicate-free; otherwise sort to check
                if not (key.size < 2 or bool(np.all(key[1:] > key[:-1]))):
                    if np.unique(key).size != key.size:
                        raise ValueError("role assertions must be a set (duplicate pair)")
            subj.append(s)
            obj.append(o)
            offs.append(offs[-1] + s.size)
        cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)
        noff, nsubj, nval = [0], [], []
        for s_, v_ in num_roles:
            s_ = np.asarray(s_, dtype=np.uint32)
            v_ = np.asarray(v_, dtype=np.float32)
            if s_.size != v_.size:
                raise ValueError("a numeric assertion needs one subject and one value")
            if s_.size and int(s_.max()) >= n:
                raise ValueError("numeric assertion names an individual >= n")
            nsubj.append(s_)
            nval.append(v_)
            noff.append(noff[-1] + s_.size)
        soff, ssubj, svals = [0], [], []
        for s_, v_ in str_roles:
            s_ = np.asarray(s_, dtype=np.uint32)
            if s_.size != len(v_):
                raise ValueError("a string assertion needs one subject and one value")
            if s_.size and int(s_.max()) >= n:
                raise ValueError("string assertion names an individual >= n")
            ssubj.append(s_)
            svals += list(v_)
            soff.append(soff[-1] + s_.size)
        sv_off, sv = _byte_table(svals)
        if str_arrays is not None:
            soff, ssubj, sv_off, sv = str_arrays
            soff, ssubj = list(soff), [np.asarray(ssubj, np.uint32)]
        t_off, t = _byte_table(strings)
        p_off, pt = _byte_table(patterns)
        return cls(n, np.asarray(member, np.uint8).reshape(-1, n) if n else np.zeros((len(member), 0), np.uint8),
                   np.array(offs, dtype=np.int64), cat(subj, np.uint32), cat(obj, np.uint32),
                   np.asarray(prop, np.float32).reshape(-1, n) if n else np.zeros((len(prop), 0), np.float32),
                   np.asarray(pos, np.uint8), np.asarray(neg, np.uint8),
                   np.array(noff, dtype=np.int64), cat(nsubj, np.uint32), cat(nval, np.float32),
                   np.array(soff, dtype=np.int64), cat(ssubj, np.uint32), sv_off, sv, t_off, t, p_off, pt)


def from_synth(kb) -> OracleKB:
    """Convert a synthetic KB (bitsets + CSR) into the oracle's layout.

    Only forward assertions are passed: the oracle reads an inverse role by
    swapping subject and object, never through the inverse CSR.
    """
    n = kb.n
    nbytes = (n + 7) // 8
    member = np.zeros((kb.n_concepts, n), dtype=np.uint8)
    for c in range(kb.n_concepts):
        member[c] = np.unpackbits(kb.concept_bits[c].view(np.uint8)[:nbytes], bitorder="little")[:n]
    edges = []
    for r in range(kb.n_roles):
        deg = np.diff(kb.row_ptr[r].astype(np.int64))
        edges.append((np.repeat(np.arange(n, dtype=np.uint32), deg), kb.col[r]))
    pos = np.zeros(n, dtype=np.uint8)
    pos[kb.pos_idx] = 1
    neg = np.zeros(n, dtype=np.uint8)
    neg[kb.neg_idx] = 1
    nums = []
    for q in range(kb.n_num_roles):
        deg = np.diff(kb.num_row_ptr[q].astype(np.int64))
        nums.append((np.repeat(np.arange(n, dtype=np.uint32), deg), kb.num_vals[q]))
    # string roles: each assertion gets its own copy of its value's bytes (the
    # oracle compares bytes; the interned ids are not passed)
    arrays = None
    if kb.n_str_roles:
        t_off, t = _byte_table(kb.strings)
        t_len = np.diff(t_off)
        soff, subj, ids = [0], [], []
        for q in range(kb.n_str_roles):
            deg = np.diff(kb.str_row_ptr[q].astype(np.int64))
            subj.append(np.repeat(np.arange(n, dtype=np.uint32), deg))
            ids.append(kb.str_ids[q].astype(np.int64))
            soff.append(soff[-1] + int(deg.sum()))
        ids = np.concatenate(ids)
        lens = t_len[ids]
        v_off = np.zeros(ids.size + 1, np.int64)
        np.cumsum(lens, out=v_off[1:])
        vals = np.empty(int(v_off[-1]), np.uint8)
        for c in range(0, ids.size, 1 << 22):    # gather each assertion's bytes, a chunk at a time
            sl = slice(c, min(c + (1 << 22), ids.size))
            b0, b1 = int(v_off[sl.start]), int(v_off[sl.stop])
            src = np.repeat(t_off[ids[sl]] - v_off[sl], lens[sl]) + np.arange(b0, b1, dtype=np.int64)
            vals[b0:b1] = t[src]
        arrays = (np.array(soff, np.int64), np.concatenate(subj), v_off, vals)
    return OracleKB.from_parts(n, member, edges, kb.prop_vals, pos, neg, nums, (), kb.strings, kb.patterns,
                               arrays)


def validate(okb: OracleKB, prog, L=None) -> int:
    p = np.ascontiguousarray(prog, dtype=np.uint64)
    return (L or lib()).oracle_validate(okb.cptr, _ptr(p) if p.size else None, p.size)


def eval_program(okb: OracleKB, prog, L=None) -> np.ndarray:
    """Instance set of one program as bool[n]; raises ValueError on a bad program."""
    p = np.ascontiguousarray(prog, dtype=np.uint64)
    out = np.zeros(max(okb.n, 1), dtype=np.uint8)
    e = (L or lib()).oracle_eval(okb.cptr, _ptr(p) if p.size else None, p.size, _ptr(out))
    if e:
        raise ValueError(ERRORS.get(e, str(e)))
    return out[: okb.n].astype(bool)


def score(okb: OracleKB, r: np.ndarray, L=None) -> np.ndarray:
    """(TP, FP, FN, TN) of an instance set (Algorithm 15 plus the complements)."""
    rr = np.ascontiguousarray(r, dtype=np.uint8)
    c = np.zeros(4, dtype=np.int64)
    (L or lib()).oracle_score(okb.n, _ptr(rr), _ptr(okb.pos), _ptr(okb.neg), _ptr(c))
    return c


def eval_batch(okb: OracleKB, progs: np.ndarray, offs: np.ndarray, threads: int = 1,
               keep_sets: bool = False, L=None, bytes_out: Optional[np.ndarray] = None
               ) -> Tuple[np.ndarray, Optional[np.ndarray], np.ndarray]:
    """Evaluate and score a batch: returns counts int64[H][4], sets uint8[H][n] or None, errs.
    bytes_out (int64[H], optional) receives each program's algorithmic bytes, score included."""
    progs = np.ascontiguousarray(progs, dtype=np.uint64)
    offs64 = np.ascontiguousarray(offs, dtype=np.int64)
    H = offs64.size - 1
    counts = np.zeros((H, 4), dtype=np.int64)
    errs = np.zeros(H, dtype=np.int32)
    sets = np.zeros((H, okb.n), dtype=np.uint8) if keep_sets else None
    if bytes_out is not None:
        assert bytes_out.dtype == np.int64 and bytes_out.shape == (H,) and bytes_out.flags.c_contiguous
    (L or lib()).oracle_eval_batch(okb.cptr, _ptr(progs) if progs.size else None, _ptr(offs64), H,
                            _ptr(okb.pos), _ptr(okb.neg), threads, _ptr(counts),
                            _ptr(sets) if sets is not None else None, _ptr(errs),
                            _ptr(bytes_out) if bytes_out is not None else None)
    return counts, sets, errs


def model_bytes(okb: OracleKB, prog, L=None) -> int:
    """Algorithmic bytes of one program (its operations as the evaluator runs them, plus its
    score): the plain method's per-operation byte model, counted while evaluating."""
    p = np.ascontiguousarray(prog, dtype=np.uint64)
    out = np.zeros(max(okb.n, 1), dtype=np.uint8)
    b = ctypes.c_int64(0)
    lb = L or lib()
    e = lb.oracle_eval_bytes(okb.cptr, _ptr(p) if p.size else None, p.size, _ptr(out), ctypes.byref(b))
    if e:
        raise ValueError(ERRORS.get(e, str(e)))
    return int(b.value) + int(lb.oracle_score_bytes(okb.n))


def accuracy_f1(counts: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """acc = (TP+TN)/(|P|+|N|), F1 = 2TP/(2TP+FP+FN) (0 when the denominator is 0), in float64."""
    c = np.asarray(counts, dtype=np.float64).reshape(-1, 4)
    tp, fp, fn, tn = c[:, 0], c[:, 1], c[:, 2], c[:, 3]
    tot = tp + fp + fn + tn
    acc = np.where(tot > 0, (tp + tn) / np.where(tot > 0, tot, 1), 0.0)
    den = 2 * tp + fp + fn
    f1 = np.where(den > 0, 2 * tp / np.where(den > 0, den, 1), 0.0)
    return acc, f1
