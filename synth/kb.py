"""Seeded synthetic knowledge bases with the shapes of the paper's workloads.

A KB here is plain host data:

* concept membership bitsets, uint32 words, bit i of word w is individual
  32*w + i (LSB first); each row padded to ``wp`` words (a multiple of 4, so a
  row starts on a 16-byte boundary); bits >= n are zero;
* per role a CSR (``row_ptr`` uint32[n+1], ``col`` uint32[E]) with sorted,
  duplicate-free rows, plus the inverse CSR (the transpose), whose rows come out
  sorted because it is built by a stable sort of the forward edges by object;
* numeric data properties as float32[n], NaN where the value is missing;
* numeric concrete roles (several values per individual, Section III-B) as a
  CSR over individuals (``num_row_ptr`` uint32[n+1], ``num_vals`` float32[M]);
  their property ids follow the one-value properties' (``n_props + q``);
* string concrete roles as a CSR of interned string ids over individuals
  (``str_row_ptr``, ``str_ids`` uint32[M]) into a table of distinct strings
  (``strings``), with a list of substring patterns (``patterns``);
* positive and negative example sets (bitsets and index lists).

Degree laws, value distributions and example counts follow the workload
descriptions.  The generator draws random numbers only from the counter-based
streams in :mod:`synth.rng`, so every array is a pure function of the seed.
It holds none of the evaluation method's arithmetic.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

from . import rng

# The heavy loops (per-row target draws, transposes, Bernoulli bitsets) have a
# multithreaded C twin in fastgen.c that produces the same arrays; the numpy
# versions below define the recipe and are kept for checking it.
USE_C = True
_HERE = os.path.dirname(os.path.abspath(__file__))
_FAST = None
_FAST_LOCK = threading.Lock()


def _fast():
    global _FAST
    with _FAST_LOCK:
        if _FAST is None:
            src = os.path.join(_HERE, "fastgen.c")
            lib = os.path.join(_HERE, "libfastgen.so")
            if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
                tmp = lib + f".{os.getpid()}.tmp"
                subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", tmp, src])
                os.replace(tmp, lib)
            L = ctypes.CDLL(lib)
            P, U64, I64, I32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32
            L.fastgen_targets.argtypes = [U64, U64, U64, U64, P, I64, U64, P, P, I64, ctypes.c_double, P, I32]
            L.fastgen_targets.restype = ctypes.c_int
            L.fastgen_transpose.argtypes = [P, P, I64, P, P]
            L.fastgen_transpose.restype = None
            L.fastgen_bernoulli.argtypes = [U64, U64, U64, ctypes.c_double, ctypes.c_double, P, P, I32]
            L.fastgen_bernoulli.restype = None
            L.fastgen_refine.argtypes = [U64, U64, P, P, I64, I64, I64, I64, I64, P, P, P, I64, P]
            L.fastgen_refine.restype = ctypes.c_int
            _FAST = L
    return _FAST


def _threads() -> int:
    return max(1, min(64, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()))

# sub-stream ids (one per component, so components are independent)
S_CONCEPT_P = 1
S_DAG = 2
S_PROP_VAL = 3
S_PROP_MISS = 4
S_EXAMPLES = 5
S_LATENT = 6
S_BIAS = 5 << 16
S_CONCEPT = 1 << 16
S_ROLE_DEG = 2 << 16
S_ROLE_TGT = 3 << 16
S_PROP = 4 << 16
S_NUM_DEG = 12 << 16
S_NUM_VAL = 13 << 16
S_STR_DEG = 14 << 16
S_STR_ID = 15 << 16
S_STR_TABLE = 16 << 16
S_PATTERN = 17 << 16


@dataclass(frozen=True)
class KBConfig:
    name: str
    seed: int
    n: int
    n_concepts: int
    p_lo: float
    p_hi: float
    dag: bool
    n_roles: int
    degree: Tuple            # ("poisson", lam) | ("zipf", a, mean, cap) | ("single",) | ("unique",)
    n_props: int
    prop_dist: Tuple         # ("uniform", lo, hi) | ("lognormal", mu, sigma) | ("normal", mu, sd)
    missing: float
    n_pos: int
    n_neg: int
    planted: bool = False    # examples from a latent class that some concepts, role 0 and property 0 track
    n_num_roles: int = 0     # numeric concrete roles (values from prop_dist)
    num_degree: Tuple = ("poisson", 3.0)   # values per individual: ("poisson", lam) | ("single", m) | ("unique",)
    n_str_roles: int = 0     # string concrete roles
    str_degree: Tuple = ("poisson", 2.0)   # values per individual, as num_degree
    n_strings: int = 0       # distinct strings in the table (lengths str_len, letters of an alphabet)
    str_len: Tuple = (3, 12)
    alphabet: int = 6
    n_patterns: int = 0      # substring patterns (the first is the empty string)

    def scaled(self, n: int, **kw) -> "KBConfig":
        """Same distributions on ``n`` individuals (example counts scaled)."""
        f = n / self.n
        d = dict(n=n, n_pos=max(1, int(round(self.n_pos * f))), n_neg=max(1, int(round(self.n_neg * f))))
        d.update(kw)
        return replace(self, **d)


CONFIGS = {
    # plain single-hypothesis evaluation on a small KB
    "small": KBConfig("small", 1, 10_000, 50, 0.02, 0.30, True, 8, ("poisson", 3.0), 4,
                   ("uniform", 0.0, 100.0), 0.20, 200, 200),
    # single large hypothesis latency
    "large": KBConfig("large", 2, 10_000_000, 200, 0.01, 0.50, False, 32, ("zipf", 2.1, 8.0, 10_000), 16,
                   ("lognormal", 0.0, 1.0), 0.10, 100_000, 100_000),
    # batched exact evaluation
    "batch": KBConfig("batch", 3, 1_000_000, 100, 0.01, 0.50, False, 16, ("poisson", 6.0), 8,
                   ("uniform", 0.0, 1000.0), 0.0, 10_000, 10_000),
    # refinement search
    "search": KBConfig("search", 5, 4_000_000, 300, 0.01, 0.50, False, 64, ("zipf", 2.3, 10.0, 10_000), 32,
                   ("normal", 50.0, 15.0), 0.15, 50_000, 50_000, planted=True),
}
CONFIGS["surrogate"] = replace(CONFIGS["large"], name="surrogate", seed=4, planted=True)
# numeric concrete roles: 10^7 individuals, 8 roles with Poisson(4) values each
# (4 * 10^7 assertions, 200 MB per role), values U[0, 1000]
CONFIGS["numeric"] = KBConfig("numeric", 6, 10_000_000, 8, 0.01, 0.50, False, 0, ("poisson", 3.0), 0,
                              ("uniform", 0.0, 1000.0), 0.0, 10_000, 10_000, n_num_roles=8,
                              num_degree=("poisson", 4.0))
# string concrete roles: 10^7 individuals, 8 roles with Poisson(2) values each
# (2 * 10^7 ids, 120 MB of row pointers and ids per role) into a table of
# 100,000 distinct strings of 3-12 letters over a 6-letter alphabet; 64 patterns
CONFIGS["strings"] = KBConfig("strings", 7, 10_000_000, 8, 0.01, 0.50, False, 0, ("poisson", 3.0), 0,
                              ("uniform", 0.0, 1.0), 0.0, 10_000, 10_000, n_str_roles=8,
                              str_degree=("poisson", 2.0), n_strings=100_000, str_len=(3, 12), alphabet=6,
                              n_patterns=64)

# Planted structure (workloads that search or learn need a signal): a latent
# class Z (a uniform 20 % of the individuals) supplies the positives, its
# complement the negatives; concepts 0-2 have higher membership inside Z,
# role 0 sends 70 % of a Z member's edges to members of concept 3, and
# property 0 is shifted upwards inside Z.  Only random draws are correlated:
# no concept is evaluated to make the examples.
LATENT_FRAC = 0.2
PLANT_P_IN = (0.7, 0.5, 0.4)
PLANT_P_OUT = (0.1, 0.15, 0.2)
PLANT_ROLE_BIAS = 0.7


def words(n: int) -> Tuple[int, int]:
    w = (n + 31) // 32
    return w, (w + 3) // 4 * 4


def pack_bits(member: np.ndarray, wp: int) -> np.ndarray:
    """bool[n] -> uint32[wp] LSB-first, zero padded."""
    b = np.packbits(member.astype(bool), bitorder="little")
    out = np.zeros(wp * 4, dtype=np.uint8)
    out[: b.size] = b
    return out.view("<u4").copy()


def unpack_bits(bits: np.ndarray, n: int) -> np.ndarray:
    """uint32[>=W] -> bool[n]."""
    b = np.ascontiguousarray(bits, dtype="<u4").view(np.uint8)
    return np.unpackbits(b, bitorder="little")[:n].astype(bool)


# --------------------------------------------------------------------------- degree laws
def poisson_cdf(lam: float, kmax: int) -> np.ndarray:
    p = np.empty(kmax + 1)
    p[0] = math.exp(-lam)
    for k in range(1, kmax + 1):
        p[k] = p[k - 1] * lam / k
    c = np.cumsum(p)
    c[-1] = 1.0
    return c


def shifted_zipf_pmf(a: float, s: float, cap: int) -> np.ndarray:
    d = np.arange(cap + 1, dtype=np.float64)
    w = (d + s) ** (-a)
    return w / w.sum()


def solve_zipf_shift(a: float, mean: float, cap: int) -> float:
    """Shift s with E[d] = mean for P(d) proportional to (d+s)^-a on {0..cap}.

    The mean grows with s, so bisection on s finds it.
    """
    d = np.arange(cap + 1, dtype=np.float64)
    lo, hi = 1e-6, 1e6
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        m = float((shifted_zipf_pmf(a, mid, cap) * d).sum())
        if m < mean:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)


def draw_degrees(cfg: KBConfig, r: int, n: int) -> Tuple[np.ndarray, dict]:
    kind = cfg.degree[0]
    meta = {}
    if kind == "poisson":
        cdf = poisson_cdf(cfg.degree[1], 200)
        u = rng.uniform_range(cfg.seed, S_ROLE_DEG + r, n)
        deg = np.searchsorted(cdf, u, side="right")
    elif kind == "zipf":
        a, mean, cap = cfg.degree[1], cfg.degree[2], int(cfg.degree[3])
        s = solve_zipf_shift(a, mean, cap)
        meta["zipf_shift"] = s
        cdf = np.cumsum(shifted_zipf_pmf(a, s, cap))
        cdf[-1] = 1.0
        u = rng.uniform_range(cfg.seed, S_ROLE_DEG + r, n)
        deg = np.searchsorted(cdf, u, side="right")
    elif kind == "single":        # the paper's "single subject" set: one subject holds every edge
        e = int(cfg.degree[1]) if len(cfg.degree) > 1 else n
        deg = np.zeros(n, dtype=np.int64)
        deg[int(rng.randint(cfg.seed, S_ROLE_DEG + r, np.array([0]), n)[0])] = min(e, n)
    elif kind == "unique":        # the paper's "unique subject" set: each subject has one edge
        deg = np.ones(n, dtype=np.int64)
    else:
        raise ValueError(kind)
    return np.minimum(deg.astype(np.int64), n), meta


def draw_targets(cfg: KBConfig, r: int, deg: np.ndarray, n: int, bias=None) -> np.ndarray:
    """Uniform targets, without replacement within a row, rows sorted ascending.

    bias = (subject mask, target pool, p): an edge of a masked subject takes a
    uniform target from the pool with probability p (before duplicates are
    redrawn uniformly)."""
    e = int(deg.sum())
    rows = np.repeat(np.arange(n, dtype=np.int64), deg)
    if cfg.degree[0] == "unique":
        # a permutation: subject i -> pi(i)
        key = rng.u64(cfg.seed, S_ROLE_TGT + r, np.arange(n, dtype=np.uint64))
        return np.argsort(key, kind="stable").astype(np.uint32)
    if USE_C and e:
        rp = np.zeros(n + 1, dtype=np.uint64)
        np.cumsum(deg, out=rp[1:])
        col = np.empty(e, dtype=np.uint32)
        smask = pool = None
        pb = 0.0
        if bias is not None:
            smask = np.ascontiguousarray(bias[0], dtype=np.uint8)
            pool = np.ascontiguousarray(bias[1], dtype=np.int64)
            pb = float(bias[2])
        rc = _fast().fastgen_targets(cfg.seed, S_ROLE_TGT + r, S_BIAS + r, S_BIAS + 1000 + r, rp.ctypes.data, n, n,
                                     smask.ctypes.data if smask is not None else None,
                                     pool.ctypes.data if pool is not None and pool.size else None,
                                     0 if pool is None else pool.size, pb, col.ctypes.data, _threads())
        if rc:
            raise RuntimeError("could not draw distinct targets")
        return col
    tgt = rng.randint(cfg.seed, S_ROLE_TGT + r, np.arange(e, dtype=np.uint64), n)
    if bias is not None and e:
        smask, pool, pb = bias
        ei = np.arange(e, dtype=np.uint64)
        take = smask[rows] & (rng.uniform(cfg.seed, S_BIAS + r, ei) < pb)
        pick = rng.randint(cfg.seed, S_BIAS + 1000 + r, ei, max(pool.size, 1))
        if pool.size:
            tgt = np.where(take, pool[np.minimum(pick, pool.size - 1)], tgt)
    attempt = 0
    while True:
        key = rows * n + tgt
        order = np.argsort(key, kind="stable")
        key = key[order]
        tgt = tgt[order]
        dup = np.zeros(e, dtype=bool)
        if e > 1:
            dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0:
            return tgt.astype(np.uint32)
        attempt += 1
        idx = np.nonzero(dup)[0].astype(np.uint64) + np.uint64(attempt) * np.uint64(1 << 40)
        tgt[dup] = rng.randint(cfg.seed, S_ROLE_TGT + r, idx, n)
        if attempt > 10_000:
            raise RuntimeError("could not draw distinct targets")


def transpose_csr(row_ptr: np.ndarray, col: np.ndarray, n: int) -> Tuple[np.ndarray, np.ndarray]:
    """Inverse CSR: a stable sort of the edges by object keeps subjects ascending per row."""
    if USE_C and col.size:
        rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
        c = np.ascontiguousarray(col, dtype=np.uint32)
        irp = np.empty(n + 1, dtype=np.uint64)
        icol = np.empty(c.size, dtype=np.uint32)
        _fast().fastgen_transpose(rp.ctypes.data, c.ctypes.data, n, irp.ctypes.data, icol.ctypes.data)
        return irp.astype(np.uint32), icol
    deg = np.diff(row_ptr.astype(np.int64))
    subj = np.repeat(np.arange(n, dtype=np.uint32), deg)
    order = np.argsort(col, kind="stable")
    inv_col = subj[order].astype(np.uint32)
    cnt = np.bincount(col.astype(np.int64), minlength=n)
    inv_ptr = np.zeros(n + 1, dtype=np.uint32)
    np.cumsum(cnt, out=inv_ptr[1:])
    return inv_ptr, inv_col


# --------------------------------------------------------------------------- the KB
@dataclass
class KB:
    cfg: KBConfig
    n: int
    w: int
    wp: int
    concept_bits: np.ndarray          # uint32 [C][wp]
    row_ptr: List[np.ndarray]         # per role uint32 [n+1]
    col: List[np.ndarray]             # per role uint32 [E]
    inv_row_ptr: List[np.ndarray]
    inv_col: List[np.ndarray]
    prop_vals: np.ndarray             # float32 [P][n]
    pos_idx: np.ndarray
    neg_idx: np.ndarray
    pos_bits: np.ndarray              # uint32 [wp]
    neg_bits: np.ndarray
    meta: dict
    num_row_ptr: List[np.ndarray] = field(default_factory=list)   # per numeric role uint32 [n+1]
    num_vals: List[np.ndarray] = field(default_factory=list)      # per numeric role float32 [M]
    str_row_ptr: List[np.ndarray] = field(default_factory=list)   # per string role uint32 [n+1]
    str_ids: List[np.ndarray] = field(default_factory=list)       # per string role uint32 [M], ids into strings
    strings: List[bytes] = field(default_factory=list)            # the table (distinct)
    patterns: List[bytes] = field(default_factory=list)

    @property
    def n_concepts(self) -> int:
        return self.concept_bits.shape[0]

    @property
    def n_roles(self) -> int:
        return len(self.row_ptr)

    @property
    def n_props(self) -> int:
        return self.prop_vals.shape[0]

    @property
    def n_num_roles(self) -> int:
        return len(self.num_row_ptr)

    @property
    def n_str_roles(self) -> int:
        return len(self.str_row_ptr)

    @property
    def n_patterns(self) -> int:
        return len(self.patterns)

    def n_edges(self, r: int) -> int:
        return int(self.col[r].size)

    def nbytes(self) -> int:
        t = self.concept_bits.nbytes + self.prop_vals.nbytes + 2 * self.pos_bits.nbytes
        for r in range(self.n_roles):
            t += 2 * self.row_ptr[r].nbytes + 2 * self.col[r].nbytes
        for q in range(self.n_num_roles):
            t += self.num_row_ptr[q].nbytes + self.num_vals[q].nbytes
        for q in range(self.n_str_roles):
            t += self.str_row_ptr[q].nbytes + self.str_ids[q].nbytes
        return t + sum(len(x) for x in self.strings)


def latent_class(cfg: KBConfig) -> np.ndarray:
    return rng.uniform_range(cfg.seed, S_LATENT, cfg.n) < LATENT_FRAC


def gen_concepts(cfg: KBConfig, wp: int, meta: dict, z=None) -> np.ndarray:
    n, c = cfg.n, cfg.n_concepts
    p = cfg.p_lo + (cfg.p_hi - cfg.p_lo) * rng.uniform_range(cfg.seed, S_CONCEPT_P, c)
    bits = np.zeros((c, wp), dtype=np.uint32)
    zz = np.ascontiguousarray(z, dtype=np.uint8) if z is not None else None
    for j in range(c):
        planted = z is not None and j < len(PLANT_P_IN)
        if USE_C:
            buf = np.zeros(wp * 4, dtype=np.uint8)
            p_out, p_in = (PLANT_P_OUT[j], PLANT_P_IN[j]) if planted else (p[j], p[j])
            _fast().fastgen_bernoulli(cfg.seed, S_CONCEPT + j, n, float(p_out), float(p_in),
                                      zz.ctypes.data if planted else None, buf.ctypes.data, _threads())
            bits[j] = buf.view("<u4")
            continue
        u = rng.uniform_range(cfg.seed, S_CONCEPT + j, n)
        if planted:
            member = u < np.where(z, PLANT_P_IN[j], PLANT_P_OUT[j])
        else:
            member = u < p[j]
        bits[j] = pack_bits(member, wp)
    if cfg.dag and c > 1:
        # random subsumption forest: concept j < C has parent pj < j with prob 1/2
        # (so the edges form a DAG); the ABox is closed downward, i.e. every
        # member of a sub-concept is also a member of its super-concept.
        j = np.arange(c, dtype=np.uint64)
        has = rng.uniform(cfg.seed, S_DAG, j * np.uint64(2)) < 0.5
        parent = np.full(c, -1, dtype=np.int64)
        for k in range(1, c):
            if has[k]:
                parent[k] = int(rng.randint(cfg.seed, S_DAG, np.array([2 * k + 1], dtype=np.uint64), k)[0])
        for k in range(c - 1, 0, -1):       # children have larger ids: finish them first
            if parent[k] >= 0:
                bits[parent[k]] |= bits[k]
        meta["dag_parent"] = parent.tolist()
    return bits


def draw_values(cfg: KBConfig, stream: int, m: int) -> np.ndarray:
    """m float64 draws from the configuration's value distribution."""
    kind = cfg.prop_dist[0]
    if kind == "uniform":
        lo, hi = cfg.prop_dist[1], cfg.prop_dist[2]
        return lo + (hi - lo) * rng.uniform_range(cfg.seed, stream, m)
    if kind == "lognormal":
        return np.exp(cfg.prop_dist[1] + cfg.prop_dist[2] * rng.normal(cfg.seed, stream, m))
    if kind == "normal":
        return cfg.prop_dist[1] + cfg.prop_dist[2] * rng.normal(cfg.seed, stream, m)
    raise ValueError(kind)


def gen_props(cfg: KBConfig, z=None) -> np.ndarray:
    n = cfg.n
    out = np.empty((cfg.n_props, n), dtype=np.float32)
    for p in range(cfg.n_props):
        v = draw_values(cfg, S_PROP + p, n)
        if z is not None and p == 0:   # planted: property 0 shifted up inside the latent class
            lo, hi = np.nanmin(v), np.nanmax(v)
            v = np.where(z, v + 0.25 * (hi - lo), v)
        v = v.astype(np.float32)
        if cfg.missing > 0:
            miss = rng.uniform_range(cfg.seed, S_PROP_MISS * 1000 + p, n) < cfg.missing
            v[miss] = np.nan
        out[p] = v
    return out


def _degrees(cfg: KBConfig, law: Tuple, stream: int) -> np.ndarray:
    n = cfg.n
    if law[0] == "poisson":
        cdf = poisson_cdf(law[1], 200)
        return np.searchsorted(cdf, rng.uniform_range(cfg.seed, stream, n), side="right")
    if law[0] == "single":       # one individual holds every value
        deg = np.zeros(n, dtype=np.int64)
        deg[int(rng.randint(cfg.seed, stream, np.array([0]), n)[0])] = int(law[1])
        return deg
    if law[0] == "unique":       # one value per individual
        return np.ones(n, dtype=np.int64)
    raise ValueError(law[0])


def gen_strings(cfg: KBConfig) -> Tuple[List[bytes], List[bytes]]:
    """The string table (distinct strings of lengths str_len over the first
    `alphabet` lowercase letters) and the patterns: the empty string, then
    substrings of length 1-4 of table strings, then (the last) a string longer
    than any in the table."""
    table, seen = [], set()
    r = rng.Rng(cfg.seed, S_STR_TABLE)
    lo, hi = cfg.str_len
    letters = b"abcdefghijklmnopqrstuvwxyz"[: cfg.alphabet]
    while len(table) < cfg.n_strings:
        k = r.randint(lo, hi)
        x = bytes(letters[r.randint(0, len(letters) - 1)] for _ in range(k))
        if x not in seen:
            seen.add(x)
            table.append(x)
    pats = []
    if cfg.n_patterns:
        pr = rng.Rng(cfg.seed, S_PATTERN)
        pats.append(b"")
        while len(pats) < cfg.n_patterns - 1 and table:
            x = table[pr.randint(0, len(table) - 1)]
            k = pr.randint(1, min(4, len(x))) if x else 0
            i = pr.randint(0, len(x) - k)
            pats.append(x[i: i + k])
        if len(pats) < cfg.n_patterns:
            pats.append(letters[:1] * (hi + 1))
    return table, pats


def gen_str_roles(cfg: KBConfig, n_strings: int) -> Tuple[List[np.ndarray], List[np.ndarray]]:
    """String concrete roles as CSR over individuals of uniform string ids."""
    rps, ids = [], []
    for q in range(cfg.n_str_roles):
        deg = _degrees(cfg, cfg.str_degree, S_STR_DEG + q)
        rp = np.zeros(cfg.n + 1, dtype=np.uint32)
        np.cumsum(deg, out=rp[1:])
        rps.append(rp)
        m = int(rp[-1])
        ids.append(rng.randint(cfg.seed, S_STR_ID + q, np.arange(m, dtype=np.uint64), max(n_strings, 1))
                   .astype(np.uint32))
    return rps, ids


def gen_num_roles(cfg: KBConfig) -> Tuple[List[np.ndarray], List[np.ndarray]]:
    """Numeric concrete roles as CSR over individuals: the number of values of
    each individual from ``num_degree`` (the paper's "single subject" and
    "unique subject" shapes included), the values from ``prop_dist``."""
    n = cfg.n
    rps, vals = [], []
    for q in range(cfg.n_num_roles):
        kind = cfg.num_degree[0]
        if kind == "poisson":
            cdf = poisson_cdf(cfg.num_degree[1], 200)
            deg = np.searchsorted(cdf, rng.uniform_range(cfg.seed, S_NUM_DEG + q, n), side="right")
        elif kind == "single":       # one individual holds every value
            deg = np.zeros(n, dtype=np.int64)
            deg[int(rng.randint(cfg.seed, S_NUM_DEG + q, np.array([0]), n)[0])] = int(cfg.num_degree[1])
        elif kind == "unique":       # one value per individual
            deg = np.ones(n, dtype=np.int64)
        else:
            raise ValueError(kind)
        rp = np.zeros(n + 1, dtype=np.uint32)
        np.cumsum(deg, out=rp[1:])
        rps.append(rp)
        vals.append(draw_values(cfg, S_NUM_VAL + q, int(rp[-1])).astype(np.float32))
    return rps, vals


def gen_examples(cfg: KBConfig, wp: int, z=None) -> Tuple[np.ndarray, np.ndarray]:
    """Disjoint uniform positive / negative sets (sorted index arrays); with a
    latent class z, positives are drawn inside it and negatives outside."""
    n = cfg.n
    if cfg.n_pos + cfg.n_neg > n:
        raise ValueError("more examples than individuals")
    key = rng.u64(cfg.seed, S_EXAMPLES, np.arange(n, dtype=np.uint64))
    perm = np.argsort(key, kind="stable")
    if z is not None:
        inside, outside = perm[z[perm]], perm[~z[perm]]
        if inside.size < cfg.n_pos or outside.size < cfg.n_neg:
            raise ValueError("latent class too small for the examples")
        return (np.sort(inside[: cfg.n_pos]).astype(np.int64), np.sort(outside[: cfg.n_neg]).astype(np.int64))
    pos = np.sort(perm[: cfg.n_pos]).astype(np.int64)
    neg = np.sort(perm[cfg.n_pos: cfg.n_pos + cfg.n_neg]).astype(np.int64)
    return pos, neg


def generate(cfg: KBConfig, roles: Optional[int] = None) -> KB:
    n = cfg.n
    w, wp = words(n)
    meta = {"seed": cfg.seed, "config": cfg.name}
    z = latent_class(cfg) if cfg.planted else None
    cb = gen_concepts(cfg, wp, meta, z)
    pool = None
    if z is not None and cfg.n_concepts > 3:
        pool = np.nonzero(unpack_bits(cb[3], n))[0].astype(np.int64)
    rps, cols, irps, icols = [], [], [], []
    for r in range(cfg.n_roles if roles is None else roles):
        deg, m = draw_degrees(cfg, r, n)
        meta.update(m)
        bias = (z, pool, PLANT_ROLE_BIAS) if (r == 0 and pool is not None) else None
        tgt = draw_targets(cfg, r, deg, n, bias)
        rp = np.zeros(n + 1, dtype=np.uint32)
        np.cumsum(deg, out=rp[1:])
        rps.append(rp)
        cols.append(tgt)
        ip, ic = transpose_csr(rp, tgt, n)
        irps.append(ip)
        icols.append(ic)
    props = gen_props(cfg, z)
    pos, neg = gen_examples(cfg, wp, z)
    mp = np.zeros(n, dtype=bool)
    mp[pos] = True
    mn = np.zeros(n, dtype=bool)
    mn[neg] = True
    nrp, nv = gen_num_roles(cfg)
    table, pats = gen_strings(cfg) if (cfg.n_str_roles or cfg.n_patterns) else ([], [])
    srp, sid = gen_str_roles(cfg, len(table))
    return KB(cfg, n, w, wp, cb, rps, cols, irps, icols, props, pos, neg,
              pack_bits(mp, wp), pack_bits(mn, wp), meta, nrp, nv, srp, sid, table, pats)


def from_arrays(n: int, concepts: List[List[int]], roles: List[List[Tuple[int, int]]],
                props: List[List[float]], pos: List[int], neg: List[int],
                num_roles: Optional[List[List[Tuple[int, float]]]] = None,
                str_roles: Optional[List[List[Tuple[int, int]]]] = None, strings: Optional[List[bytes]] = None,
                patterns: Optional[List[bytes]] = None) -> KB:
    """Small hand-written KB (fixtures): concepts as member lists, roles as edge
    lists, numeric concrete roles as (individual, value) lists in any order,
    string concrete roles as (individual, string id) lists into `strings`."""
    w, wp = words(n)
    cb = np.zeros((max(len(concepts), 0), wp), dtype=np.uint32)
    for j, mem in enumerate(concepts):
        m = np.zeros(n, dtype=bool)
        m[list(mem)] = True
        cb[j] = pack_bits(m, wp)
    rps, cols, irps, icols = [], [], [], []
    for edges in roles:
        es = sorted(set((int(a), int(b)) for a, b in edges))
        rp = np.zeros(n + 1, dtype=np.uint32)
        for a, _ in es:
            rp[a + 1] += 1
        rp = np.cumsum(rp).astype(np.uint32)
        col = np.array([b for _, b in es], dtype=np.uint32)
        rps.append(rp)
        cols.append(col)
        ip, ic = transpose_csr(rp, col, n)
        irps.append(ip)
        icols.append(ic)
    pv = np.array(props, dtype=np.float32).reshape(len(props), n) if props else np.zeros((0, n), np.float32)
    mp = np.zeros(n, dtype=bool)
    mp[list(pos)] = True
    mn = np.zeros(n, dtype=bool)
    mn[list(neg)] = True
    cfg = KBConfig("fixture", 0, n, len(concepts), 0, 0, False, len(roles), ("fixture",), len(props),
                   ("fixture",), 0.0, len(pos), len(neg))
    nrp, nv = [], []
    for assertions in num_roles or []:
        order = sorted(range(len(assertions)), key=lambda k: int(assertions[k][0]))   # stable: keeps value order
        rp = np.zeros(n + 1, dtype=np.uint32)
        for a, _ in assertions:
            rp[int(a) + 1] += 1
        nrp.append(np.cumsum(rp).astype(np.uint32))
        nv.append(np.array([assertions[k][1] for k in order], dtype=np.float32))
    srp, sid = [], []
    for assertions in str_roles or []:
        order = sorted(range(len(assertions)), key=lambda k: int(assertions[k][0]))
        rp = np.zeros(n + 1, dtype=np.uint32)
        for a, _ in assertions:
            rp[int(a) + 1] += 1
        srp.append(np.cumsum(rp).astype(np.uint32))
        sid.append(np.array([assertions[k][1] for k in order], dtype=np.uint32))
    return KB(cfg, n, w, wp, cb, rps, cols, irps, icols, pv, np.array(sorted(pos), dtype=np.int64),
              np.array(sorted(neg), dtype=np.int64), pack_bits(mp, wp), pack_bits(mn, wp), {}, nrp, nv,
              srp, sid, list(strings or []), list(patterns or []))
