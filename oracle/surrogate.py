"""Oracle of the learned surrogate (TEST INFRASTRUCTURE).

The paper has no learned component; the surrogate only orders and prunes the
exact-evaluation queue.  This module is the plain reference it is checked
against, written from the definitions below (no code shared with the GPU
library):

* ``encode``: the 512-dimensional structural encoding of a postfix program,
  computed by direct counting over the program;
* ``forward`` / ``backward``: the MLP 512 -> 512 -> 512 -> 2 with ReLU,
  mean-squared-error loss (optionally on targets standardised by a target
  map, rows of the upper tail weighted more), in float64; ``bf16`` rounding (round to nearest,
  ties to even, from the float32 bit pattern) is applied where the GPU stores
  bfloat16 (inputs, weights, hidden activations, their gradients);
* ``adam``: one Adam step (Kingma and Ba, 2015) on float32 master weights;
* ``ranking``: the total order used to rank hypotheses (accuracy desc, F1
  desc, length asc, program bytes asc, index asc) and recall@k.

Encoding (feature index ranges; every value but the prior is an integer
count scaled by 1/4, exact in bfloat16).  Node depth is the distance from the
root (root 0); "height" is the tree height (leaves 1), clamped to 8.
Polarity is 0 at the root; NOT and ATMOST flip it for their operand, every
other constructor passes it on, so a node's polarity says whether the
hypothesis grows (0) or shrinks (1) with its instance set.  A *signed* count
adds +1 for an occurrence at polarity 0 and -1 at polarity 1.  A data
threshold t of property p falls in bucket q = #{g in grid[p] : g < t} of a
per-property grid of 15 increasing boundaries (the property's quantiles,
supplied with the programs; q = 0 without a grid or for NaN t).  String
restrictions (SEQ, SCONTAINS) have no features of their own: they count only
in the length, depth and height features.
  [  0, 84) op histogram per depth: min(depth, 5)*14 + op-1
  [ 84,180) atomic concept, signed: concept id mod 96
  [180,244) role: (role id mod 32)*2 + inverse flag
  [244,284) role-restriction kind per depth: min(depth, 7)*5 + (op - EXISTS)
  [284,308) cardinality: (op - ATLEAST)*8 + min(n, 7)
  [308,436) >= and <= restrictions, signed: ((property id mod 16)*2 + (op - DGE))*4 + q // 4
  [436,493) role restriction over an atom, signed: ((role*2 + inverse)*131 + concept) mod 57
  [493,497) length bucket: min(len, 39) // 10
  [497,504) statistics, signed sums of the KB's own per-symbol scores (a table
            the caller computes with the engine; 0 without one): atoms by
            depth bucket min(depth // 2, 2) (497-499), >= / <= restrictions
            by depth bucket (500-502) with the score of their (property,
            compare, threshold bucket q), the atom fillers of role
            restrictions (503)
  [504,508) counts of leaves, role restrictions, data restrictions, NOTs
  [508]     height - 1 (clamped to 7)
  [509]     constant 4 (a bias input; 4 * 1/4 = 1)
  [510,512) prior: two caller-supplied values per program (the search passes
            the exact accuracy and F1 of the hypothesis a candidate refines),
            rounded to bfloat16, not scaled; 0 without a prior
"""
from __future__ import annotations

import math
from typing import Optional, Dict, List, Sequence, Tuple

import numpy as np

D_IN = 512
D_H = 512
D_OUT = 2
_ATOM, _TOP, _BOT, _NOT, _AND, _OR = 1, 2, 3, 4, 5, 6
_EX, _ALL, _MIN, _MAX, _EXACT = 7, 8, 9, 10, 11
_GE, _LE, _EQ = 12, 13, 14


def _arity(op: int) -> int:
    if op in (_NOT, _EX, _ALL, _MIN, _MAX, _EXACT):
        return 1
    if op in (_AND, _OR):
        return 2
    return 0


def encode(prog: Sequence[int], grid=None, prior=None, stats=None) -> np.ndarray:
    """Structural encoding of one postfix program (float32[512]).

    grid: per-property threshold boundaries, float32 [n_props][15], or None.
    prior: two floats (features 510, 511), or None.
    stats: (atom_scores int[n_concepts], threshold_scores int[n_props][2][16])
    or None; a symbol outside the tables scores 0.
    A program longer than 256 instructions is encoded by its last 256 (the
    root and the nodes nearest to it)."""
    prog = list(prog)[-256:]
    L = len(prog)
    # node depths and polarities: read the postfix backwards (a pre-order
    # walk, right child first); NOT and ATMOST flip their operand's polarity
    depth = [0] * L
    pol = [0] * L
    pending = [(0, 0)]
    height = 0
    for k in range(L - 1, -1, -1):
        d, pl = pending.pop()
        depth[k] = d
        pol[k] = pl
        height = max(height, d + 1)
        op = int(prog[k]) & 0xFF
        child_pol = pl ^ 1 if op in (_NOT, _MAX) else pl
        for _ in range(_arity(op)):
            pending.append((d + 1, child_pol))
    atoms_t, thr_t = (None, None) if stats is None else stats

    def atom_score(c):
        return int(atoms_t[c]) if atoms_t is not None and c < len(atoms_t) else 0

    def thr_score(p, o, q):
        return int(thr_t[p][o][q]) if thr_t is not None and p < len(thr_t) else 0

    f = np.zeros(D_IN, dtype=np.int64)
    leaves = roles = datas = nots = 0
    for k in range(L):
        w = int(prog[k])
        op, inv, a, b = w & 0xFF, (w >> 8) & 1, (w >> 16) & 0xFFFF, (w >> 32) & 0xFFFFFFFF
        sign = 1 - 2 * pol[k]
        if not 1 <= op <= 14:       # no feature: not an op, or a string restriction (ops 15-16)
            continue
        f[min(depth[k], 5) * 14 + op - 1] += 1
        if _arity(op) == 0:
            leaves += 1
        if op == _ATOM:
            f[84 + a % 96] += sign
            f[497 + min(depth[k] // 2, 2)] += sign * atom_score(a)
        elif _EX <= op <= _EXACT:
            roles += 1
            f[180 + (a % 32) * 2 + inv] += 1
            f[244 + min(depth[k], 7) * 5 + (op - _EX)] += 1
            if op >= _MIN:
                f[284 + (op - _MIN) * 8 + min(b, 7)] += 1
            child = int(prog[k - 1])       # the filler ends right before its restriction
            if child & 0xFF == _ATOM:
                c = (child >> 16) & 0xFFFF
                f[436 + ((a * 2 + inv) * 131 + c) % 57] += sign
                f[503] += sign * atom_score(c)
        elif _GE <= op <= _EQ:
            datas += 1
            if op != _EQ:
                t = np.array([b], np.uint32).view(np.float32)[0]
                q = 0
                if grid is not None and a < len(grid) and not np.isnan(t):
                    q = int(np.sum(np.asarray(grid[a], np.float32) < t))
                f[308 + ((a % 16) * 2 + (op - _GE)) * 4 + q // 4] += sign
                f[500 + min(depth[k] // 2, 2)] += sign * thr_score(a, op - _GE, q)
        elif op == _NOT:
            nots += 1
    f[493 + min(L, 39) // 10] += 1
    f[504] += leaves
    f[505] += roles
    f[506] += datas
    f[507] += nots
    f[508] += min(height, 8) - 1
    f[509] += 4
    out = (f.astype(np.float64) * 0.25).astype(np.float32)
    if prior is not None:
        out[510:512] = bf16(np.asarray(prior, np.float32).reshape(2))
    return out


def threshold_grid(prop_vals: np.ndarray) -> np.ndarray:
    """15 quantile boundaries (1/16 .. 15/16) of each property's present values, float32."""
    out = np.zeros((prop_vals.shape[0], 15), np.float32)
    for p in range(prop_vals.shape[0]):
        v = prop_vals[p][~np.isnan(prop_vals[p])]
        if v.size:
            out[p] = np.quantile(v.astype(np.float64), np.arange(1, 16) / 16.0).astype(np.float32)
    return out


def encode_batch(progs: Sequence[Sequence[int]], grid=None, prior=None, stats=None) -> np.ndarray:
    """prior: float [H][2] or None; stats as for ``encode``."""
    if not len(progs):
        return np.zeros((0, D_IN), np.float32)
    return np.stack([encode(p, grid, None if prior is None else prior[i], stats) for i, p in enumerate(progs)])


def stat_score(acc: float) -> int:
    """Table entry of a symbol whose exact accuracy on the examples is acc: round((acc - 1/2) * 32),
    ties to even (float64)."""
    return int(np.rint((np.float64(acc) - 0.5) * 32.0))


# ---------------------------------------------------------------------------- bfloat16
def bf16(x) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    nan = np.isnan(a)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    out = np.where(nan, a, out)
    return out.astype(np.float32)


# ---------------------------------------------------------------------------- MLP
def init_params(seed: int) -> Dict[str, np.ndarray]:
    """Weights uniform in +-1/sqrt(fan_in) from a seeded numpy generator, zero biases (float32)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, (o, i) in (("w1", (D_H, D_IN)), ("w2", (D_H, D_H)), ("w3", (D_OUT, D_H))):
        lim = 1.0 / math.sqrt(i)
        p[name] = rng.uniform(-lim, lim, size=(o, i)).astype(np.float32)
    p["b1"] = np.zeros(D_H, np.float32)
    p["b2"] = np.zeros(D_H, np.float32)
    p["b3"] = np.zeros(D_OUT, np.float32)
    return p


def forward(p: Dict[str, np.ndarray], X: np.ndarray, rounding: bool = True, tmap=None) -> Tuple[np.ndarray, dict]:
    """Y = (relu(relu(X W1^T + b1) W2^T + b2)) W3^T + b3, float64 accumulation.

    With rounding, X, the weights and the hidden activations are rounded to
    bfloat16 where the GPU stores them.  With a target map tmap = (mean0,
    mean1, scale0, scale1, tail), the raw output u is mapped back to the
    target scale, Y = u * scale + mean (the raw u is in the cache)."""
    r = bf16 if rounding else (lambda v: np.asarray(v, np.float64))
    x = np.asarray(r(X), np.float64)
    w1, w2, w3 = (np.asarray(r(p[k]), np.float64) for k in ("w1", "w2", "w3"))
    h1 = np.maximum(x @ w1.T + p["b1"], 0.0)
    h1 = np.asarray(r(h1), np.float64)
    h2 = np.maximum(h1 @ w2.T + p["b2"], 0.0)
    h2 = np.asarray(r(h2), np.float64)
    u = h2 @ w3.T + p["b3"]
    y = u if tmap is None else u * np.asarray(tmap[2:4], np.float64) + np.asarray(tmap[0:2], np.float64)
    return y, {"x": x, "h1": h1, "h2": h2, "w1": w1, "w2": w2, "w3": w3, "u": u}


def loss(y: np.ndarray, t: np.ndarray) -> float:
    """Mean over the batch of the summed squared error of the two outputs."""
    return float(((y - t) ** 2).sum() / y.shape[0])


def mapped_targets(T: np.ndarray, tmap) -> Tuple[np.ndarray, np.ndarray]:
    """(t, w): targets standardised by the map, t = (T - mean) / scale, and row
    weights w = 1 + tail * max(0, t[:, 0])."""
    T = np.asarray(T, np.float64)
    if tmap is None:
        return T, np.ones(T.shape[0])
    t = (T - np.asarray(tmap[0:2], np.float64)) / np.asarray(tmap[2:4], np.float64)
    return t, 1.0 + float(tmap[4]) * np.maximum(t[:, 0], 0.0)


def fit_target_map(T: np.ndarray, tail: float) -> np.ndarray:
    """Column means, population standard deviations (1 where below 1e-6), tail weight."""
    T = np.asarray(T, np.float64)
    m = T.mean(0)
    sd = np.sqrt(((T - m) ** 2).mean(0))
    sd = np.where(sd < 1e-6, 1.0, sd)
    return np.array([m[0], m[1], sd[0], sd[1], tail], np.float64)


def backward(p: Dict[str, np.ndarray], X: np.ndarray, T: np.ndarray, rounding: bool = True,
             tmap=None, operands: Optional[dict] = None) -> Tuple[float, dict]:
    """Gradients of the (weighted) loss by the chain rule (relu'(0) = 0), float64:
    mean_b w_b sum_j (u_bj - t_bj)^2 on the raw output u and the mapped targets
    (``mapped_targets``); without a map, the plain ``loss`` of Y against T.

    With rounding, the gradients flowing into the hidden layers are rounded to
    bfloat16 where the GPU stores them.  With a dict ``operands``, it receives the
    two factors of each weight gradient (g[w] = A^T C over the batch; a bias
    gradient is the column sum of its A): w3 <- (dy, h2), w2 <- (dh2, h1),
    w1 <- (dh1, x)."""
    r = bf16 if rounding else (lambda v: np.asarray(v, np.float64))
    _, c = forward(p, X, rounding)
    u = c["u"]
    B = u.shape[0]
    t, w = mapped_targets(T, tmap)
    dy = 2.0 * (u - t) * w[:, None] / B
    lval = float((w[:, None] * (u - t) ** 2).sum() / B)
    g = {"w3": dy.T @ c["h2"], "b3": dy.sum(0)}
    dh2 = (dy @ c["w3"]) * (c["h2"] > 0)
    dh2 = np.asarray(r(dh2), np.float64)
    g["w2"] = dh2.T @ c["h1"]
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ c["w2"]) * (c["h1"] > 0)
    dh1 = np.asarray(r(dh1), np.float64)
    g["w1"] = dh1.T @ c["x"]
    g["b1"] = dh1.sum(0)
    if operands is not None:
        operands.update({"w3": (dy, c["h2"]), "w2": (dh2, c["h1"]), "w1": (dh1, c["x"])})
    return lval, g


def adam(p: Dict[str, np.ndarray], g: Dict[str, np.ndarray], m: dict, v: dict, step: int, lr: float,
         b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam step in place (bias-corrected moments), float64 then stored float32."""
    for k in p:
        m[k] = b1 * m.get(k, 0.0) + (1 - b1) * g[k]
        v[k] = b2 * v.get(k, 0.0) + (1 - b2) * g[k] ** 2
        mh = m[k] / (1 - b1 ** step)
        vh = v[k] / (1 - b2 ** step)
        p[k] = (p[k] - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32)


# ---------------------------------------------------------------------------- ranking
def rank_order(acc: np.ndarray, f1: np.ndarray, progs: Sequence[Sequence[int]]) -> List[int]:
    """Indices sorted by accuracy desc, F1 desc, length asc, program bytes asc, index asc."""
    keys = [(-float(acc[i]), -float(f1[i]), len(progs[i]), np.asarray(progs[i], np.uint64).tobytes(), i)
            for i in range(len(progs))]
    return [k[-1] for k in sorted(keys)]


def recall_at(k: int, exact_order: Sequence[int], selected: Sequence[int]) -> float:
    """|top-k of the exact order  intersect  selected| / k."""
    top = set(exact_order[:k])
    return len(top & set(selected)) / float(k)
