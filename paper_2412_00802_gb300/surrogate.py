"""Surrogate-ranked evaluation: encode candidates, predict (accuracy, F1) with
the library's BF16 MLP, keep the top fraction, score those exactly.

Only orchestration lives here (batching, the training loop, bookkeeping);
every computation runs in libhedl.so's kernels: the structural encoder, the
tensor-core MLP forward / backward / Adam, exact scores from coverage
counts, and the top-k selection.  The surrogate never reports a score: it
only decides which candidates are evaluated exactly first.
"""
from __future__ import annotations

import math
from typing import Optional, Sequence, Tuple

import numpy as np

from . import (DeviceKB, hedl_encode, hedl_mlp_create, hedl_mlp_fit_target_map, hedl_mlp_forward, hedl_mlp_get,
               hedl_mlp_get_target_map, hedl_mlp_param_count, hedl_mlp_set_target_map,
               hedl_mlp_train_step, hedl_mlp_workspace_size, hedl_plan_batch, hedl_plan_execute, hedl_stat_scores,
               hedl_plan_info_get, hedl_scores_from_counts, hedl_select_top, hedl_select_workspace_size,
               hedl_sync_status)

D_IN, D_H, D_OUT = 512, 512, 2


def init_params(seed: int) -> np.ndarray:
    """Weights uniform in +-1/sqrt(fan_in), zero biases, in the flat order of hedl_mlp_param_count."""
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in ((D_H, D_IN), (D_H, D_H), (D_OUT, D_H)):
        lim = 1.0 / math.sqrt(i)
        parts += [rng.uniform(-lim, lim, size=o * i).astype(np.float32), np.zeros(o, np.float32)]
    p = np.concatenate(parts)
    assert p.size == hedl_mlp_param_count()
    return p


def split_params(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in (("w1", (D_H, D_IN)), ("b1", (D_H,)), ("w2", (D_H, D_H)), ("b2", (D_H,)),
                        ("w3", (D_OUT, D_H)), ("b3", (D_OUT,))):
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def threshold_grid(prop_vals: np.ndarray) -> np.ndarray:
    """15 quantile boundaries (1/16 .. 15/16) of each property's present values (a KB statistic)."""
    out = np.zeros((prop_vals.shape[0], 15), np.float32)
    for p in range(prop_vals.shape[0]):
        v = prop_vals[p][~np.isnan(prop_vals[p])]
        if v.size:
            out[p] = np.quantile(v.astype(np.float64), np.arange(1, 16) / 16.0).astype(np.float32)
    return out


class Surrogate:
    def __init__(self, params: Optional[np.ndarray] = None, seed: int = 0, device: str = "cuda",
                 grid: Optional[np.ndarray] = None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.mlp = hedl_mlp_create(init_params(seed) if params is None else params)
        self.grid = None if grid is None else torch.from_numpy(np.ascontiguousarray(grid, np.float32)).to(self.device)
        self._grid_host = None if grid is None else np.ascontiguousarray(grid, np.float32)
        self.stats = None            # device int32 statistics table (see fit_statistics)
        self.n_stat_concepts = 0
        self._ws = None

    def _workspace(self, B: int):
        n = hedl_mlp_workspace_size(B)
        if self._ws is None or self._ws.numel() < n:
            self._ws = self.torch.empty(n, dtype=self.torch.uint8, device=self.device)
        return self._ws

    def params(self) -> np.ndarray:
        return hedl_mlp_get(self.mlp)[0]

    def statistic_programs(self, n_concepts: int) -> list:
        """The symbols the statistics table scores: every atom, then every (property, >= / <=,
        threshold bucket q) at the bucket's upper boundary (above the last boundary for q = 15)."""
        from synth import programs as P
        out = [np.array([P.insn(P.ATOM, 0, c)], np.uint64) for c in range(n_concepts)]
        g = self._grid_host if self._grid_host is not None else np.zeros((0, 15), np.float32)
        for p in range(g.shape[0]):
            for op in (P.DGE, P.DLE):
                for q in range(16):
                    t = g[p][q] if q < 15 else np.nextafter(g[p][14], np.float32(np.inf))
                    out.append(np.array([P.insn(op, 0, p, P.f32_bits(float(t)))], np.uint64))
        return out

    def fit_statistics(self, dkb: DeviceKB, n_concepts: int):
        """Score the statistic programs exactly with the engine and keep their table entries."""
        torch = self.torch
        progs = self.statistic_programs(n_concepts)
        flat = np.concatenate(progs)
        offs = np.arange(len(progs) + 1, dtype=np.uint32)
        _, T = exact_scores(dkb, flat, offs)
        self.stats = torch.empty(len(progs), dtype=torch.int32, device=self.device)
        hedl_stat_scores(T, self.stats)
        self.n_stat_concepts = n_concepts
        return self.stats

    def encode(self, progs: np.ndarray, offs: np.ndarray, prior: Optional[np.ndarray] = None):
        """bf16 [H][512] encodings of host programs (copied to the device first); prior: float
        [H][2] per-program inputs (features 510-511) or None."""
        torch = self.torch
        p = torch.from_numpy(np.ascontiguousarray(progs, np.uint64).view(np.int64)).to(self.device)
        o = torch.from_numpy(np.ascontiguousarray(offs, np.uint32).view(np.int32)).to(self.device)
        pr = None if prior is None else torch.from_numpy(np.ascontiguousarray(prior, np.float32)).to(self.device)
        X = torch.empty((len(offs) - 1, D_IN), dtype=torch.bfloat16, device=self.device)
        hedl_encode(p, o, X, self.grid, pr, self.stats, self.n_stat_concepts)
        return X

    def predict(self, X, batch: int = 65536):
        torch = self.torch
        Y = torch.empty((X.shape[0], D_OUT), dtype=torch.float32, device=self.device)
        for b0 in range(0, X.shape[0], batch):
            xb = X[b0:b0 + batch]
            hedl_mlp_forward(self.mlp, xb, Y[b0:b0 + xb.shape[0]], self._workspace(xb.shape[0]))
        return Y

    def train(self, X, T, epochs: int = 4, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
              tail_weight: Optional[float] = 4.0, schedule: str = "cos"):
        """Mini-batch Adam on (X, T); returns the mean loss of each epoch.

        tail_weight: fit the target map on T first (standardised targets, the
        upper tail of the accuracy weighted by 1 + tail_weight * z); None keeps
        the network's current map.  schedule: "cos" decays the learning rate
        from lr to 0 along a half cosine over all steps, "const" keeps it."""
        torch = self.torch
        n = X.shape[0]
        if tail_weight is not None:
            hedl_mlp_fit_target_map(self.mlp, T, tail_weight)
        g = torch.Generator(device="cpu").manual_seed(seed)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        hist = []
        per_epoch = max((n - batch) // batch + 1, 0)
        total, step = max(epochs * per_epoch, 1), 0
        for ep in range(epochs):
            perm = torch.randperm(n, generator=g).to(self.device)
            tot = 0.0
            steps = 0
            for b0 in range(0, n - batch + 1, batch):
                idx = perm[b0:b0 + batch]
                xb = X.index_select(0, idx).contiguous()
                tb = T.index_select(0, idx).contiguous()
                lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * step / total)) if schedule == "cos" else lr
                hedl_mlp_train_step(self.mlp, xb, tb, lr_t, self._workspace(batch), loss)
                tot += float(loss.item())
                steps += 1
                step += 1
            hist.append(tot / max(steps, 1))
        return hist

    def target_map(self) -> np.ndarray:
        return hedl_mlp_get_target_map(self.mlp)

    def set_target_map(self, tmap) -> None:
        hedl_mlp_set_target_map(self.mlp, tmap)

    def select(self, Y, k: int):
        """Indices (ascending) of the k best predictions (accuracy, then F1, then index)."""
        torch = self.torch
        idx = torch.empty(k, dtype=torch.int32, device=self.device)
        ws = torch.empty(hedl_select_workspace_size(Y.shape[0]), dtype=torch.uint8, device=self.device)
        hedl_select_top(Y, k, idx, ws)
        return idx


def exact_scores(dkb: DeviceKB, progs: np.ndarray, offs: np.ndarray, flags: int = 0):
    """(counts uint32 [H][4], scores float [H][2]) on the device, by exact evaluation."""
    torch = dkb.torch
    H = len(offs) - 1
    plan = hedl_plan_batch(dkb.handle, progs, offs, flags)
    ws = dkb.workspace(hedl_plan_info_get(plan)["workspace_bytes"])
    counts = torch.zeros((H, 4), dtype=torch.int32, device=dkb.device)
    hedl_plan_execute(dkb.handle, plan, counts, None, ws)
    scores = torch.empty((H, 2), dtype=torch.float32, device=dkb.device)
    hedl_scores_from_counts(counts, scores)
    hedl_sync_status(dkb.handle)
    return counts, scores
