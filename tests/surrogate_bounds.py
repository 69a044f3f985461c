"""Element-wise tolerances for the surrogate's gradients and Adam step, derived
from where the GPU's arithmetic can differ from the oracle's.

Gradients.  Each weight gradient is a sum over the batch, G = A^T C (b3 / b2 /
b1: the column sums of A).  The oracle computes it in float64 from the same
bf16-rounded operands the GPU stores (x, the weights, h1, h2, dh2, dh1); the
GPU accumulates in FP32 and in another order.  Two effects follow:

* accumulation: each FP32 partial sum carries a relative error of 2^-24, so
  |dG_ij| stays far below 2^-18 S_ij with S_ij = sum_b |A_bi| |C_bj| (the
  running error of a sum of B = 4096 terms, with a wide margin);
* rounding flips: an operand the GPU rounds to bf16 (h1, h2, dh2, dh1) is
  computed in FP32 first, so where the exact value lies within the FP32 error
  of a bf16 rounding boundary the two sides round to neighbouring bf16 values.
  One flip moves one term A_bi C_bj by at most one bf16 ulp, 2^-7 of its
  magnitude, so k flips in the terms of G_ij move it by at most
  k 2^-7 M_ij, M_ij = max_b |A_bi| |C_bj|.  A flip needs the exact value within
  about 2^-24 sqrt(512) of a boundary 2^-8 apart (probability ~3e-4 per
  element), so a column of B = 4096 operands holds about one: allowing
  k = 8 gives 2^-4 M_ij.

The tolerance is therefore |G_gpu - G_oracle| <= 2^-4 M + 2^-18 S, element by
element.  A float32 emulation of the GPU's arithmetic (same rounding points)
stays below 2^-7 M on the test batches, a quarter of the allowance; a wrong
tile, a dropped block of batch rows or one mis-masked ReLU row moves single
elements by a whole term or more, 2^-4 to several times M, and is rejected.

Adam.  Given the GPU's own gradient g, the oracle's float64 step (with the
decay rates the GPU holds, 0.9 and 0.999 rounded to float32) is compared with
the GPU's FP32 step: each moment is one multiply-add pair, within 4 * 2^-24 of
its terms' magnitudes; the weight moves by u = lr m^/(sqrt(v^) + eps), which
FP32 computes within 16 * 2^-24 |u| plus the error of its bias corrections
1 - b^t (2 ulps of b^t relative to 1 - b^t: 500 ulps of 1 - 0.999^2), and is
then stored in FP32 (half an ulp of the result, bounded by 2^-23 |w'|).
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

FLIP_ALLOWANCE = 2.0 ** -4      # 8 bf16 rounding flips of one ulp (2^-7) in a gradient's terms
ACCUM_ALLOWANCE = 2.0 ** -18    # FP32 accumulation over the batch, relative to sum |terms|


def _max_products(A: np.ndarray, C: np.ndarray, chunk: int = 8) -> np.ndarray:
    """M_ij = max_b |A_bi| |C_bj|."""
    A = np.abs(A).astype(np.float32)
    C = np.abs(C).astype(np.float32)
    M = np.zeros((A.shape[1], C.shape[1]), np.float32)
    for i0 in range(0, A.shape[1], chunk):
        M[i0:i0 + chunk] = np.max(A[:, i0:i0 + chunk].T[:, :, None] * C[None, :, :], axis=1)
    return M.astype(np.float64)


def gradient_tolerances(operands: Dict[str, Tuple[np.ndarray, np.ndarray]]) -> Dict[str, np.ndarray]:
    """Per-element tolerances of w1..w3 and b1..b3 from the oracle's gradient operands
    (oracle.surrogate.backward(..., operands=d))."""
    tol = {}
    for k in ("1", "2", "3"):
        A, C = operands["w" + k]
        A = np.asarray(A, np.float64)
        C = np.asarray(C, np.float64)
        S = np.abs(A).T @ np.abs(C)
        tol["w" + k] = FLIP_ALLOWANCE * _max_products(A, C) + ACCUM_ALLOWANCE * S
        tol["b" + k] = FLIP_ALLOWANCE * np.abs(A).max(0) + ACCUM_ALLOWANCE * np.abs(A).sum(0)
    return tol


def gradient_violations(got: Dict[str, np.ndarray], ref: Dict[str, np.ndarray],
                        tol: Dict[str, np.ndarray]) -> List[str]:
    """Elements outside their tolerance (empty list: every element within)."""
    bad = []
    for name in ("w1", "b1", "w2", "b2", "w3", "b3"):
        d = np.abs(np.asarray(got[name], np.float64) - np.asarray(ref[name], np.float64))
        over = d > tol[name]
        if over.any():
            idx = np.argwhere(over)
            worst = np.unravel_index(np.argmax(d - tol[name]), d.shape)
            bad.append(f"{name}: {int(over.sum())} elements out of bound (first {idx[0].tolist()}, worst "
                       f"{list(worst)}: |diff| {d[worst]:.3e} > {tol[name][worst]:.3e})")
    return bad


def adam_tolerances(w: np.ndarray, m: np.ndarray, v: np.ndarray, g: np.ndarray, step: int, lr: float,
                    b1: float, b2: float):
    """Per-element tolerances (tol_w, tol_m, tol_v) of the GPU's FP32 Adam step against the float64
    one from the same weights, moments and gradient, with the decay rates b1, b2 the float32 values
    the GPU holds (so 1 - b1 and 1 - b2 are exact in FP32).  Each moment is a multiply-add pair
    (4 roundings); the step u = lr m^/(sqrt(v^) + eps) adds a division, a square root and two bias
    corrections 1 - b^t whose FP32 powers carry 2 ulps of b^t, i.e. a relative error of
    2^-23 b^t / (1 - b^t) (large at the first steps, where 1 - b2^t is small); the new weight is
    stored in FP32 (half an ulp, within 2^-23 |w'|)."""
    w, m, v, g = (np.asarray(a, np.float64) for a in (w, m, v, g))
    ulp = 2.0 ** -24
    m1 = b1 * m + (1 - b1) * g
    v1 = b2 * v + (1 - b2) * g * g
    u = lr * (m1 / (1 - b1 ** step)) / (np.sqrt(v1 / (1 - b2 ** step)) + 1e-8)
    rel_u = 16 * ulp + 2 * ulp * b1 ** step / (1 - b1 ** step) + ulp * b2 ** step / (1 - b2 ** step)
    tol_m = 4 * ulp * (np.abs(b1 * m) + np.abs((1 - b1) * g)) + 1e-45
    tol_v = 4 * ulp * (np.abs(b2 * v) + (1 - b2) * g * g) + 1e-45
    tol_w = 2 * rel_u * np.abs(u) + 2.0 ** -23 * np.abs(w - u) + 1e-45
    return tol_w, tol_m, tol_v


def fp32_emulation(p: Dict[str, np.ndarray], X: np.ndarray, T: np.ndarray, bf16, tmap=None) -> Dict[str, np.ndarray]:
    """The GPU's gradient arithmetic emulated on the host, to test the bound itself: float32
    products and sums, bf16 rounding where the GPU stores bf16 (the same points as the oracle)."""
    r = bf16
    x = r(X).astype(np.float32)
    w1, w2, w3 = (r(p[k]).astype(np.float32) for k in ("w1", "w2", "w3"))
    h1 = r(np.maximum(x @ w1.T + p["b1"], 0))
    h2 = r(np.maximum(h1 @ w2.T + p["b2"], 0))
    u = h2 @ w3.T + p["b3"]
    B = X.shape[0]
    T = np.asarray(T, np.float32)
    if tmap is None:
        t, wr = T, np.ones(B, np.float32)
    else:
        t = ((T - np.asarray(tmap[0:2], np.float32)) / np.asarray(tmap[2:4], np.float32)).astype(np.float32)
        wr = (1 + np.float32(tmap[4]) * np.maximum(t[:, 0], 0)).astype(np.float32)
    dy = (2 * (u - t) * wr[:, None] / B).astype(np.float32)
    g = {"w3": dy.T @ h2, "b3": dy.sum(0)}
    dh2 = r((dy @ w3) * (h2 > 0))
    g["w2"] = dh2.T @ h1
    g["b2"] = dh2.sum(0)
    dh1 = r((dh2 @ w2) * (h1 > 0))
    g["w1"] = dh1.T @ x
    g["b1"] = dh1.sum(0)
    return g
