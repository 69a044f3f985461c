"""Pins of the surrogate's oracle (no GPU): hand-computed encodings, bf16
rounding against a library conversion and hand cases, finite-difference
gradients, Adam's first step in closed form, ranking and recall."""
import numpy as np
import pytest

from oracle import surrogate as S
from synth import programs as P


def _want(entries):
    w = np.zeros(512, np.float32)
    for i, c in entries.items():
        w[i] = 0.25 * c
    return w


def test_encoding_hand_worked():
    # (and A1 (some r2- A3)), postfix A1 A3 EXISTS AND: AND depth 0; A1, EXISTS depth 1; A3 depth 2;
    # every node has polarity 0 (signed counts +1)
    f = S.encode(P.compile_text("(and A1 (some r2- A3))"))
    assert ((2 * 2 + 1) * 131 + 3) % 57 == 31
    assert np.array_equal(f, _want({0 * 14 + 4: 1, 1 * 14 + 0: 1, 1 * 14 + 6: 1, 2 * 14 + 0: 1,   # op x depth
                                    84 + 1: 1, 84 + 3: 1,                 # concepts 1 and 3
                                    180 + 2 * 2 + 1: 1,                   # role 2 inverted
                                    244 + 1 * 5 + 0: 1,                   # EXISTS at depth 1
                                    436 + 31: 1,                          # role 2^- over atom 3
                                    493 + 4 // 10: 1,                     # length 4
                                    504: 2, 505: 1, 508: 3 - 1, 509: 4}))  # leaves, roles, height, bias
    # (min 3 r0 (ge p9 1.0)): ATLEAST depth 0, DGE depth 1; property 9, >=, bucket 0 without a grid
    f = S.encode(P.compile_text("(min 3 r0 (ge p9 1.0))"))
    assert np.array_equal(f, _want({0 * 14 + 8: 1, 1 * 14 + 11: 1, 180 + 0: 1, 244 + 2: 1, 284 + 0 * 8 + 3: 1,
                                    308 + (9 * 2 + 0) * 4 + 0: 1, 493: 1, 504: 1, 505: 1, 506: 1, 508: 1,
                                    509: 4}))
    # with a grid, 1.0 lies above 7 of property 9's 15 boundaries (0.3 .. 1.7 step 0.1, 1.0 excluded):
    # bucket 7, feature bucket 7 // 4 = 1
    grid = np.zeros((10, 15), np.float32)
    grid[9] = np.float32(0.3) + np.float32(0.1) * np.arange(15, dtype=np.float32)
    g = S.encode(P.compile_text("(min 3 r0 (ge p9 1.0))"), grid)
    assert int(np.sum(grid[9] < np.float32(1.0))) == 7
    assert g[308 + 18 * 4 + 1] == 0.25 and g[308 + 18 * 4] == 0.0
    # polarity: (not (and A1 (max 2 r1 A50))), postfix A1 A50 ATMOST AND NOT.  NOT puts the
    # conjunction and its operands at polarity 1 (count -1); ATMOST flips again, A50 is at 0.
    assert ((1 * 2) * 131 + 50) % 57 == 27
    f = S.encode(P.compile_text("(not (and A1 (max 2 r1 A50)))"))
    assert np.array_equal(f, _want({0 * 14 + 3: 1, 1 * 14 + 4: 1, 2 * 14 + 0: 1, 2 * 14 + 9: 1, 3 * 14 + 0: 1,
                                    84 + 1: -1, 84 + 50: 1,
                                    180 + 1 * 2: 1, 244 + 2 * 5 + 3: 1, 284 + 1 * 8 + 2: 1,
                                    436 + 27: -1,                          # the restriction sits at polarity 1
                                    493 + 5 // 10: 1, 504: 2, 505: 1, 507: 1, 508: 4 - 1, 509: 4}))
    # seven nested NOTs over A0: depths 0..6 and 7, op x depth clamps depth at 5, A0 at polarity 1
    f = S.encode(P.compile_text("(not " * 7 + "A0" + ")" * 7))
    assert np.array_equal(f, _want({**{d * 14 + 3: 1 for d in range(5)}, 5 * 14 + 3: 2, 5 * 14 + 0: 1,
                                    84 + 0: -1, 493: 1, 504: 1, 507: 7, 508: 7, 509: 4}))
    # statistics: atom scores summed by depth bucket with the polarity sign, threshold scores of
    # (property, compare, bucket), the atom fillers of role restrictions
    atoms = np.array([0, 7, 0, -3], np.int64)
    thr = np.zeros((10, 2, 16), np.int64)
    thr[9, 0, 7] = 5
    st = (atoms, thr)
    f = S.encode(P.compile_text("(and A1 (some r2- A3))"), None, None, st)
    # A1 depth 1 -> bucket 0: +7; A3 depth 2 -> bucket 1: -3; role filler A3: -3
    assert f[497] == 0.25 * 7 and f[498] == 0.25 * -3 and f[503] == 0.25 * -3 and f[499] == 0
    g = S.encode(P.compile_text("(not (min 3 r0 (ge p9 1.0)))"), grid, None, st)
    # the DGE sits at depth 2 (bucket 1) under one NOT: -5
    assert g[501] == 0.25 * -5 and g[500] == 0 and g[502] == 0
    assert np.array_equal(S.encode(P.compile_text("(ge p9 1.0)"), grid, None, None)[497:504], np.zeros(7))
    assert S.stat_score(0.80095) == 10 and S.stat_score(0.5) == 0 and S.stat_score(0.0) == -16
    # a prior lands in features 510 and 511, rounded to bfloat16 and not scaled
    g = S.encode(P.compile_text("A0"), None, (0.8125, 0.3))
    assert g[510] == np.float32(0.8125) and g[511] == np.float32(0.30078125)
    assert np.array_equal(g[:510], S.encode(P.compile_text("A0"))[:510])


def test_bf16_rounding():
    torch = pytest.importorskip("torch")
    x = np.concatenate([np.random.default_rng(1).normal(size=4000).astype(np.float32) * 10.0 ** np.arange(-20, 20)
                        .repeat(100)[:4000].astype(np.float32),
                        np.array([0.0, -0.0, 1.0, 65504.0, 3.4e38, -3.4e38, 1e-40], np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(S.bf16(x), ref)
    # hand cases: 1 + 2^-8 ties to 1; 1 + 3 * 2^-8 ties to 1 + 2^-6 (even mantissa)
    assert S.bf16(np.float32(1 + 2 ** -8)) == 1.0
    assert S.bf16(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)


def test_backward_matches_finite_differences():
    p = S.init_params(3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(6, 512)).astype(np.float32)
    T = rng.uniform(size=(6, 2)).astype(np.float32)
    p64 = {k: v.astype(np.float64) for k, v in p.items()}
    _, g = S.backward(p64, X, T, rounding=False)
    eps = 1e-6
    for name in ("w1", "b1", "w2", "b2", "w3", "b3"):
        flat = p64[name].reshape(-1)
        for i in rng.choice(flat.size, size=min(8, flat.size), replace=False):
            old = flat[i]
            flat[i] = old + eps
            lp = S.loss(S.forward(p64, X, rounding=False)[0], T)
            flat[i] = old - eps
            lm = S.loss(S.forward(p64, X, rounding=False)[0], T)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            an = g[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 + 1e-5 * abs(fd), (name, i, fd, an)


def test_mapped_weighted_loss_matches_finite_differences():
    """With a target map the loss is taken on standardised targets with upper-tail row
    weights, written out here directly (not through the oracle's helpers)."""
    p = S.init_params(5)
    rng = np.random.default_rng(6)
    X = rng.normal(size=(7, 512)).astype(np.float32)
    T = rng.uniform(size=(7, 2)).astype(np.float32)
    tmap = (0.4, 0.3, 0.2, 0.25, 3.0)
    p64 = {k: v.astype(np.float64) for k, v in p.items()}

    def direct(pp):
        u = S.forward(pp, X, rounding=False)[1]["u"]
        t0 = (T[:, 0].astype(np.float64) - 0.4) / 0.2
        t1 = (T[:, 1].astype(np.float64) - 0.3) / 0.25
        w = 1.0 + 3.0 * np.maximum(t0, 0.0)
        return float(np.sum(w * ((u[:, 0] - t0) ** 2 + (u[:, 1] - t1) ** 2)) / 7)
    lval, g = S.backward(p64, X, T, rounding=False, tmap=tmap)
    assert abs(lval - direct(p64)) <= 1e-9 * abs(lval)
    eps = 1e-6
    for name in ("w1", "b2", "w3", "b3"):
        flat = p64[name].reshape(-1)
        for i in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[i]
            flat[i] = old + eps
            lp = direct(p64)
            flat[i] = old - eps
            lm = direct(p64)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[i]) <= 1e-6 + 1e-5 * abs(fd), (name, i)
    # predictions come back on the target scale
    y = S.forward(p64, X, rounding=False, tmap=tmap)[0]
    u = S.forward(p64, X, rounding=False)[0]
    assert np.allclose(y, u * np.array([0.2, 0.25]) + np.array([0.4, 0.3]))
    # the fitted map: column means and population standard deviations
    m = S.fit_target_map(T, 2.0)
    assert np.allclose(m[:2], T.mean(0)) and np.allclose(m[2:4], T.std(0)) and m[4] == 2.0


def test_adam_first_step_closed_form():
    p = {"w": np.array([1.0, -2.0, 3.0], np.float32)}
    g = {"w": np.array([0.5, -0.25, 1e-3])}
    m, v = {}, {}
    S.adam(p, g, m, v, step=1, lr=0.01)
    # bias-corrected first step moves each weight by lr * g / (|g| + eps)
    np.testing.assert_allclose(p["w"], np.array([1.0, -2.0, 3.0]) - 0.01 * np.sign(g["w"]), rtol=1e-5)


def test_ranking_and_recall():
    progs = [[1], [1, 1, 5], [2], [3]]
    acc = np.array([0.5, 0.9, 0.9, 0.1])
    f1 = np.array([0.2, 0.3, 0.3, 0.9])
    order = S.rank_order(acc, f1, progs)
    assert order == [2, 1, 0, 3]                      # tie on (acc, F1): shorter program first
    assert S.recall_at(2, order, [1, 2, 3]) == 1.0
    assert S.recall_at(2, order, [0, 3]) == 0.0


def test_statistic_programs_land_in_their_buckets():
    """The statistics table scores, for each (property, compare, q), a threshold whose grid
    bucket is q, so an encoded threshold finds its own table entry."""
    torch = pytest.importorskip("torch")
    from paper_2412_00802_gb300 import surrogate as sg
    rng = np.random.default_rng(5)
    vals = rng.lognormal(size=(3, 5000)).astype(np.float32)
    grid = sg.threshold_grid(vals)
    s = sg.Surrogate.__new__(sg.Surrogate)            # host-side helpers only, no device state
    s._grid_host = grid
    progs = s.statistic_programs(7)
    assert len(progs) == 7 + 3 * 2 * 16
    for i, p in enumerate(progs[:7]):
        assert int(p[0]) & 0xFF == P.ATOM and (int(p[0]) >> 16) & 0xFFFF == i
    for k, p in enumerate(progs[7:]):
        prop, rest = divmod(k, 32)
        o, q = divmod(rest, 16)
        w = int(p[0])
        assert w & 0xFF == (P.DGE, P.DLE)[o] and (w >> 16) & 0xFFFF == prop
        t = np.float32(P.bits_f32(w >> 32))
        assert int(np.sum(grid[prop] < t)) == q, (prop, o, q)


def _grad_case(B=4096, seed=4, tmap=None):
    from synth import hyps, kb as K
    kb = K.generate(K.CONFIGS["small"])
    X = S.encode_batch(hyps.batch_hyps(kb, seed, 0, B))
    T = np.random.default_rng(seed).uniform(size=(B, 2)).astype(np.float32)
    p = S.init_params(6)
    ops = {}
    _, ref = S.backward(p, X, T, rounding=True, tmap=tmap, operands=ops)
    return p, X, T, ref, ops


@pytest.mark.parametrize("mapped", [False, True])
def test_gradient_bound_accepts_fp32_and_rejects_planted_mistakes(mapped):
    """The element-wise gradient tolerance (tests/surrogate_bounds.py) holds a float32 emulation of
    the GPU's arithmetic at a training-size batch, and rejects perturbed copies of the oracle's own
    gradient (host arrays only): one 128 x 256 tile of dW1 summed without its last 64 batch rows,
    one tile of dW2 holding its neighbour's values, one ReLU-mask row of h1 flipped."""
    from tests import surrogate_bounds as SB
    tmap = np.array([0.5, 0.2, 0.3, 0.5, 3.0]) if mapped else None
    p, X, T, ref, ops = _grad_case(tmap=tmap)
    tol = SB.gradient_tolerances(ops)
    emu = SB.fp32_emulation(p, X, T, S.bf16, tmap=tmap)
    assert not SB.gradient_violations(emu, ref, tol)
    # a tile of dW1 missing its last K block (64 batch rows)
    dh1, x = ops["w1"]
    bad = {k: v.copy() for k, v in ref.items()}
    bad["w1"][:128, :256] -= dh1[-64:, :128].T @ x[-64:, :256]
    assert any(v.startswith("w1") for v in SB.gradient_violations(bad, ref, tol))
    # a tile of dW2 holding the values of the tile beside it
    bad = {k: v.copy() for k, v in ref.items()}
    bad["w2"][128:256, 0:256] = ref["w2"][128:256, 256:512]
    assert any(v.startswith("w2") for v in SB.gradient_violations(bad, ref, tol))
    # one batch row's ReLU mask of h1 inverted in the backward pass
    dh2, h1 = ops["w2"]
    b = 17
    pre = dh2[b] @ S.bf16(p["w2"]).astype(np.float64)
    row = S.bf16((pre * (h1[b] <= 0)).astype(np.float32)).astype(np.float64)
    bad = {k: v.copy() for k, v in ref.items()}
    bad["w1"] += np.outer(row - dh1[b], x[b])
    bad["b1"] += row - dh1[b]
    v = SB.gradient_violations(bad, ref, tol)
    assert any(s.startswith("w1") for s in v) and any(s.startswith("b1") for s in v), v


def test_adam_bound_accepts_fp32_and_rejects_wrong_steps():
    """The element-wise Adam tolerance holds a float32 step with the GPU kernel's arithmetic, against
    the oracle's float64 step (oracle.surrogate.adam, with the float32 decay rates), over two
    steps; it rejects a step without bias correction, with the moments' decay rates swapped, or
    with the first step's moments lost."""
    from tests import surrogate_bounds as SB
    f = np.float32
    B1, B2 = f(0.9), f(0.999)
    rng = np.random.default_rng(3)
    n = 20000
    w = rng.normal(0, 0.05, n).astype(np.float32)
    g1 = (rng.normal(0, 1e-2, n) * rng.choice([1e-4, 1.0], n)).astype(np.float32)
    g2 = rng.normal(0, 1e-2, n).astype(np.float32)

    def step32(w, m, v, g, t, lr, b1=B1, b2=B2, correct=True):
        m = b1 * m + (f(1) - b1) * g
        v = b2 * v + (f(1) - b2) * g * g
        c1 = f(1) - b1 ** f(t) if correct else f(1)
        c2 = f(1) - b2 ** f(t) if correct else f(1)
        return (w - f(lr) * (m / c1) / (np.sqrt(v / c2) + f(1e-8))).astype(np.float32), m, v

    def ref(w, m, v, g, t, lr):
        p, mm, vv = {"x": w.astype(np.float64)}, {"x": m.astype(np.float64)}, {"x": v.astype(np.float64)}
        S.adam(p, {"x": g.astype(np.float64)}, mm, vv, step=t, lr=lr, b1=float(B1), b2=float(B2))
        return (p["x"], mm["x"], vv["x"]) + SB.adam_tolerances(w, m, v, g, t, lr, float(B1), float(B2))

    ok = lambda got, r: all(np.all(np.abs(np.float64(a) - b) <= t) for a, b, t in zip(got, r[:3], r[3:]))
    z = np.zeros(n, np.float32)
    w1, m1, v1 = step32(w, z, z, g1, 1, 1e-3)
    assert ok((w1, m1, v1), ref(w, z, z, g1, 1, 1e-3))
    r2 = ref(w1, m1, v1, g2, 2, 1e-3)
    assert ok(step32(w1, m1, v1, g2, 2, 1e-3), r2)
    assert not ok(step32(w1, m1, v1, g2, 2, 1e-3, correct=False), r2)
    assert not ok(step32(w1, m1, v1, g2, 2, 1e-3, b1=B2, b2=B1), r2)
    assert not ok(step32(w1, z, z, g2, 2, 1e-3), r2)
