"""The surrogate's kernels against its oracle (oracle/surrogate.py), and a
check that the trained network ranks better than chance."""
import numpy as np
import pytest

import oracle
from oracle import surrogate as S
from synth import hyps, kb as K, programs as P
from synth.rng import Rng
from tests import oracle_pins as pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2412_00802_gb300 import build
    build.build()
    import paper_2412_00802_gb300 as H
    from paper_2412_00802_gb300 import surrogate as sg
    kb = K.generate(K.CONFIGS["small"])
    return torch, H, sg, kb


def _programs(kb, n=600):
    r = Rng(8, 8)
    progs = [np.array(pins.random_program(r, kb, r.randint(1, 7)).postfix(), np.uint64) for _ in range(n // 2)]
    return progs + hyps.batch_hyps(kb, 9, 0, n - n // 2)


def test_encoder_bit_exact(env):
    torch, H, sg, kb = env
    progs = _programs(kb)
    long = [P.insn(P.ATOM, 0, 1)]
    for i in range(149):                       # a valid 299-instruction program (left-deep AND chain)
        long += [P.insn(P.ATOM, 0, (i * 7) % 50), P.insn(P.AND)]
    progs.append(np.array(long, np.uint64))
    flat, offs = P.pack_batch(progs)
    got = sg.Surrogate().encode(flat, offs).float().cpu().numpy()
    want = S.encode_batch(progs)
    assert np.array_equal(got, want)
    grid = S.threshold_grid(kb.prop_vals)
    got = sg.Surrogate(grid=grid).encode(flat, offs).float().cpu().numpy()
    assert np.array_equal(got, S.encode_batch(progs, grid))
    prior = np.random.default_rng(7).uniform(size=(len(progs), 2)).astype(np.float32)
    got = sg.Surrogate(grid=grid).encode(flat, offs, prior).float().cpu().numpy()
    assert np.array_equal(got, S.encode_batch(progs, grid, prior))
    # with a statistics table (values large enough for bf16 rounding of the sums)
    rng = np.random.default_rng(8)
    atoms = rng.integers(-16, 17, size=kb.n_concepts)
    thr = rng.integers(-16, 17, size=(kb.n_props, 2, 16))
    s = sg.Surrogate(grid=grid)
    s.stats = torch.from_numpy(np.concatenate([atoms, thr.reshape(-1)]).astype(np.int32)).to("cuda")
    s.n_stat_concepts = kb.n_concepts
    got = s.encode(flat, offs, prior).float().cpu().numpy()
    assert np.array_equal(got, S.encode_batch(progs, grid, prior, (atoms, thr)))
    assert np.abs(got[:, 497:504]).max() > 0
    assert np.array_equal(grid, sg.threshold_grid(kb.prop_vals))


def _xt(torch, kb, n, seed):
    progs = hyps.batch_hyps(kb, seed, 0, n)
    X = S.encode_batch(progs)
    T = np.random.default_rng(seed).uniform(size=(n, 2)).astype(np.float32)
    return X, T


def test_forward_matches_oracle(env):
    torch, H, sg, kb = env
    X, _ = _xt(torch, kb, 700, 3)
    p = sg.init_params(5)
    s = sg.Surrogate(p)
    Y = s.predict(torch.from_numpy(X).to("cuda").to(torch.bfloat16)).cpu().numpy()
    ref, _ = S.forward(sg.split_params(p), X, rounding=True)
    err = np.abs(Y - ref)
    # bf16 storage of the hidden layers: a sum in float32 may round to a neighbouring
    # bf16 value where float64 does not (one ulp, 2^-8 relative) -> small output error
    assert err.max() <= 2e-2 * max(1.0, np.abs(ref).max()), err.max()
    assert err.mean() <= 2e-3 * max(1.0, np.abs(ref).mean())


@pytest.mark.parametrize("B", [1, 700, 8192])
def test_tcgen05_forward_matches_mma_sync_and_oracle(env, B):
    """The tcgen05 dense layers (accumulators in tensor memory) give the mma.sync path's
    outputs up to FP32 summation order, and the oracle's within bf16 bounds."""
    torch, H, sg, kb = env
    X, _ = _xt(torch, kb, B, 11)
    p = sg.init_params(12)
    Xd = torch.from_numpy(X).to("cuda").to(torch.bfloat16)
    s = sg.Surrogate(p)
    y_tc = s.predict(Xd).cpu().numpy()
    H.hedl_mlp_status(s.mlp)
    H.hedl_mlp_set_gemm(s.mlp, H.HEDL_GEMM_MMA_SYNC)
    y_ms = s.predict(Xd).cpu().numpy()
    ref, _ = S.forward(sg.split_params(p), X, rounding=True)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(y_tc - y_ms).max() <= 2e-2 * scale
    assert np.abs(y_tc - ref).max() <= 2e-2 * scale
    assert np.abs(y_tc - ref).mean() <= 2e-3 * max(1.0, np.abs(ref).mean())
    with pytest.raises(H.HedlError):
        H.hedl_mlp_set_gemm(s.mlp, 7)


def _check_gradients(g, p, X, T, tmap=None):
    """Every element of every gradient within its derived bound of the oracle's (tests/surrogate_bounds.py)."""
    from tests import surrogate_bounds as SB
    from paper_2412_00802_gb300 import surrogate as sg
    ops = {}
    ref_loss, ref = S.backward(sg.split_params(p), X, T, rounding=True, tmap=tmap, operands=ops)
    bad = SB.gradient_violations(sg.split_params(g), ref, SB.gradient_tolerances(ops))
    assert not bad, bad
    return ref_loss


@pytest.mark.parametrize("engine,B", [("tcgen05", 4096), ("mma_sync", 4096), ("tcgen05", 1024),
                                      ("mma_sync", 1024), ("tcgen05", 768), ("tcgen05", 700)])
def test_gradients_match_oracle(env, engine, B):
    """Weight and bias gradients on tcgen05 (batches that are multiples of 64; 700 falls back to
    mma.sync) and on mma.sync, against the oracle's element by element: each within the bound that
    bf16 storage of the operands and FP32 accumulation allow (tests/surrogate_bounds.py)."""
    torch, H, sg, kb = env
    X, T = _xt(torch, kb, B, 4)
    p = sg.init_params(6)
    s = sg.Surrogate(p)
    H.hedl_mlp_set_gemm(s.mlp, H.HEDL_GEMM_TCGEN05 if engine == "tcgen05" else H.HEDL_GEMM_MMA_SYNC)
    Xd = torch.from_numpy(X).to("cuda").to(torch.bfloat16)
    Td = torch.from_numpy(T).to("cuda")
    loss = torch.zeros(1, device="cuda")
    H.hedl_mlp_gradients(s.mlp, Xd, Td, s._workspace(B), loss)
    H.hedl_mlp_status(s.mlp)
    _, g, _ = H.hedl_mlp_get(s.mlp)
    ref_loss = _check_gradients(g, p, X, T)
    assert abs(float(loss.item()) - ref_loss) <= 1e-3 * abs(ref_loss)


def test_target_map_fit_forward_and_gradients(env):
    """The fitted map equals the oracle's; mapped predictions and the weighted loss's
    gradients match the oracle's with the same map (gradients element by element)."""
    torch, H, sg, kb = env
    X, T = _xt(torch, kb, 4096, 9)
    T = (T * np.array([0.3, 0.5], np.float32) + np.array([0.5, 0.2], np.float32)).astype(np.float32)
    p = sg.init_params(10)
    s = sg.Surrogate(p)
    Xd = torch.from_numpy(X).to("cuda").to(torch.bfloat16)
    Td = torch.from_numpy(T).to("cuda")
    H.hedl_mlp_fit_target_map(s.mlp, Td, 3.0)
    m = s.target_map()
    ref_m = S.fit_target_map(T, 3.0)
    assert np.allclose(m, ref_m, rtol=1e-5, atol=1e-6)
    Y = s.predict(Xd).cpu().numpy()
    ref_y, _ = S.forward(sg.split_params(p), X, rounding=True, tmap=m)
    assert np.abs(Y - ref_y).max() <= 2e-2 * max(1.0, np.abs(ref_y).max())
    loss = torch.zeros(1, device="cuda")
    H.hedl_mlp_gradients(s.mlp, Xd, Td, s._workspace(4096), loss)
    _, g, _ = H.hedl_mlp_get(s.mlp)
    ref_loss = _check_gradients(g, p, X, T, tmap=m)
    assert abs(float(loss.item()) - ref_loss) <= 1e-3 * abs(ref_loss)
    with pytest.raises(H.HedlError):
        s.set_target_map([0, 0, 0.0, 1, 0])


@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
def test_train_step_matches_oracle_adam(env, engine):
    """Two Adam steps at a training-size batch: after each, the FP32 master weights and both
    moments equal the oracle's Adam step (oracle.surrogate.adam, float64, with the GPU's float32
    decay rates) from the previous state and the step's own gradient, element by element within
    the FP32 bound (tests/surrogate_bounds.py); the gradient itself is checked against the
    oracle's as in test_gradients_match_oracle."""
    from tests import surrogate_bounds as SB
    torch, H, sg, kb = env
    b1, b2 = float(np.float32(0.9)), float(np.float32(0.999))
    p = sg.init_params(8)
    s = sg.Surrogate(p)
    H.hedl_mlp_set_gemm(s.mlp, H.HEDL_GEMM_TCGEN05 if engine == "tcgen05" else H.HEDL_GEMM_MMA_SYNC)
    w = p.copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for step, seed in ((1, 7), (2, 8)):
        X, T = _xt(torch, kb, 4096, seed)
        Xd = torch.from_numpy(X).to("cuda").to(torch.bfloat16)
        Td = torch.from_numpy(T).to("cuda")
        H.hedl_mlp_train_step(s.mlp, Xd, Td, 1e-3, s._workspace(4096))
        H.hedl_mlp_status(s.mlp)
        got_w, g, n = H.hedl_mlp_get(s.mlp)
        got_m, got_v = H.hedl_mlp_get_moments(s.mlp)
        assert n == step
        _check_gradients(g, w, X, T)
        rp, rm, rv = {"x": w.astype(np.float64)}, {"x": m.astype(np.float64)}, {"x": v.astype(np.float64)}
        S.adam(rp, {"x": g.astype(np.float64)}, rm, rv, step=step, lr=1e-3, b1=b1, b2=b2)
        tw, tm, tv = SB.adam_tolerances(w, m, v, g, step, 1e-3, b1, b2)
        for name, got, want, tol in (("w", got_w, rp["x"], tw), ("m", got_m, rm["x"], tm), ("v", got_v, rv["x"], tv)):
            d = np.abs(got.astype(np.float64) - want)
            assert np.all(d <= tol), (step, name, int((d > tol).sum()), float((d - tol).max()))
        w, m, v = got_w, got_m, got_v


def test_stat_scores_exact(env):
    torch, H, sg, kb = env
    acc = np.concatenate([np.random.default_rng(3).uniform(size=997), [0.5, 0.515625, 0.484375, 0.0, 1.0]])
    sc = np.stack([acc, acc], 1).astype(np.float32)
    out = torch.empty(len(acc), dtype=torch.int32, device="cuda")
    H.hedl_stat_scores(torch.from_numpy(sc).to("cuda"), out)
    assert out.cpu().numpy().tolist() == [S.stat_score(a) for a in sc[:, 0]]


def test_scores_from_counts_exact(env):
    torch, H, sg, kb = env
    rng = np.random.default_rng(2)
    c = rng.integers(0, 1000, size=(5000, 4)).astype(np.uint32)
    c[:10] = 0
    got = torch.empty((5000, 2), device="cuda")
    H.hedl_scores_from_counts(torch.from_numpy(c.view(np.int32)).to("cuda"), got)
    acc, f1 = oracle.accuracy_f1(c)
    assert np.array_equal(got.cpu().numpy(), np.stack([acc, f1], 1).astype(np.float32))


@pytest.mark.parametrize("H_,k", [(1, 1), (100, 7), (5000, 250), (65536, 3277)])
def test_select_top_exact(env, H_, k):
    """Documented order: accuracy desc, F1 desc, index asc; NaN last; values compare by
    their float ordering with -0.0 below +0.0."""
    torch, H, sg, kb = env
    rng = np.random.default_rng(H_)
    Y = rng.integers(0, 20, size=(H_, 2)).astype(np.float32) / 20.0   # many ties
    if H_ > 10:
        Y[3, 0] = np.nan
        Y[5, 0] = -0.0
        Y[6, 0] = 0.0
    idx = sg.Surrogate().select(torch.from_numpy(Y).to("cuda"), k).cpu().numpy()

    def key(x):
        if np.isnan(x):
            return (0, 0.0)
        return (1, float(x) if not (x == 0 and np.signbit(x)) else -1e-300)
    ranked = sorted(range(H_), key=lambda i: (key(Y[i, 0]), key(Y[i, 1]), -i), reverse=True)
    assert np.array_equal(idx, np.sort(ranked[:k]))


def test_trained_surrogate_ranks_better_than_chance(env):
    """On a planted KB (the surrogate workload's shape, 20,000 individuals) the network, trained
    on exactly scored hypotheses, keeps most of the exact top 100 in its top 5 %."""
    torch, H, sg, _ = env
    kb = K.generate(K.CONFIGS["surrogate"].scaled(20000, n_pos=500, n_neg=500, n_roles=8, n_props=4, n_concepts=50))
    dkb = H.DeviceKB.from_synth(kb)
    gen = hyps.TreeGen(kb, 51, share=0.3)
    train = hyps.batch_hyps(kb, 51, 0, 24576, lmax=20, dmax=6, gen=gen)
    flat, offs = P.pack_batch(train)
    _, T = sg.exact_scores(dkb, flat, offs)
    s = sg.Surrogate(seed=1, grid=sg.threshold_grid(kb.prop_vals))
    X = s.encode(flat, offs)
    losses = s.train(X, T, epochs=20, batch=2048, lr=2e-3)
    assert losses[-1] < losses[0]
    cand = hyps.batch_hyps(kb, 52, 0, 8192, lmax=20, dmax=6, gen=gen)
    cflat, coffs = P.pack_batch(cand)
    _, Tc = sg.exact_scores(dkb, cflat, coffs)
    sel = s.select(s.predict(s.encode(cflat, coffs)), 410).cpu().numpy()   # top 5 %
    Tc = Tc.cpu().numpy()
    order = S.rank_order(Tc[:, 0], Tc[:, 1], cand)
    recall = S.recall_at(100, order, sel)
    assert recall >= 0.35, recall         # chance is 0.05
