"""Seeded input generators: determinism and structural invariants (no GPU)."""
import numpy as np
import pytest

from synth import hyps as Hy
from synth import kb as K
from synth import programs as P
from synth import rng


def test_counter_rng_is_stateless():
    a = rng.u64(7, 3, np.arange(100, dtype=np.uint64))
    r = rng.Rng(7, 3)
    b = [r.next_u64() for _ in range(100)]
    assert [int(x) for x in a] == b
    assert np.array_equal(rng.u64(7, 3, np.arange(50, 100, dtype=np.uint64)), a[50:])


@pytest.fixture(scope="module")
def small():
    return K.generate(K.CONFIGS["small"])


def test_deterministic(small):
    again = K.generate(K.CONFIGS["small"])
    assert np.array_equal(again.concept_bits, small.concept_bits)
    for r in range(small.n_roles):
        assert np.array_equal(again.col[r], small.col[r])
    assert np.array_equal(again.prop_vals, small.prop_vals, equal_nan=True)


def test_csr_and_transpose(small):
    n = small.n
    for r in range(small.n_roles):
        rp, col = small.row_ptr[r].astype(np.int64), small.col[r].astype(np.int64)
        assert rp[0] == 0 and rp[-1] == col.size and np.all(np.diff(rp) >= 0)
        assert col.max() < n
        rows = np.repeat(np.arange(n), np.diff(rp))
        key = rows * n + col
        assert np.all(np.diff(key) > 0), "rows sorted, no duplicate assertion"
        ip, ic = small.inv_row_ptr[r], small.inv_col[r]
        ikey = np.repeat(np.arange(n), np.diff(ip.astype(np.int64))) * n + ic.astype(np.int64)
        assert np.all(np.diff(ikey) > 0)
        # transpose of the transpose is the original
        rp2, col2 = K.transpose_csr(ip, ic, n)
        assert np.array_equal(rp2, small.row_ptr[r]) and np.array_equal(col2, small.col[r])


def test_tails_zero_and_dag_closed(small):
    w = small.n // 32
    tail = small.n % 32
    if tail:
        assert not (small.concept_bits[:, w] >> np.uint32(tail)).any()
    assert not small.concept_bits[:, small.w:].any()
    parent = small.meta["dag_parent"]
    for j, p in enumerate(parent):
        if p >= 0:
            assert not (small.concept_bits[j] & ~small.concept_bits[p]).any(), "sub-concept members are in the parent"


def test_degree_laws():
    cfg = K.CONFIGS["batch"].scaled(200_000, n_roles=1)
    deg, _ = K.draw_degrees(cfg, 0, cfg.n)
    assert abs(deg.mean() - 6.0) < 0.05
    cfg = K.CONFIGS["large"].scaled(200_000, n_roles=1)
    deg, meta = K.draw_degrees(cfg, 0, cfg.n)
    assert abs(deg.mean() - 8.0) < 0.5 and deg.max() <= 10_000
    s = meta["zipf_shift"]
    pmf = K.shifted_zipf_pmf(2.1, s, 10_000)
    assert abs((pmf * np.arange(10_001)).sum() - 8.0) < 1e-6


def test_props_and_examples(small):
    v = small.prop_vals
    miss = np.isnan(v).mean()
    assert 0.18 < miss < 0.22
    assert np.nanmin(v) >= 0 and np.nanmax(v) <= 100
    assert small.pos_idx.size == 200 and small.neg_idx.size == 200
    assert not np.intersect1d(small.pos_idx, small.neg_idx).size


def test_hypothesis_shapes(small):
    g = Hy.TreeGen(small, 5)
    r = rng.Rng(5, 1)
    for _ in range(300):
        L, D = Hy.random_shape(r, 40, 1, 8)
        t = g._gen(r, L, D)
        assert t.size() == L and t.height() == D
        assert len(t.postfix()) == L
    batch = Hy.batch_hyps(small, 9, 0, 256)
    assert all(1 <= len(p) <= 40 for p in batch)
    for p in Hy.chain_hyps(small, 4, 8):
        assert P.from_postfix(p).height() == 6


def test_text_roundtrip():
    for s in ["(and A1 (not (some r2- (min 3 r0 (ge p1 2.5)))))", "(or TOP BOT)", "(exactly 2 r1 (le p0 -0.0))",
              "(all r3 (eq p2 1e+30))", "(and (seq s0 17) (not (contains s3 0)))", "(some r1 (seq s2 4294967295))"]:
        assert P.to_text(P.parse(s)) == s
    assert P.fields(P.compile_text("(contains s5 9)")[-1]) == (P.SCONTAINS, 0, 5, 9)
    assert P.to_text(P.parse("(some r2-- A0)")) == "(some r2 A0)"
    assert P.to_text(P.parse("(some r2--- A0)")) == "(some r2- A0)"
    prog = P.compile_text("(min 3 r7- A9)")
    assert P.fields(prog[-1]) == (P.ATLEAST, 1, 7, 3)


@pytest.mark.parametrize("cfg", [K.CONFIGS["small"].scaled(3001, seed=9),
                                 K.CONFIGS["large"].scaled(20_000, seed=8, n_roles=3, n_concepts=6),
                                 K.CONFIGS["surrogate"].scaled(5_000, n_roles=2, n_concepts=6),
                                 K.CONFIGS["small"].scaled(300, seed=3, degree=("single", 250), n_roles=1)])
def test_c_helpers_match_numpy(cfg):
    """fastgen.c reproduces the numpy recipe array for array."""
    try:
        K.USE_C = True
        a = K.generate(cfg)
        K.USE_C = False
        b = K.generate(cfg)
    finally:
        K.USE_C = True
    assert np.array_equal(a.concept_bits, b.concept_bits)
    for r in range(a.n_roles):
        assert np.array_equal(a.row_ptr[r], b.row_ptr[r])
        assert np.array_equal(a.col[r], b.col[r])
        assert np.array_equal(a.inv_row_ptr[r], b.inv_row_ptr[r])
        assert np.array_equal(a.inv_col[r], b.inv_col[r])


def test_refine_postfix_matches_the_python_generator():
    """The C refinement generator draws exactly the Python generator's candidates."""
    from synth.refine import Refiner
    for cfg in (K.CONFIGS["search"].scaled(3000, n_roles=6, n_props=4, n_concepts=20),
                K.CONFIGS["search"].scaled(2000, n_roles=0, n_props=3, n_concepts=9),
                K.CONFIGS["search"].scaled(2000, n_roles=4, n_props=0, n_concepts=7)):
        kb = K.generate(cfg)
        ref = Refiner(kb, 505)
        beam = [P.Node(P.TOP)]
        for step in range(1, 5):
            want = [np.array(n.postfix(), np.uint64) for n in ref.refine(beam, step, 700)]
            flat, offs = ref.refine_postfix([np.array(b.postfix(), np.uint64) for b in beam], step, 700)
            got = [flat[offs[i]:offs[i + 1]] for i in range(700)]
            assert all(np.array_equal(a, b) for a, b in zip(want, got)), step
            beam = [P.from_postfix(w) for w in want[::23]]      # a varied beam for the next step


def test_concrete_roles():
    """Numeric and string concrete roles: CSR over individuals with the stated shapes; the string
    table holds distinct strings (ids are interned); patterns start with the empty string and end
    with one no table string holds; the generator's leaves restrict both kinds."""
    base = K.CONFIGS["small"]
    kb = K.generate(base.scaled(4000, seed=31, n_num_roles=2, num_degree=("poisson", 3.0), n_str_roles=2,
                                str_degree=("poisson", 2.0), n_strings=300, str_len=(2, 6), alphabet=5,
                                n_patterns=10))
    for rp, vals in zip(kb.num_row_ptr, kb.num_vals):
        assert rp[0] == 0 and rp[-1] == vals.size and np.all(np.diff(rp.astype(np.int64)) >= 0)
        assert abs(vals.size / kb.n - 3.0) < 0.2 and not np.isnan(vals).any()
    assert len(set(kb.strings)) == len(kb.strings) == 300
    assert all(2 <= len(x) <= 6 and set(x) <= set(b"abcde") for x in kb.strings)
    assert kb.patterns[0] == b"" and len(kb.patterns) == 10
    assert not any(kb.patterns[-1] in x for x in kb.strings)
    assert all(any(p in x for x in kb.strings) for p in kb.patterns[1:-1])
    for rp, ids in zip(kb.str_row_ptr, kb.str_ids):
        assert rp[-1] == ids.size and int(ids.max()) < len(kb.strings)
    for nd, want in ((("single", 50), [50]), (("unique",), [1])):
        k2 = K.generate(base.scaled(300, seed=32, n_num_roles=1, num_degree=nd, n_str_roles=1, str_degree=nd,
                                    n_strings=20, n_patterns=3))
        for rp in (k2.num_row_ptr[0], k2.str_row_ptr[0]):
            deg = np.diff(rp.astype(np.int64))
            assert sorted(set(deg.tolist()) - {0}) == want
    leaves = [P.fields(int(w))[0] for p in Hy.small_hyps(kb, 3, 200) for w in p]
    assert P.SEQ in leaves and P.SCONTAINS in leaves and P.DEQ in leaves
