"""String concrete roles on the GPU (Section III-B; EQUAL, Algorithms 11-12, and
CONTAIN, Algorithms 13-14): bit-exact parity with the oracle through the C ABI.
The oracle compares each assertion's bytes; the library compares interned ids
and reads a containment bitmap it computed at load."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import paper_2412_00802_gb300 as H
from synth import hyps, kb as K, programs as P
from synth.rng import Rng
from tests import oracle_pins as pins
from tests.gpu_util import compare_batch, device_kb

pytestmark = pytest.mark.gpu

MODES = {"default": 0, "no_cse": H.HEDL_NO_CSE, "no_graph": H.HEDL_NO_GRAPH, "levels": H.HEDL_LEVELS,
         "plain": H.HEDL_PLAIN, "no_slice": H.HEDL_NO_SLICE, "slice_all": H.HEDL_SLICE_ALL}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_00802_gb300 import build
    build.build()
    oracle.build()


def string_kb(n, seed, sd=("poisson", 2.0), **kw):
    d = dict(seed=seed, n_concepts=6, n_roles=2, n_props=1, degree=("poisson", 2.0), n_pos=max(1, n // 5),
             n_neg=max(1, n // 5) if n > 1 else 0, n_str_roles=3, str_degree=sd, n_strings=300,
             str_len=(0, 9), alphabet=4, n_patterns=24, n_num_roles=1)
    d.update(kw)
    cfg = K.CONFIGS["small"].scaled(n, **d)
    if cfg.n_pos + cfg.n_neg > n:
        cfg = cfg.scaled(n, n_pos=1, n_neg=0)
    return K.generate(cfg)


def string_restrictions(kb, q):
    """SEQ on a few table strings (and one id past the table), SCONTAINS on every pattern."""
    ids = [0, 1, len(kb.strings) // 2, len(kb.strings) - 1, len(kb.strings), 0xFFFFFFFF]
    if kb.str_ids[q].size:
        ids.append(int(kb.str_ids[q][kb.str_ids[q].size // 2]))
    out = [np.array([P.insn(P.SEQ, 0, q, b)], np.uint64) for b in ids]
    out += [np.array([P.insn(P.SCONTAINS, 0, q, k)], np.uint64) for k in range(kb.n_patterns)]
    return out


@pytest.fixture(scope="module")
def mixed():
    kb = string_kb(5000, 601)
    return kb, device_kb(kb)


def test_hand_worked_equal_and_contain():
    """Role 0 asserts 0:{catalog, dog} 1:{cat} 2:{""} 3:{at, dog} 5:{catalog}; role 1 asserts 4:{dog}.
    Expected sets worked out by hand."""
    strings = [b"cat", b"catalog", b"dog", b"", b"at"]
    patterns = [b"", b"cat", b"og", b"atalogue", b"t", b"a"]
    r0 = [(5, 1), (0, 2), (1, 0), (2, 3), (3, 4), (0, 1), (3, 2)]
    kb = K.from_arrays(6, [[0, 1, 4]], [], [], [0, 4], [2, 5], str_roles=[r0, [(4, 2)]], strings=strings,
                       patterns=patterns)
    dkb = device_kb(kb)
    cases = [("(seq s0 0)", {1}), ("(seq s0 1)", {0, 5}), ("(seq s0 2)", {0, 3}), ("(seq s0 3)", {2}),
             ("(seq s0 4)", {3}), ("(seq s0 5)", set()), ("(seq s0 4294967295)", set()), ("(seq s1 2)", {4}),
             ("(contains s0 0)", {0, 1, 2, 3, 5}), ("(contains s0 1)", {0, 1, 5}), ("(contains s0 2)", {0, 3, 5}),
             ("(contains s0 3)", set()), ("(contains s0 4)", {0, 1, 3, 5}), ("(contains s0 5)", {0, 1, 3, 5}),
             ("(contains s1 2)", {4}), ("(and A0 (contains s0 2))", {0}), ("(not (contains s0 0))", {4})]
    progs = [P.compile_text(t) for t, _ in cases]
    for mode in MODES.values():
        counts, bits = dkb.score(*P.pack_batch(progs), mode, out_bits=True)
        for h, (t, want) in enumerate(cases):
            got = set(np.nonzero(K.unpack_bits(bits[h], 6))[0].tolist())
            assert got == want, (mode, t, sorted(got))
            tp, fp = len(want & {0, 4}), len(want & {2, 5})
            assert tuple(int(x) for x in counts[h]) == (tp, fp, 2 - tp, 2 - fp), (mode, t)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_mixed_programs_every_mode(mixed, mode):
    kb, dkb = mixed
    r = Rng(602, 1)
    progs = [np.array(pins.random_program(r, kb, r.randint(1, 6)).postfix(), np.uint64) for _ in range(300)]
    progs += hyps.small_hyps(kb, 603, 200)
    for q in range(kb.n_str_roles):
        progs += string_restrictions(kb, q)
    assert sum(any(P.fields(int(w))[0] in P.STRING_OPS for w in p) for p in progs) > 150
    compare_batch(kb, dkb, progs, MODES[mode])


def test_eval_concept(mixed):
    kb, dkb = mixed
    okb = oracle.from_synth(kb)
    r = Rng(604, 2)
    for _ in range(30):
        prog = pins.random_program(r, kb, r.randint(1, 5)).postfix()
        want = oracle.eval_program(okb, prog)
        got = K.unpack_bits(dkb.eval(np.array(prog, np.uint64)), kb.n)
        assert np.array_equal(got, want), P.to_text(P.from_postfix(prog))


@pytest.mark.parametrize("n", [1, 2, 31, 33, 65, 129, 1000, 4097])
def test_ragged_sizes(n):
    kb = string_kb(n, 700 + n, sd=("poisson", 3.0))
    dkb = device_kb(kb)
    r = Rng(n, 7)
    progs = [np.array(pins.random_program(r, kb, r.randint(1, 4)).postfix(), np.uint64) for _ in range(60)]
    for q in range(kb.n_str_roles):
        progs += string_restrictions(kb, q)
    for mode in (0, H.HEDL_PLAIN, H.HEDL_SLICE_ALL):
        compare_batch(kb, dkb, progs, mode)


@pytest.mark.parametrize("sd", [("single", 20_000), ("unique",), ("poisson", 0.2), ("poisson", 30.0)])
def test_stress_shapes(sd):
    kb = string_kb(9000, 800, sd=sd)
    dkb = device_kb(kb)
    progs = []
    for q in range(kb.n_str_roles):
        progs += string_restrictions(kb, q)
    for mode in (0, H.HEDL_PLAIN, H.HEDL_LEVELS):
        compare_batch(kb, dkb, progs, mode)


def test_bad_string_data_rejected():
    kb = string_kb(500, 900, n_str_roles=1)
    rp, ids = kb.str_row_ptr[0], kb.str_ids[0]
    k = 1 + int(np.nonzero(np.diff(rp[1:].astype(np.int64)) >= 1)[0][0])
    down = rp.copy()
    down[k], down[k + 1] = rp[k + 1], rp[k]
    big = ids.copy()
    big[0] = len(kb.strings)
    dev = lambda **kw: H.DeviceKB(kb.n, kb.concept_bits, kb.row_ptr, kb.col, kb.inv_row_ptr, kb.inv_col,
                                  kb.prop_vals, **kw)
    for what, kw in (("row_ptr decreases", dict(str_row_ptr=[down], str_ids=[ids])),
                     ("id past the table", dict(str_row_ptr=[rp], str_ids=[big]))):
        with pytest.raises(H.HedlError) as e:
            dev(strings=kb.strings, patterns=kb.patterns, **kw)
        assert e.value.code == -6, what
    dev(str_row_ptr=[rp], str_ids=[ids], strings=kb.strings, patterns=kb.patterns)   # the valid one loads


@pytest.fixture(scope="module")
def strings_full():
    return K.generate(K.CONFIGS["strings"])


def test_full_size_string_workload(strings_full):
    """10^7 individuals, 8 string roles of 2 * 10^7 ids each into 100,000 strings, 64 patterns, in the
    benchmark's launch configuration: counts of restrictions on roles 0 and 1 against the oracle
    (which holds those two roles' assertions as bytes), instance sets of a sample."""
    kb = strings_full
    dkb = device_kb(kb)
    progs = []
    for q in (0, 1):
        ids = kb.str_ids[q]
        progs += [np.array([P.insn(P.SEQ, 0, q, int(ids[(q * 7919) % ids.size]))], np.uint64),
                  np.array([P.insn(P.SEQ, 0, q, len(kb.strings))], np.uint64)]
        progs += [np.array([P.insn(P.SCONTAINS, 0, q, k)], np.uint64) for k in (0, 1, 5, 17, 63)]
    progs += [P.compile_text("(and (contains s0 3) (not (seq s1 42)))"), P.compile_text("(or A1 (contains s1 9))")]
    small = replace(kb, str_row_ptr=kb.str_row_ptr[:2], str_ids=kb.str_ids[:2])
    counts, _ = compare_batch(small, dkb, progs, 0, check_bits=False)
    okb = oracle.from_synth(small)
    for h in (0, 3, len(progs) - 1):
        got = K.unpack_bits(dkb.eval(progs[h]), kb.n)
        assert np.array_equal(got, oracle.eval_program(okb, progs[h])), h
    assert np.array_equal(dkb.score(*P.pack_batch(progs), H.HEDL_PLAIN), counts)
