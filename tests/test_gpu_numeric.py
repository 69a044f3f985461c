"""Numeric concrete roles on the GPU (several values per subject, Section III-B;
existential compare, Algorithms 9-10): bit-exact parity with the oracle through
the C ABI, on every execution mode, ragged sizes, the paper's single- and
unique-subject shapes, special thresholds and the full-size workload."""
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


def numeric_kb(n, seed, nd=("poisson", 2.5), n_num=3, **kw):
    d = dict(seed=seed, n_concepts=6, n_roles=2, n_props=2, degree=("poisson", 2.0), n_pos=max(1, n // 5),
             n_neg=max(1, n // 5) if n > 1 else 0, n_num_roles=n_num, num_degree=nd)
    d.update(kw)
    cfg = K.CONFIGS["small"].scaled(n, **d)
    if cfg.n_pos + cfg.n_neg > n:
        cfg = cfg.scaled(n, n_pos=1, n_neg=0)
    return K.generate(cfg)


def restrictions(kb, q, extra=()):
    """DGE / DLE / DEQ on numeric role q at thresholds drawn from its values, its extremes and `extra`."""
    vals = np.sort(kb.num_vals[q])
    ts = list(extra)
    if vals.size:
        ts += [float(vals[0]), float(vals[vals.size // 3]), float(vals[-1]), float(np.nextafter(vals[-1], np.inf)),
               float(np.nextafter(vals[0], -np.inf))]
    p = kb.n_props + q
    return [np.array([P.insn(op, 0, p, P.f32_bits(t))], np.uint64) for t in ts for op in (P.DGE, P.DLE, P.DEQ)]


@pytest.fixture(scope="module")
def mixed():
    kb = numeric_kb(5000, 201)
    return kb, device_kb(kb)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_mixed_programs_every_mode(mixed, mode):
    """Random programs over every constructor, numeric-role restrictions inside role fillers,
    boolean combinations and next to one-value properties."""
    kb, dkb = mixed
    r = Rng(202, 1)
    progs = [np.array(pins.random_program(r, kb, r.randint(1, 6)).postfix(), np.uint64) for _ in range(300)]
    progs += hyps.small_hyps(kb, 203, 200)
    for q in range(kb.n_num_roles):
        progs += restrictions(kb, q, (0.0, -0.0, 50.0))
    assert sum(any(P.fields(int(w))[0] in P.DATA_OPS and P.fields(int(w))[2] >= kb.n_props for w in p)
               for p in progs) > 120
    compare_batch(kb, dkb, progs, MODES[mode])


def test_eval_concept(mixed):
    kb, dkb = mixed
    okb = oracle.from_synth(kb)
    r = Rng(204, 2)
    for _ in range(30):
        prog = pins.random_program(r, kb, r.randint(1, 5)).postfix()
        want = oracle.eval_program(okb, prog)
        got = K.unpack_bits(dkb.eval(np.array(prog, np.uint64)), kb.n)
        assert np.array_equal(got, want), P.to_text(P.from_postfix(prog))


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 63, 65, 127, 129, 1000, 4097])
def test_ragged_sizes(n):
    kb = numeric_kb(n, 300 + n, nd=("poisson", 3.0))
    dkb = device_kb(kb)
    r = Rng(n, 5)
    progs = [np.array(pins.random_program(r, kb, r.randint(1, 4)).postfix(), np.uint64) for _ in range(60)]
    for q in range(kb.n_num_roles):
        progs += restrictions(kb, q)
    for mode in (0, H.HEDL_PLAIN, H.HEDL_SLICE_ALL):
        compare_batch(kb, dkb, progs, mode)


@pytest.mark.parametrize("nd", [("single", 20_000), ("unique",), ("poisson", 0.3), ("poisson", 40.0)])
def test_stress_shapes(nd):
    """One subject holding 20,000 values (a run that spans many warp steps), one value per
    subject, mostly empty rows, and 40 values per subject."""
    kb = numeric_kb(9000, 400, nd=nd, n_num=2)
    dkb = device_kb(kb)
    progs = []
    for q in range(kb.n_num_roles):
        progs += restrictions(kb, q, (500.0,))
    r = Rng(401, 1)
    progs += [np.array(pins.random_program(r, kb, r.randint(2, 4)).postfix(), np.uint64) for _ in range(40)]
    for mode in (0, H.HEDL_PLAIN, H.HEDL_LEVELS):
        compare_batch(kb, dkb, progs, mode)


@pytest.mark.parametrize("nd", [("poisson", 3.0), ("single", 20_000)])
def test_value_arrays_not_16_byte_aligned(nd):
    """The value walk reads 16-byte vectors and hints row pointers into L2 only from 16-byte
    aligned arrays; row pointers and values that start 4 bytes past a boundary take the scalar
    loads and must give the same sets (a ragged size, and a run spanning many windows)."""
    import torch
    kb = numeric_kb(4099, 410, nd=nd, n_num=2)
    dkb = device_kb(kb)

    def shifted(x):
        big = torch.zeros(x.numel() + 1, dtype=x.dtype, device=x.device)
        big[1:] = x
        return big[1:]
    dkb.num_roles = [(shifted(rp), shifted(v)) for rp, v in dkb.num_roles]
    assert all(rp.data_ptr() % 16 and v.data_ptr() % 16 for rp, v in dkb.num_roles)
    with torch.cuda.device(dkb.device):
        dkb.handle = H.hedl_kb_load(kb.n, dkb.concepts, dkb.roles, dkb.inv_roles, dkb.props,
                                    num_roles=dkb.num_roles)
        dkb.set_examples(kb.pos_bits, kb.neg_bits)
    progs = []
    for q in range(kb.n_num_roles):
        progs += restrictions(kb, q, (500.0,))
    r = Rng(411, 1)
    progs += [np.array(pins.random_program(r, kb, r.randint(1, 4)).postfix(), np.uint64) for _ in range(60)]
    for mode in (0, H.HEDL_PLAIN):
        compare_batch(kb, dkb, progs, mode)


def test_hand_worked_nan_and_signed_zero():
    """Individual 0 holds {1.5, NaN}, 2 holds {-0.0}, 3 holds {NaN}, 4 holds {7, 2, 9},
    5 holds {+0.0}; 1 has no value.  Expected sets worked out by hand."""
    nan = float("nan")
    assertions = [(4, 7.0), (0, 1.5), (2, -0.0), (4, 2.0), (3, nan), (0, nan), (4, 9.0), (5, 0.0)]
    kb = K.from_arrays(6, [[0, 1, 4]], [], [[nan] * 6], [0, 4], [2, 5], num_roles=[assertions, []])
    dkb = device_kb(kb)
    cases = [("(ge p1 2.0)", {4}), ("(le p1 1.5)", {0, 2, 5}), ("(eq p1 0.0)", {2, 5}), ("(eq p1 -0.0)", {2, 5}),
             ("(eq p1 2.0)", {4}), ("(eq p1 nan)", set()), ("(ge p1 nan)", set()), ("(ge p1 -inf)", {0, 2, 4, 5}),
             ("(le p1 inf)", {0, 2, 4, 5}), ("(ge p1 9.5)", set()), ("(le p1 -1.0)", set()),
             ("(not (ge p1 -inf))", {1, 3}), ("(and A0 (ge p1 1.5))", {0, 4}), ("(ge p2 0.0)", set()),
             ("(le p0 1.0)", set())]
    progs = [P.compile_text(t) for t, _ in cases]
    for mode in MODES.values():
        counts, bits = dkb.score(*P.pack_batch(progs), mode, out_bits=True)
        for h, (t, want) in enumerate(cases):
            got = set(np.nonzero(K.unpack_bits(bits[h], 6))[0].tolist())
            assert got == want, (mode, t, sorted(got))
            tp, fp = len(want & {0, 4}), len(want & {2, 5})
            assert tuple(int(x) for x in counts[h]) == (tp, fp, 2 - tp, 2 - fp), (mode, t)


def test_bad_numeric_role_rejected():
    kb = numeric_kb(500, 500, n_num=1)
    rp, vals = kb.num_row_ptr[0].copy(), kb.num_vals[0]
    k = 1 + int(np.nonzero(np.diff(rp[1:].astype(np.int64)) >= 1)[0][0])   # rp[k] < rp[k + 1], k >= 1
    down = rp.copy()
    down[k], down[k + 1] = rp[k + 1], rp[k]
    short = rp.copy()
    short[-1] -= 1
    start = rp.copy()
    start[0] = 1
    for what, bad in (("decreasing", down), ("end != n_vals", short), ("start != 0", start)):
        with pytest.raises(H.HedlError) as e:
            H.DeviceKB(kb.n, kb.concept_bits, kb.row_ptr, kb.col, kb.inv_row_ptr, kb.inv_col, kb.prop_vals,
                       num_row_ptr=[bad], num_vals=[vals])
        assert e.value.code == -6, what


@pytest.fixture(scope="module")
def numeric_full():
    return K.generate(K.CONFIGS["numeric"])


def test_full_size_numeric_workload(numeric_full):
    """10^7 individuals, 8 numeric roles of 4 * 10^7 values each, in the benchmark's launch
    configuration: every restriction's counts against the oracle, instance sets of a sample."""
    kb = numeric_full
    dkb = device_kb(kb)
    progs = []
    for q in range(kb.n_num_roles):
        vals = kb.num_vals[q]
        t = float(vals[(q * 7919) % vals.size])
        for op in (P.DGE, P.DLE, P.DEQ):
            progs.append(np.array([P.insn(op, 0, q, P.f32_bits(t))], np.uint64))
    progs += [P.compile_text("(and (ge p0 900.0) (le p1 100.0))"), P.compile_text("(or A1 (not (eq p7 nan)))"),
              P.compile_text("(and A2 (ge p3 999.99))")]
    counts, _ = compare_batch(kb, dkb, progs, 0, check_bits=False)
    okb = oracle.from_synth(kb)
    for h in (0, 4, 23, len(progs) - 1):
        got = K.unpack_bits(dkb.eval(progs[h]), kb.n)
        assert np.array_equal(got, oracle.eval_program(okb, progs[h])), h
    assert np.array_equal(dkb.score(*P.pack_batch(progs), H.HEDL_PLAIN), counts)
