"""Parity of the CUDA path with the oracle (bit-exact), through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_2412_00802_gb300 as H
from synth import hyps, kb as K, programs as P
from synth.rng import Rng
from tests import golden_io
from tests import oracle_pins as pins
from tests.gpu_util import compare_batch, device_kb

pytestmark = pytest.mark.gpu

MODES = {"default": 0, "no_cse": H.HEDL_NO_CSE, "no_graph": H.HEDL_NO_GRAPH, "levels": H.HEDL_LEVELS,
         "plain": H.HEDL_PLAIN, "no_slice": H.HEDL_NO_SLICE, "no_slice_levels": H.HEDL_NO_SLICE | H.HEDL_LEVELS,
         "slice_all": H.HEDL_SLICE_ALL, "slice_all_levels": H.HEDL_SLICE_ALL | H.HEDL_LEVELS}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_00802_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("name", golden_io.fixtures())
def test_hand_worked_fixtures(name):
    """The GPU reproduces the hand-derived instance sets and counts."""
    fx = golden_io.load(name)
    kb = K.from_arrays(fx.n, fx.concept_list(), fx.role_list(), fx.prop_rows(), sorted(fx.pos), sorted(fx.neg))
    dkb = device_kb(kb)
    progs = [P.compile_text(q) for q, _, _ in fx.queries]
    for mode in MODES.values():
        counts, bits = dkb.score(*P.pack_batch(progs), mode, out_bits=True)
        for h, (q, inst, cnt) in enumerate(fx.queries):
            got = set(np.nonzero(K.unpack_bits(bits[h], fx.n))[0].tolist())
            assert got == inst, (mode, q, sorted(got))
            assert tuple(int(x) for x in counts[h]) == cnt, (mode, q, counts[h])


@pytest.fixture(scope="module")
def small():
    return K.generate(K.CONFIGS["small"])


@pytest.fixture(scope="module")
def small_dev(small):
    return device_kb(small)


@pytest.fixture(scope="module")
def small_progs(small):
    return hyps.small_hyps(small, 11, 1000)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_small_kb_all_hypotheses(small, small_dev, small_progs, mode):
    """Workload 1: 1,000 hypotheses of depth <= 4, every instance set and count."""
    compare_batch(small, small_dev, small_progs, MODES[mode])


@pytest.mark.parametrize("flags", [0, H.HEDL_SLICE_ALL, H.HEDL_NO_SLICE])
def test_repeated_execution_through_the_graph(small, small_dev, small_progs, flags):
    """First execution launches directly, the second captures a CUDA graph, the third and
    a replay run the graph: every one matches the oracle."""
    import torch
    flat, offs = P.pack_batch(small_progs)
    okb = oracle.from_synth(small)
    oc, osets, errs = oracle.eval_batch(okb, flat, offs, threads=4, keep_sets=True)
    plan = H.hedl_plan_batch(small_dev.handle, flat, offs, flags)
    ws = small_dev.workspace(H.hedl_plan_info_get(plan)["workspace_bytes"])
    for call in (H.hedl_plan_execute, H.hedl_plan_execute, H.hedl_plan_execute, H.hedl_plan_replay):
        counts = torch.zeros((len(small_progs), 4), dtype=torch.int32, device=small_dev.device)
        bits = torch.zeros((len(small_progs), small_dev.wp), dtype=torch.int32, device=small_dev.device)
        call(small_dev.handle, plan, counts, bits, ws)
        H.hedl_sync_status(small_dev.handle)
        assert np.array_equal(counts.cpu().numpy().astype(np.int64), oc)
        bb = bits.cpu().numpy().view(np.uint32)
        for h in range(len(small_progs)):
            assert np.array_equal(K.unpack_bits(bb[h], small.n), osets[h].astype(bool)), (call, h)


def test_small_kb_batched_shapes(small, small_dev):
    """Uneven lengths 1..40, depths 1..8, shared sub-concepts."""
    progs = hyps.batch_hyps(small, 21, 0, 512)
    compare_batch(small, small_dev, progs, 0)
    compare_batch(small, small_dev, progs, H.HEDL_LEVELS)


@pytest.mark.parametrize("tuning", [dict(warps_per_cta=4, words_per_lane=4, rounds=2),
                                    dict(warps_per_cta=16, words_per_lane=1, rounds=3),
                                    dict(warps_per_cta=8, words_per_lane=4, rounds=1, ctas_per_sm=1),
                                    dict(warps_per_cta=32, words_per_lane=1, stage_fillers=1),
                                    dict(warps_per_cta=8, words_per_lane=1, stage_fillers=0),
                                    dict(warps_per_cta=16, words_per_lane=4, rounds=2, stage_fillers=0),
                                    dict(warps_per_cta=16, role_block=4, rounds=2, stage_fillers=1),
                                    dict(warps_per_cta=8, role_block=4, stage_fillers=0),
                                    dict(warps_per_cta=8, role_block=8, stage_fillers=0, full_occupancy=1, rounds=4),
                                    dict(warps_per_cta=1, role_block=8, rounds=1),
                                    dict(warps_per_cta=2, role_block=4, rounds=4, stage_fillers=1)])
def test_launch_shapes(small, tuning):
    dkb = device_kb(small)
    H.hedl_tuning_set(dkb.handle, **tuning)
    compare_batch(small, dkb, hyps.batch_hyps(small, 22, 0, 300), 0)


def test_autotune_picks_a_shape_and_stays_exact(small, tmp_path):
    dkb = device_kb(small)
    probe = P.pack_batch(hyps.batch_hyps(small, 41, 0, 128))
    cache = str(tmp_path / "tune.txt")
    chosen = dkb.autotune(*probe, cache_path=cache)
    assert H.hedl_tuning_get(dkb.handle) == chosen
    assert open(cache).read().count("\n") == 1
    compare_batch(small, dkb, hyps.batch_hyps(small, 42, 0, 200), 0)
    other = device_kb(small)                      # the cached result is reused
    assert other.autotune(*probe, cache_path=cache) == chosen
    assert open(cache).read().count("\n") == 1


def test_launch_shape_that_does_not_fit_is_rejected(small):
    dkb = device_kb(small)
    with pytest.raises(H.HedlError) as e:
        H.hedl_tuning_set(dkb.handle, warps_per_cta=32, words_per_lane=4)
    assert e.value.code == -1
    with pytest.raises(H.HedlError):
        H.hedl_tuning_set(dkb.handle, warps_per_cta=12)


def test_eval_concept(small, small_dev):
    okb = oracle.from_synth(small)
    r = Rng(9, 9)
    for i in range(40):
        prog = pins.random_program(r, small, r.randint(1, 6)).postfix()
        want = oracle.eval_program(okb, prog)
        for flags in (0, H.HEDL_SLICE_ALL):
            got = K.unpack_bits(small_dev.eval(np.array(prog, np.uint64), flags), small.n)
            assert np.array_equal(got, want), (flags, P.to_text(P.from_postfix(prog)))


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 63, 64, 65, 100, 127, 129, 1000, 4097])
def test_ragged_sizes_every_constructor(n):
    """Sizes around word and 128-bit boundaries, every constructor incl. TOP/BOT/EXACTLY/DEQ."""
    cfg = K.CONFIGS["small"].scaled(n, seed=1000 + n, n_concepts=6, n_roles=3, n_props=2,
                                 degree=("poisson", min(3.0, max(n - 1, 0) / 2 + 0.5)),
                                 n_pos=max(1, n // 4), n_neg=max(1, n // 4) if n > 1 else 0)
    cfg = cfg if cfg.n_pos + cfg.n_neg <= n else cfg.scaled(n, n_pos=1, n_neg=0)
    kb = K.generate(cfg)
    dkb = device_kb(kb)
    r = Rng(n, 3)
    progs = [np.array(pins.random_program(r, kb, r.randint(1, 5)).postfix(), np.uint64) for _ in range(120)]
    for mode in (0, H.HEDL_PLAIN, H.HEDL_NO_SLICE, H.HEDL_SLICE_ALL):
        compare_batch(kb, dkb, progs, mode)


def test_stress_shapes_single_and_unique_subject():
    """The paper's two assertion-set shapes: one subject holding every assertion (a 6,000-edge row)
    and one assertion per subject (a permutation)."""
    base = K.CONFIGS["small"]
    for deg in (("single", 6000), ("unique",)):
        kb = K.generate(base.scaled(9000, seed=77, n_concepts=5, n_roles=2, degree=deg))
        dkb = device_kb(kb)
        r = Rng(5, 1)
        progs = [np.array(pins.random_program(r, kb, r.randint(2, 4)).postfix(), np.uint64) for _ in range(80)]
        progs += [P.compile_text(t) for t in ("(min 3000 r0 A1)", "(max 2999 r0 TOP)", "(exactly 6000 r0 TOP)",
                                                "(all r0 A2)", "(some r0- A0)", "(min 1 r1- (not A3))")]
        for mode in (0, H.HEDL_LEVELS, H.HEDL_PLAIN, H.HEDL_NO_SLICE, H.HEDL_SLICE_ALL):
            compare_batch(kb, dkb, progs, mode)


def test_zipf_heavy_rows():
    kb = K.generate(K.CONFIGS["large"].scaled(40_000, seed=55, n_concepts=12, n_roles=3, n_props=3))
    dkb = device_kb(kb)
    progs = hyps.batch_hyps(kb, 5, 0, 300, lmax=30, dmax=7)
    compare_batch(kb, dkb, progs, 0)
    compare_batch(kb, dkb, progs, H.HEDL_NO_SLICE)
    compare_batch(kb, dkb, progs, H.HEDL_SLICE_ALL)


def test_special_thresholds_and_counts(small, small_dev):
    texts = ["(ge p0 -0.0)", "(le p0 0.0)", "(eq p0 -0.0)", "(ge p1 inf)", "(le p1 -inf)", "(ge p2 nan)",
             "(not (le p3 nan))", "(min 0 r1 BOT)", "(max 4294967295 r2 TOP)", "(exactly 4294967295 r2 TOP)",
             "(min 4294967295 r2 TOP)", "(exactly 0 r3- A5)", "TOP", "BOT", "(not TOP)", "A0"]
    progs = [P.compile_text(t) for t in texts]
    deep = np.array([P.insn(P.ATOM, 0, i % 50) for i in range(64)] + [P.insn(P.AND)] * 32 + [P.insn(P.OR)] * 31,
                    np.uint64)
    progs.append(deep)
    for mode in MODES.values():
        compare_batch(small, small_dev, progs, mode)


def test_role_groups_with_every_kind_and_many_slices(small, small_dev):
    """More than 32 restrictions of one role in one level, every kind, n = 0..6 sliced and
    n = 7.. on the per-restriction walk, complemented fillers, heavy rows."""
    texts = []
    for k, kind in enumerate(("some", "all", "min", "max", "exactly")):
        for n in range(0, 9):
            for inv in ("", "-"):
                c = f"A{(k * 9 + n) % 50}"
                texts.append(f"({kind} r1{inv} {c})" if kind in ("some", "all") else f"({kind} {n} r1{inv} {c})")
    texts += [f"(and A{i} (some r2 (or A{i + 1} (min {i % 5} r2- A{i + 2}))))" for i in range(40)]
    progs = [P.compile_text(t) for t in texts]
    for mode in (0, H.HEDL_LEVELS, H.HEDL_NO_SLICE, H.HEDL_SLICE_ALL):
        compare_batch(small, small_dev, progs, mode)


def test_kb_without_roles_or_props():
    kb = K.generate(K.CONFIGS["small"].scaled(3000, seed=3, n_roles=0, n_props=0))
    dkb = device_kb(kb)
    progs = [P.compile_text(t) for t in ("(and A1 (not A2))", "(or A3 TOP)", "BOT")]
    compare_batch(kb, dkb, progs, 0)


def test_examples_counts(small, small_dev):
    assert H.hedl_examples_counts(small_dev.handle) == (small.pos_idx.size, small.neg_idx.size)


def test_replay_and_workspace_checks(small, small_dev):
    import torch
    progs = hyps.batch_hyps(small, 31, 0, 200)
    flat, offs = P.pack_batch(progs)
    plan = H.hedl_plan_batch(small_dev.handle, flat, offs)
    info = H.hedl_plan_info_get(plan)
    ws = torch.empty(info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    counts = torch.zeros((200, 4), dtype=torch.int32, device="cuda")
    H.hedl_plan_execute(small_dev.handle, plan, counts, None, ws)
    first = counts.clone()
    for _ in range(3):
        counts.zero_()
        H.hedl_plan_replay(small_dev.handle, plan, counts, None, ws)
        H.hedl_sync_status(small_dev.handle)
        assert torch.equal(counts, first)
    small = torch.empty(info["workspace_bytes"] - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(H.HedlError) as e:
        H.hedl_plan_execute(small_dev.handle, plan, counts, None, small)
    assert e.value.code == -3
    big = torch.empty(info["workspace_bytes"] + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(H.HedlError) as e:   # large enough, but not 256-byte aligned
        H.hedl_plan_execute(small_dev.handle, plan, counts, None, big[1:])
    assert e.value.code == -1


def test_score_batch_one_shot(small, small_dev):
    import torch
    progs = hyps.batch_hyps(small, 32, 0, 100)
    flat, offs = P.pack_batch(progs)
    n = H.hedl_workspace_size(small_dev.handle, flat, offs)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    counts = torch.zeros((100, 4), dtype=torch.int32, device="cuda")
    H.hedl_score_batch(small_dev.handle, flat, offs, counts, ws)
    H.hedl_sync_status(small_dev.handle)
    okb = oracle.from_synth(small)
    oc, _, _ = oracle.eval_batch(okb, flat, offs, threads=4)
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), oc)


def test_bounded_wait_reports_timeout(small):
    """A dependency nothing satisfies: the device wait gives up, the call reports
    HEDL_ERR_TIMEOUT, and the context stays usable."""
    dkb = device_kb(small)
    H.hedl_tuning_set(dkb.handle, wait_timeout_ms=100)
    progs = hyps.batch_hyps(small, 33, 0, 50)
    flat, offs = P.pack_batch(progs)
    with pytest.raises(H.HedlError) as e:
        dkb.score(flat, offs, H.HEDL_TEST_UNSAT_DEP | H.HEDL_NO_GRAPH)
    assert e.value.code == -5
    compare_batch(small, dkb, progs, 0)


def test_bad_kb_rejected():
    import torch
    kb = K.generate(K.CONFIGS["small"].scaled(500, seed=4, n_roles=2))
    cases = {}
    col = kb.col[0].copy()
    k = int(np.nonzero(np.diff(kb.row_ptr[0].astype(np.int64)) >= 2)[0][0])
    s = int(kb.row_ptr[0][k])
    col[s], col[s + 1] = col[s + 1], col[s]
    cases["unsorted row"] = dict(col0=col)
    col = kb.col[0].copy()
    col[s + 1] = col[s]
    cases["duplicate assertion"] = dict(col0=col)
    col = kb.col[0].copy()
    col[0] = 500
    cases["id out of range"] = dict(col0=col)
    icol = kb.inv_col[0].copy()
    icol[[0, -1]] = icol[[-1, 0]]
    cases["not the transpose"] = dict(icol0=icol)
    cb = kb.concept_bits.copy()
    cb[0, kb.w - 1] |= np.uint32(1 << 31)
    cases["concept tail"] = dict(cb=cb)
    for what, ch in cases.items():
        cols = list(kb.col)
        icols = list(kb.inv_col)
        if "col0" in ch:
            cols[0] = ch["col0"]
        if "icol0" in ch:
            icols[0] = ch["icol0"]
        with pytest.raises(H.HedlError) as e:
            H.DeviceKB(kb.n, ch.get("cb", kb.concept_bits), kb.row_ptr, cols, kb.inv_row_ptr, icols, kb.prop_vals)
        assert e.value.code == -6, what


@pytest.fixture(scope="module")
def batch_kb():
    return K.generate(K.CONFIGS["batch"])


@pytest.mark.parametrize("stage,flags", [(1, 0), (0, 0), (1, 16)])
def test_batch_full_size_sampled(batch_kb, stage, flags):
    """Workload 3 at full size (N = 1,000,000) in the bench's launch configuration: a whole
    4,096-hypothesis batch on the GPU; 48 sampled hypotheses checked bit-exactly (sets and
    counts) against the oracle, and the counts of all against the plain path."""
    dkb = device_kb(batch_kb)
    H.hedl_tuning_set(dkb.handle, stage_fillers=stage)
    progs = hyps.batch_hyps(batch_kb, 1003, 0, 4096, gen=hyps.TreeGen(batch_kb, 1003, share=0.3))
    sample = sorted(set(list(range(8)) + list(range(0, 4096, 97)) + [4095]))
    counts, _ = compare_batch(batch_kb, dkb, progs, flags, sample=sample, check_bits=False)
    # instance sets of the sampled hypotheses, through eval (bench-shaped plan for the counts above)
    okb = oracle.from_synth(batch_kb)
    for h in sample[:12]:
        got = K.unpack_bits(dkb.eval(progs[h]), batch_kb.n)
        assert np.array_equal(got, oracle.eval_program(okb, progs[h])), h
    if stage and not flags:
        plain = dkb.score(*P.pack_batch(progs), H.HEDL_PLAIN)
        assert np.array_equal(plain, counts)
