"""The C-ABI library without a GPU: it loads, exports every declared symbol,
and its host-side logic (validation, planning) behaves (no compute calls)."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_2412_00802_gb300 as H
from synth import hyps, kb as K, programs as P
from synth.rng import Rng
from tests import oracle_pins as pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hedl.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_00802_gb300 import build
    build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hedl_\w+)\s*\(", src)))


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", H.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (hedl_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert sorted(H.SYMBOLS) == names
    lib = H.library()
    for n in names:
        assert getattr(lib, n) is not None


def test_op_codes_agree_with_the_format():
    hdr = open(HEADER).read()
    ops = dict((k, int(v)) for k, v in re.findall(r"HEDL_OP_(\w+)\s*=\s*(\d+)", hdr))
    for code, name in P.OP_NAMES.items():
        assert ops[name] == code
    src = open(os.path.join(os.path.dirname(oracle.__file__), "hedl_oracle.c")).read()
    for name, code in ops.items():
        assert getattr(P, name) == code
        assert re.search(rf"#define O_{name} {code}\b", src), name


def test_row_words():
    for n in (1, 31, 32, 33, 127, 128, 129, 10_000, 1_000_000):
        w = (n + 31) // 32
        assert H.hedl_row_words(n) == (w + 3) // 4 * 4


@pytest.fixture(scope="module")
def small():
    return K.generate(K.CONFIGS["small"])


def plan_kb(kb):
    return H.hedl_kb_plan_only(kb.n, kb.n_concepts, [kb.n_edges(r) for r in range(kb.n_roles)], kb.n_props)


def test_validation_agrees_with_the_oracle(small):
    """Accept / reject decisions match the oracle's on malformed programs."""
    hk = plan_kb(small)
    okb = oracle.from_synth(small)
    r = np.random.default_rng(3)
    good = hyps.small_hyps(small, 5, 30)
    cases = []
    for g in good:
        cases.append(g)
        g = g.copy()
        i = r.integers(len(g))
        kind = r.integers(5)
        if kind == 0:
            g[i] = (int(g[i]) & ~0xFF) | int(r.integers(15, 256))        # bad op
        elif kind == 1:
            g = g[:-1] if len(g) > 1 else g[:0]                            # truncated
        elif kind == 2:
            g = np.concatenate([g, g])                                    # two values left
        elif kind == 3:
            g[i] = P.insn(P.ATOM, 0, 50)                                  # id out of range
        else:
            g = np.concatenate([g, [P.insn(P.AND)]])                      # underflow
        cases.append(g)
    cases += [np.array([P.insn(P.ATOM, 0, 0)] * 65 + [P.insn(P.AND)] * 64, np.uint64),
              np.array([P.insn(P.ATOM, 0, 0)] * 64 + [P.insn(P.AND)] * 63, np.uint64),
              np.array([P.insn(P.EXISTS, 1, 8)], np.uint64), np.array([P.insn(P.DGE, 0, 4, 0)], np.uint64),
              np.zeros(0, np.uint64)]
    for c in cases:
        want_ok = oracle.validate(okb, c) == 0
        try:
            H.hedl_validate(hk, c)
            got_ok = True
        except H.HedlError as e:
            assert e.code == -2
            got_ok = False
        assert got_ok == want_ok, P.to_text(P.from_postfix(c)) if want_ok else c


def test_plan_batch_rejects_and_names_the_program(small):
    hk = plan_kb(small)
    progs = hyps.small_hyps(small, 5, 10)
    progs[7] = np.array([P.insn(P.AND)], np.uint64)
    flat, offs = P.pack_batch(progs)
    with pytest.raises(H.HedlError) as e:
        H.hedl_plan_batch(hk, flat, offs)
    assert "program 7" in str(e.value)
    # a string restriction naming a pattern the handle does not hold
    sk = H.hedl_kb_plan_only(small.n, small.n_concepts, [small.n_edges(r) for r in range(small.n_roles)],
                             small.n_props, str_role_vals=[10], n_strings=5, n_patterns=2)
    progs = [P.compile_text("(contains s0 1)"), P.compile_text("(and A0 (contains s0 2))")]
    with pytest.raises(H.HedlError) as e:
        H.hedl_plan_batch(sk, *P.pack_batch(progs))
    assert "program 1" in str(e.value) and "pattern 2" in str(e.value)


def test_plan_sharing_and_levels(small):
    hk = plan_kb(small)
    x = "(and A1 (some r2 (min 2 r3- (or A4 (le p1 20)))))"
    progs = [P.compile_text(x)] * 10 + [P.compile_text(f"(or A{i} {x})") for i in range(5)]
    flat, offs = P.pack_batch(progs)
    shared = H.hedl_plan_info_get(H.hedl_plan_batch(hk, flat, offs))
    plain = H.hedl_plan_info_get(H.hedl_plan_batch(hk, flat, offs, H.HEDL_NO_CSE))
    # two role restrictions in x, evaluated once with sharing
    assert shared["n_role_ops"] == 2 and plain["n_role_ops"] == 30
    # every restriction bit-sliced: filler 0, the min-restriction's transpose 1 and walk 2,
    # the some-restriction's transpose 3 and walk 4, the roots 5 (the shared conjunction
    # is inlined: its role restriction is already a slot)
    every = H.hedl_plan_info_get(H.hedl_plan_batch(hk, flat, offs, H.HEDL_SLICE_ALL))
    assert every["n_levels"] == 6 and every["n_role_groups"] == 2
    # one walk per restriction: filler, the min-restriction, the shared conjunction
    # (materialized, it holds a role restriction), the roots.  By default too: the two
    # restrictions differ in role, so neither has a partner to share a walk with.
    solo = H.hedl_plan_info_get(H.hedl_plan_batch(hk, flat, offs, H.HEDL_NO_SLICE))
    assert solo["n_levels"] == 4 and solo["n_role_groups"] == 0 and solo["n_role_ops"] == 2
    assert (shared["n_levels"], shared["n_role_groups"]) == (4, 0)
    assert shared["n_nodes"] < plain["n_nodes"]
    assert shared["model_bytes"] < plain["model_bytes"]
    # two restrictions of one role and direction at the same depth share a walk; at
    # different depths, or with different directions, they do not
    def groups(texts, flags=0):
        return H.hedl_plan_info_get(H.hedl_plan_batch(hk, *P.pack_batch([P.compile_text(t) for t in texts]),
                                                       flags))["n_role_groups"]
    assert groups(["(some r1 A2)", "(all r1 A3)"]) == 1
    assert groups(["(some r1 A2)", "(some r1- A3)"]) == 0
    assert groups(["(some r1 A2)", "(some r1 (some r2 A3))"]) == 0
    assert groups(["(some r1 A2)", "(some r1 (some r2 A3))"], H.HEDL_SLICE_ALL) == 3
    assert groups(["(some r1 A2)", "(some r1 (some r1 A3))"]) == 1     # the two inner ones
    assert groups(["(some r1 A2)", "(all r1 A3)"], H.HEDL_NO_SLICE | H.HEDL_SLICE_ALL) == 0
    # commuted operands and double negation share too
    a = [P.compile_text("(and A1 (some r0 A2))"), P.compile_text("(and (some r0 A2) A1)"),
         P.compile_text("(not (not (and A1 (some r0 A2))))")]
    i = H.hedl_plan_info_get(H.hedl_plan_batch(hk, *P.pack_batch(a)))
    assert i["n_role_ops"] == 1


def test_workspace_accounts_for_slots(small):
    hk = plan_kb(small)
    progs = hyps.batch_hyps(small, 9, 0, 200)
    flat, offs = P.pack_batch(progs)
    info = H.hedl_plan_info_get(H.hedl_plan_batch(hk, flat, offs))
    assert info["workspace_bytes"] >= info["n_slots"] * 4 * small.wp
    assert info["n_items"] == info["n_segments"] * -(-small.wp // info["tile_words"])


def test_planning_only_handle_refuses_launches(small):
    hk = plan_kb(small)
    with pytest.raises(H.HedlError) as e:
        H.hedl_sync_status(hk, stream=0)
    assert e.value.code == -1


def test_narrow_tiles_for_single_hypotheses():
    """A lone hypothesis's walks would leave most warps idle with 32-word warps: the plan
    narrows them (one round per item); a large batch keeps 32.  Role groups keep 32."""
    hk = H.hedl_kb_plan_only(1_000_000, 200, [8_000_000] * 32, 16)   # sizes only
    one = H.hedl_plan_info_get(H.hedl_plan_batch(hk, *P.pack_batch([P.compile_text("(some r1 (min 2 r2 A3))")])))
    assert one["warp_words"] == 4 and one["tile_words"] == 8 * 4
    batch = [P.compile_text(f"(some r{i % 8} (min 2 r{(i + 3) % 8} A{i % 50}))") for i in range(2000)]
    many = H.hedl_plan_info_get(H.hedl_plan_batch(hk, *P.pack_batch(batch)))
    assert many["warp_words"] == 32
    paired = H.hedl_plan_info_get(H.hedl_plan_batch(hk, *P.pack_batch([P.compile_text("(some r1 A2)"),
                                                                         P.compile_text("(all r1 A3)")])))
    assert paired["n_role_groups"] == 1 and paired["warp_words"] == 32


def test_canonical_batch_agrees_with_the_search_oracle(small):
    """The library's canonical form equals the independently written one of the search oracle."""
    from oracle import search as OS
    r = Rng(17, 4)
    progs = [np.array(pins.random_program(r, small, r.randint(1, 7)).postfix(), np.uint64) for _ in range(400)]
    progs += [P.compile_text("(and (or A2 A1) (or A1 A2))"), P.compile_text("(and A1 A1)"), P.compile_text("TOP")]
    flat, offs = P.pack_batch(progs)
    got = H.hedl_canonical_batch(flat, offs)
    for i, p in enumerate(progs):
        assert got[offs[i]:offs[i + 1]].tobytes() == OS.canonical(p), i
    with pytest.raises(H.HedlError):
        H.hedl_canonical_batch(np.array([P.insn(P.AND)], np.uint64), np.array([0, 1], np.uint32))


def test_interpreter_digest_ignores_comments_not_code():
    from paper_2412_00802_gb300 import build
    assert build._code_only('int a = 1; // note\n/* block\n comment */ int b = "x//y" [0];') == \
        'int a = 1; int b = "x//y" [0];'
    assert build._code_only("x  =\n\n y;") == "x = y;"
    assert build._code_only("a = 1;") != build._code_only("a = 2;")


def test_numeric_roles_on_a_planning_handle():
    """Numeric concrete roles take the property ids after the one-value properties; a restriction
    on one costs its row pointers and values in the byte model (4(N+1) + 4M, Algorithms 9-10)."""
    n, M = 10_000, [30_000, 5]
    hk = H.hedl_kb_plan_only(n, 3, [100], 2, num_role_vals=M)
    insn = lambda p: np.array([P.insn(P.DGE, 0, p, P.f32_bits(1.5))], np.uint64)
    for p in (0, 1, 2, 3):
        H.hedl_validate(hk, insn(p))
    with pytest.raises(H.HedlError) as e:
        H.hedl_validate(hk, insn(4))
    assert e.value.code == -2   # HEDL_ERR_BAD_PROGRAM
    B = 4 * H.hedl_row_words(n)
    for flags in (0, H.HEDL_PLAIN):
        for p, want in ((1, 4 * n), (2, 4 * (n + 1) + 4 * M[0]), (3, 4 * (n + 1) + 4 * M[1])):
            info = H.hedl_plan_info_get(H.hedl_plan_batch(hk, insn(p), np.array([0, 1], np.uint32), flags))
            assert info["n_data_ops"] == 1
            assert info["model_bytes"] == want + 2 * B + 16, (flags, p)


def test_numeric_role_limits():
    with pytest.raises(H.HedlError) as e:
        H.hedl_kb_plan_only(100, 1, [], 65_000, num_role_vals=[1] * 537)
    assert e.value.code == -1   # HEDL_ERR_INVALID_ARG
    with pytest.raises(H.HedlError) as e:
        H.hedl_kb_plan_only(100, 1, [], 0, num_role_vals=[1 << 31])
    assert e.value.code == -1   # HEDL_ERR_INVALID_ARG
    H.hedl_kb_plan_only(100, 1, [], 65_000, num_role_vals=[1] * 536)


def test_string_roles_on_a_planning_handle():
    """String restrictions name a string role below n_str_roles; SCONTAINS a pattern below
    n_patterns; SEQ any string id.  Byte model: 4(N+1) + 4M, plus the pattern's bitmap row."""
    n, M, S = 10_000, [20_000, 7], 1000
    hk = H.hedl_kb_plan_only(n, 3, [100], 1, str_role_vals=M, n_strings=S, n_patterns=4)
    one = lambda op, a, b: np.array([P.insn(op, 0, a, b)], np.uint64)
    for op, a, b in ((P.SEQ, 0, 5), (P.SEQ, 1, 0xFFFFFFFF), (P.SCONTAINS, 1, 3)):
        H.hedl_validate(hk, one(op, a, b))
    for op, a, b in ((P.SEQ, 2, 0), (P.SCONTAINS, 0, 4), (P.SCONTAINS, 2, 0)):
        with pytest.raises(H.HedlError) as e:
            H.hedl_validate(hk, one(op, a, b))
        assert e.value.code == -2, (op, a, b)
    B = 4 * H.hedl_row_words(n)
    for flags in (0, H.HEDL_PLAIN):
        for op, a, want in ((P.SEQ, 0, 4 * (n + 1) + 4 * M[0]), (P.SCONTAINS, 1, 4 * (n + 1) + 4 * M[1] + 4 * 32)):
            info = H.hedl_plan_info_get(H.hedl_plan_batch(hk, one(op, a, 1), np.array([0, 1], np.uint32), flags))
            assert info["n_data_ops"] == 1
            assert info["model_bytes"] == want + 2 * B + 16, (flags, op)
    with pytest.raises(H.HedlError) as e:
        H.hedl_kb_plan_only(100, 1, [], 0, str_role_vals=[1] * 65537, n_strings=1)
    assert e.value.code == -1
    with pytest.raises(H.HedlError) as e:     # values but no table
        H.hedl_kb_plan_only(100, 1, [], 0, str_role_vals=[3], n_strings=0)
    assert e.value.code == -1


def test_canonical_form_keeps_string_leaves():
    progs = [P.compile_text("(or (contains s1 2) (seq s0 7))"), P.compile_text("(or (seq s0 7) (contains s1 2))")]
    flat, offs = P.pack_batch(progs)
    got = H.hedl_canonical_batch(flat, offs)
    assert got[offs[0]:offs[1]].tobytes() == got[offs[1]:offs[2]].tobytes()


def test_header_is_plain_c(tmp_path):
    """include/hedl.h compiles as C99 with every warning on, and a C program links against the
    library through it (no torch or C++ types in the boundary)."""
    src = tmp_path / "use.c"
    src.write_text('#include "hedl.h"\n#include <stdio.h>\n'
                   "int main(void) { hedl_kb_desc d = {0}; hedl_kb *kb = 0; d.n_indiv = 1000;\n"
                   "  int rc = hedl_kb_plan_only(&d, &kb); printf(\"%d %u\\n\", rc, hedl_row_words(1000));\n"
                   "  hedl_kb_free(kb); return rc; }\n")
    exe = tmp_path / "use"
    libdir = os.path.dirname(H.LIB_PATH)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                           os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lhedl",
                           f"-Wl,-rpath,{libdir}"])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.split() == ["0", "32"], out


def test_planner_accepts_every_construct_in_every_mode():
    """Random batches over every constructor (numeric and string roles included), plus a
    600-instruction chain and a 64-leaf balanced tree, plan in every mode: the planner keeps each
    segment within the device stack by materialising, never fails on a valid program."""
    kb = K.generate(K.CONFIGS["small"].scaled(3000, seed=5, n_num_roles=2, n_str_roles=2, n_strings=50,
                                              n_patterns=6))
    hk = H.hedl_kb_plan_only(kb.n, kb.n_concepts, [kb.n_edges(r) for r in range(kb.n_roles)], kb.n_props,
                             num_role_vals=[v.size for v in kb.num_vals],
                             str_role_vals=[v.size for v in kb.str_ids], n_strings=len(kb.strings),
                             n_patterns=kb.n_patterns)
    r = Rng(77, 1)
    modes = [0, H.HEDL_NO_CSE, H.HEDL_NO_SLICE, H.HEDL_SLICE_ALL, H.HEDL_PLAIN, H.HEDL_LEVELS,
             H.HEDL_NO_CSE | H.HEDL_NO_SLICE]
    for it in range(40):
        progs = [np.array(pins.random_program(r, kb, r.randint(1, 9)).postfix(), np.uint64)
                 for _ in range(r.randint(1, 60))]
        if it % 10 == 0:
            d = 300
            progs.append(np.array([P.insn(P.ATOM, 0, 0)] + [x for i in range(d) for x in (
                P.insn(P.ATOM, 0, i % kb.n_concepts), P.insn(P.AND if i % 2 else P.OR))], np.uint64))
            progs.append(np.array([P.insn(P.ATOM, 0, i % kb.n_concepts) for i in range(64)] + [P.insn(P.AND)] * 63,
                                  np.uint64))
        flat, offs = P.pack_batch(progs)
        for f in modes:
            info = H.hedl_plan_info_get(H.hedl_plan_batch(hk, flat, offs, f))
            assert info["n_hyps"] == len(progs)


@pytest.mark.parametrize("n", [3000, 1_000_000])
def test_no_sharing_plans_have_a_data_parallel_formulation(n):
    """The plan image of a batch planned without sharing or bit slicing equals, byte for byte, the
    one written by a formulation whose steps are independent per hypothesis or prefix sums, a stable
    sort and a reduction (tests/plan_model.py): the shape of a device-side planner.  Workspace size
    and algorithmic bytes agree too.  Random batches over every construct, deep chains that force
    materialisation, narrow and full-width tiles."""
    from tests import plan_model as M
    kb = K.generate(K.CONFIGS["small"].scaled(3000, seed=5, n_num_roles=2, n_str_roles=2, n_strings=50,
                                              n_patterns=6))
    w = (n + 31) // 32
    sizes = dict(n=n, wp=(w + 3) // 4 * 4, n_props=kb.n_props, num_vals=[v.size for v in kb.num_vals],
                 str_vals=[v.size for v in kb.str_ids], contain_words=(len(kb.strings) + 31) // 32,
                 role_edges=[kb.n_edges(r) for r in range(kb.n_roles)])
    hk = H.hedl_kb_plan_only(n, kb.n_concepts, sizes["role_edges"], kb.n_props, num_role_vals=sizes["num_vals"],
                             str_role_vals=sizes["str_vals"], n_strings=len(kb.strings), n_patterns=kb.n_patterns)
    F = H.HEDL_NO_CSE | H.HEDL_NO_SLICE
    r = Rng(99, 3)
    for it in range(60):
        progs = [np.array(pins.random_program(r, kb, r.randint(1, 9)).postfix(), np.uint64)
                 for _ in range(r.randint(1, 80))]
        if it % 7 == 0:
            progs.append(np.array([P.insn(P.ATOM, 0, 0)] + [x for i in range(200) for x in (
                P.insn(P.ATOM, 0, i % kb.n_concepts), P.insn(P.AND if i % 2 else P.OR))], np.uint64))
        if it % 5 == 0:
            progs += hyps.small_hyps(kb, it, 50)
        flat, offs = P.pack_batch(progs)
        pl = H.hedl_plan_batch(hk, flat, offs, F)
        info = H.hedl_plan_info_get(pl)
        img, ws, model = M.plan_image(progs, sizes, F)
        assert np.array_equal(H.hedl_plan_image(pl), img), it
        assert (ws, model) == (info["workspace_bytes"], info["model_bytes"]), it
    import ctypes
    size = ctypes.c_size_t(0)
    buf = np.zeros(16, np.uint8)   # a buffer too small is refused, with the size reported
    assert H.library().hedl_plan_image(pl.ptr, buf.ctypes.data, buf.size, ctypes.byref(size)) == -1
    assert size.value == info["image_bytes"]


@pytest.mark.parametrize("n,stage", [(3000, 0), (1_000_000, 0), (3000, 1), (1_000_000, 1)])
def test_parallel_planner_equals_the_host_planner(n, stage):
    """hedl_plan_batch_parallel (per-hypothesis steps on host threads, the paper's parallel plan
    generation) gives the same plan as hedl_plan_batch with HEDL_NO_CSE | HEDL_NO_SLICE: image byte
    for byte and every field of the plan info, with and without HEDL_LEVELS, on 1 to 4 threads, with
    role fillers staged in shared memory (one role restriction per segment) or not."""
    kb = K.generate(K.CONFIGS["small"].scaled(3000, seed=5, n_num_roles=2, n_str_roles=2, n_strings=50,
                                              n_patterns=6))
    hk = H.hedl_kb_plan_only(n, kb.n_concepts, [kb.n_edges(r) for r in range(kb.n_roles)], kb.n_props,
                             num_role_vals=[v.size for v in kb.num_vals], str_role_vals=[v.size for v in kb.str_ids],
                             n_strings=len(kb.strings), n_patterns=kb.n_patterns)
    H.hedl_tuning_set(hk, stage_fillers=stage)
    F = H.HEDL_NO_CSE | H.HEDL_NO_SLICE
    r = Rng(5, 9)
    for it in range(40):
        progs = [np.array(pins.random_program(r, kb, r.randint(1, 9)).postfix(), np.uint64)
                 for _ in range(r.randint(1, 80))]
        if it % 7 == 0:
            progs.append(np.array([P.insn(P.ATOM, 0, 0)] + [x for i in range(250) for x in (
                P.insn(P.ATOM, 0, i % kb.n_concepts), P.insn(P.AND if i % 2 else P.OR))], np.uint64))
        if it % 5 == 0:
            progs += hyps.small_hyps(kb, it, 50)
        flat, offs = P.pack_batch(progs)
        for extra in (0, H.HEDL_LEVELS):
            a = H.hedl_plan_batch(hk, flat, offs, F | extra)
            b = H.hedl_plan_batch_parallel(hk, flat, offs, F | extra, n_threads=1 + it % 4)
            assert np.array_equal(H.hedl_plan_image(a), H.hedl_plan_image(b)), (it, extra)
            assert H.hedl_plan_info_get(a) == H.hedl_plan_info_get(b), (it, extra)
    progs = hyps.small_hyps(kb, 1, 10)
    progs[6] = np.array([P.insn(P.OR)], np.uint64)
    with pytest.raises(H.HedlError) as e:
        H.hedl_plan_batch_parallel(hk, *P.pack_batch(progs), n_threads=3)
    assert e.value.code == -2 and "program 6" in str(e.value)
    for bad_flags in (H.HEDL_PLAIN, H.HEDL_SLICE_ALL):
        with pytest.raises(H.HedlError) as e:
            H.hedl_plan_batch_parallel(hk, *P.pack_batch(progs[:3]), bad_flags)
        assert e.value.code == -1
    if n == 3000 and not stage:
        # A chain of nested restrictions makes one dependency level per link.  The sort key holds
        # 14 bits of level: 16,000 links still plan identically, 17,000 are refused by the
        # per-hypothesis planner (not mis-sorted) and still planned by the host planner.
        for links, ok in ((16_000, True), (17_000, False)):
            chain = [P.insn(P.ATOM, 0, 1)] + [P.insn(P.EXISTS, 0, 0)] * links
            batch = P.pack_batch([np.array(chain, np.uint64)] + progs[:3])
            a = H.hedl_plan_batch(hk, *batch, F)
            assert H.hedl_plan_info_get(a)["n_levels"] >= links
            if ok:
                b = H.hedl_plan_batch_parallel(hk, *batch, F, n_threads=2)
                assert np.array_equal(H.hedl_plan_image(a), H.hedl_plan_image(b))
            else:
                with pytest.raises(H.HedlError) as e:
                    H.hedl_plan_batch_parallel(hk, *batch, F, n_threads=2)
                assert e.value.code == -1 and "16,384 dependency levels" in str(e.value)
    if stage:   # staging split restrictions into more segments than without
        r2 = Rng(6, 1)
        progs = [np.array(pins.random_program(r2, kb, 6).postfix(), np.uint64) for _ in range(200)]
        staged = H.hedl_plan_info_get(H.hedl_plan_batch_parallel(hk, *P.pack_batch(progs), F))
        H.hedl_tuning_set(hk, stage_fillers=0)
        plain = H.hedl_plan_info_get(H.hedl_plan_batch_parallel(hk, *P.pack_batch(progs), F))
        assert staged["n_segments"] > plain["n_segments"]


def test_bitonic_step_sorts_on_the_host(tmp_path):
    """The device planner's sort is a bitonic network over the padded unique keys (the host driver
    uses std::sort): run the network's compare-exchange step on the host and check it sorts."""
    src = tmp_path / "bitonic.cu"
    src.write_text('#include "devplan.cu"\n#include <algorithm>\n#include <cstdio>\n#include <random>\n'
                   "int main() {\n"
                   "  std::mt19937_64 g(7);\n"
                   "  for (uint64_t n : {1ull, 2ull, 3ull, 5ull, 100ull, 1000ull, 4099ull}) {\n"
                   "    const uint64_t n2 = hedl::dp::pow2_at_least(n);\n"
                   "    std::vector<uint64_t> k(n2, ~0ull), ref(n);\n"
                   "    for (uint64_t i = 0; i < n; ++i) ref[i] = k[i] = (g() >> 8) << 8 | (i & 255);\n"
                   "    for (uint64_t kk = 2; kk <= n2; kk <<= 1)\n"
                   "      for (uint64_t j = kk >> 1; j > 0; j >>= 1)\n"
                   "        for (uint64_t i = 0; i < n2; ++i) hedl::dp::bitonic_step(k.data(), i, j, kk);\n"
                   "    std::sort(ref.begin(), ref.end());\n"
                   "    for (uint64_t i = 0; i < n; ++i) if (k[i] != ref[i]) { printf(\"bad %llu\\n\", (unsigned long long)n); return 1; }\n"
                   "  }\n  printf(\"ok\\n\");\n  return 0;\n}\n")
    exe = tmp_path / "bitonic"
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    libdir = os.path.dirname(H.LIB_PATH)
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I",
                           os.path.join(ROOT, "paper_2412_00802_gb300", "csrc"), str(src), "-o", str(exe),
                           "-L", libdir, "-lhedl", "-Xlinker", f"-rpath={libdir}"])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out


def test_device_validation_agrees_with_the_host(tmp_path):
    """The device planner validates programs with dp::validate (codes, no messages); on random and
    malformed programs it decides as hedl_validate does (run on the host through the library)."""
    src = tmp_path / "validate.cu"
    src.write_text('#include "devplan.cu"\n#include <cstdio>\n#include <random>\n'
                   "int main() {\n"
                   "  hedl_csr roles[3] = {{0, 0, 10}, {0, 0, 10}, {0, 0, 10}};\n"
                   "  hedl_numeric_role nums[2] = {{0, 0, 5}, {0, 0, 5}};\n"
                   "  hedl_string_role strs[2] = {{0, 0, 5}, {0, 0, 5}};\n"
                   "  hedl_kb_desc d = {0};\n"
                   "  d.n_indiv = 1000; d.n_concepts = 7; d.n_roles = 3; d.roles = roles; d.inv_roles = roles;\n"
                   "  d.n_props = 2; d.n_num_roles = 2; d.num_roles = nums; d.n_str_roles = 2; d.str_roles = strs;\n"
                   "  d.n_strings = 9; d.n_patterns = 4;\n"
                   "  hedl_kb *kb = 0; if (hedl_kb_plan_only(&d, &kb)) return 2;\n"
                   "  std::mt19937_64 g(11); int agree = 0, bad = 0;\n"
                   "  for (int it = 0; it < 20000; ++it) {\n"
                   "    std::vector<uint64_t> p(1 + g() % 12);\n"
                   "    for (auto &w : p) {\n"
                   "      const uint64_t op = 1 + g() % 17, a = g() % 9, b = g() % 6;\n"
                   "      w = op | ((g() % 2) << 8) | (a << 16) | (b << 32);\n"
                   "    }\n"
                   "    const uint32_t offs[2] = {0, (uint32_t)p.size()};\n"
                   "    hedl::dp::Ctx c{}; c.progs = p.data(); c.offs = offs; c.H = 1;\n"
                   "    c.n_concepts = 7; c.n_roles = 3; c.n_data = 4; c.n_str = 2; c.n_patterns = 4;\n"
                   "    const bool dev = hedl::dp::validate(c, 0, (uint32_t)p.size()) == 0;\n"
                   "    const bool host = hedl_validate(kb, p.data(), (uint32_t)p.size()) == 0;\n"
                   "    if (dev != host) { if (++bad < 4) printf(\"disagree at %d\\n\", it); } else agree += dev;\n"
                   "  }\n"
                   "  // the stack limit's edge: 64 operands on the stack are legal, 65 are not, both ways\n"
                   "  for (int depth = 63; depth <= 66; ++depth) {\n"
                   "    std::vector<uint64_t> p;\n"
                   "    for (int i = 0; i < depth; ++i) p.push_back(1 | (uint64_t)(i % 7) << 16);\n"
                   "    for (int i = 1; i < depth; ++i) p.push_back(5);\n"
                   "    const uint32_t offs[2] = {0, (uint32_t)p.size()};\n"
                   "    hedl::dp::Ctx c{}; c.progs = p.data(); c.offs = offs; c.H = 1;\n"
                   "    c.n_concepts = 7; c.n_roles = 3; c.n_data = 4; c.n_str = 2; c.n_patterns = 4;\n"
                   "    const bool dev = hedl::dp::validate(c, 0, (uint32_t)p.size()) == 0;\n"
                   "    const bool host = hedl_validate(kb, p.data(), (uint32_t)p.size()) == 0;\n"
                   "    if (dev != host || dev != (depth <= 64)) { ++bad; printf(\"depth %d: dev %d host %d\\n\", depth, dev, host); }\n"
                   "  }\n"
                   "  hedl_kb_free(kb);\n"
                   "  printf(bad ? \"bad\\n\" : \"ok %d\\n\", agree);\n  return bad ? 1 : 0;\n}\n")
    exe = tmp_path / "validate"
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    libdir = os.path.dirname(H.LIB_PATH)
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I",
                           os.path.join(ROOT, "paper_2412_00802_gb300", "csrc"), str(src), "-o", str(exe),
                           "-L", libdir, "-lhedl", "-Xlinker", f"-rpath={libdir}"])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out
    assert int(out.stdout.split()[1]) > 100   # some random programs are valid, so both branches are seen

@pytest.mark.parametrize("n", [3000, 641])
def test_plan_byte_model_equals_the_oracles_count(n):
    """The algorithmic bytes a plan reports (plan.cpp, devplan.cu) are the oracle's per-operation
    count, taken while it evaluates (oracle/hedl_oracle.c): equal, program by program summed,
    whenever nothing is shared (HEDL_NO_CSE, with or without bit slicing, per-level launches, the
    plain path, the per-hypothesis planner); with sharing the plan counts each common sub-concept
    once, so never more.  The plan-only handle has the sizes of the KB the oracle evaluates on."""
    import oracle
    kb = K.generate(K.CONFIGS["small"].scaled(n, seed=5, n_num_roles=2, n_str_roles=2,
                                              n_strings=50, n_patterns=6))
    okb = oracle.from_synth(kb)
    hk = H.hedl_kb_plan_only(kb.n, kb.n_concepts, [kb.n_edges(r) for r in range(kb.n_roles)], kb.n_props,
                             num_role_vals=[v.size for v in kb.num_vals], str_role_vals=[v.size for v in kb.str_ids],
                             n_strings=len(kb.strings), n_patterns=kb.n_patterns)
    r = Rng(31, n % 97)
    exact = [H.HEDL_NO_CSE, H.HEDL_NO_CSE | H.HEDL_NO_SLICE, H.HEDL_NO_CSE | H.HEDL_SLICE_ALL,
             H.HEDL_NO_CSE | H.HEDL_LEVELS, H.HEDL_PLAIN]
    for it in range(12):
        progs = [np.array(pins.random_program(r, kb, r.randint(1, 8)).postfix(), np.uint64)
                 for _ in range(r.randint(1, 60))]
        if it % 4 == 0:
            progs += hyps.small_hyps(kb, it, 30)
        flat, offs = P.pack_batch(progs)
        per = np.zeros(len(progs), np.int64)
        _, _, errs = oracle.eval_batch(okb, flat, offs, threads=4, bytes_out=per)
        assert not errs.any()
        want = int(per.sum())
        for f in exact:
            assert H.hedl_plan_info_get(H.hedl_plan_batch(hk, flat, offs, f))["model_bytes"] == want, (it, f)
        par = H.hedl_plan_batch_parallel(hk, flat, offs, H.HEDL_NO_CSE | H.HEDL_NO_SLICE, n_threads=2)
        assert H.hedl_plan_info_get(par)["model_bytes"] == want
        for f in (0, H.HEDL_NO_SLICE, H.HEDL_SLICE_ALL):
            assert H.hedl_plan_info_get(H.hedl_plan_batch(hk, flat, offs, f))["model_bytes"] <= want, (it, f)
